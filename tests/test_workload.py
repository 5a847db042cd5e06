"""The seeded synthetic workloads (workload/__init__.py): reproducible, and drawn from the
stated distributions (batched problems, the Poisson request stream, the perturbation)."""

import numpy as np

import workload as W


def test_batched_problems_ranges_and_reproducibility():
    a, b = W.batched_problems(), W.batched_problems()
    assert a == b and len(a) == 256
    ne = np.array([q["n_elem"] for q in a])
    p = np.array([q["p"] for q in a])
    r0 = np.array([q["r0"] for q in a])
    assert ne.min() >= 32 and ne.max() <= 512 and len(set(ne)) > 150
    assert set(p) == {2, 3, 4, 5, 6}
    assert r0.min() >= 0.5 and r0.max() <= 1.5
    assert all(q["r1"] == q["r0"] + 1.0 and q["nrhs"] == 8 and q["d"] == 2 for q in a)
    assert len({q["rhs_seed"] for q in a}) == 256
    assert W.batched_problems(seed=5) != a


def test_served_stream_is_poisson_with_the_stated_mix():
    reqs = W.served_requests(rate=2000.0, duration=10.0)
    assert reqs == W.served_requests(rate=2000.0, duration=10.0)
    n = len(reqs)
    assert abs(n - 20000) < 4 * np.sqrt(20000)  # Poisson count, mean rate x duration
    t = np.array([r["t_arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and t[-1] <= 10.0
    assert abs(gaps.mean() - 1 / 2000) < 4 * (1 / 2000) / np.sqrt(n)
    # exponential gaps: coefficient of variation 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    d2 = [r for r in reqs if r["d"] == 2]
    d3 = [r for r in reqs if r["d"] == 3]
    assert abs(len(d2) / n - 0.5) < 4 * 0.5 / np.sqrt(n)
    assert min(r["n_elem"] for r in d2) >= 64 and max(r["n_elem"] for r in d2) <= 1024
    assert min(r["n_elem"] for r in d3) >= 32 and max(r["n_elem"] for r in d3) <= 160
    assert {r["p"] for r in d2} == {2, 3, 4, 5, 6} and {r["p"] for r in d3} == {3, 4, 5, 6}


def test_perturbation_is_additive_and_seeded():
    f = np.linspace(-2.0, 3.0, 1000)
    g = W.perturb(f, 1e-3, seed=0)
    z = (g - f) / (1e-3 * 3.0)
    assert np.allclose(z, np.random.Generator(np.random.PCG64(0)).standard_normal(1000))
    assert np.array_equal(W.perturb(f, 0.0), f)
    assert not np.array_equal(W.perturb(f, 1e-3, seed=1), g)


def test_gaussian_rhs_shape_and_seed():
    B = W.gaussian_rhs(1000, 8, seed=4)
    assert B.shape == (8, 1000)
    assert np.array_equal(B, W.gaussian_rhs(1000, 8, seed=4))
    assert abs(B.mean()) < 0.05 and abs(B.std() - 1.0) < 0.05


def test_dofs():
    assert W.dofs(3, 64, 3) == 274625 and W.dofs(2, 32, 3) == 1089
