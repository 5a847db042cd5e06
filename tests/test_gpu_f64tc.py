"""FP64 form with the FD mode products on the BF16 tensor cores by exact integer slice
products (precision "fp64tc", IGA_PREC_FP64_TC; csrc/kernels_fd_f64tc.cu).

Each value is written as a power of two per row (per factor column) times eight base-2^7
digits; the digit products are summed exactly in FP32 and recombined exactly before one
rounding (error-free splitting, Ozaki et al. 2012).  The error of one product entry is below
13 K 2^-56 of its row/column scale -- an FP64 dot product's worst-case rounding (pinned on the
host in test_f64tc_scheme.py) -- so the FD must agree with the oracle's FP64 FD to the FP64
form's tolerance, GMRES must take the FP64 form's steps, and the solutions must agree to far
below the GMRES tolerance.  n <= 148 (beyond it a group sum could round).
"""

import numpy as np
import pytest
import torch

from tests.oracle_ref import ref

pytestmark = pytest.mark.gpu


def _problem(d, ne, p, precision, geometry="annulus"):
    from paper_1705_04384_gb300.api import Problem
    return Problem(d, ne, p, geometry=geometry, precision=precision)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# n = ne + p - 2: 1..3 K-chunks of 64, a partial last column tile, n = 148 (the limit)
@pytest.mark.parametrize("d,ne,p", [(2, 3, 2), (2, 40, 3), (2, 70, 5), (2, 147, 3), (3, 9, 3),
                                     (3, 20, 4), (3, 64, 3), (3, 30, 6)])
def test_f64tc_fd_matches_oracle_and_fp64_fd(d, ne, p):
    R = ref(d, ne, p, assemble=False)
    b = np.random.Generator(np.random.PCG64(21)).standard_normal(R.N)
    b[:: 7] *= 1e-6  # entries of very different size within a row
    want = R.fd(b)
    bt = torch.from_numpy(b).cuda()
    with _problem(d, ne, p, "fp64tc") as P:
        assert P.fd_kernel(1) == "fp64_slices"
        got = P.precond_apply(bt).cpu().numpy()
        got2 = P.precond_apply(bt).cpu().numpy()
    assert np.array_equal(got, got2)  # deterministic
    with _problem(d, ne, p, "fp64") as P:
        nat = P.precond_apply(bt).cpu().numpy()
    e_or, e_nat = _rel(got, want), _rel(got, nat)
    print(f"fp64tc FD d={d} ne={ne} p={p}: vs oracle {e_or:.2e}, vs FP64 FD {e_nat:.2e}, "
          f"FP64 FD vs oracle {_rel(nat, want):.2e}")
    assert e_or <= 1e-11, e_or  # the FP64 form's FD tolerance
    assert e_nat <= 1e-12, e_nat


def test_f64tc_fd_zero_and_scaled_inputs():
    """Zero rows give zero, and the slicing is scale-free: FD(2^k b) = 2^k FD(b) exactly
    (the row exponents absorb 2^k; the digits do not change)."""
    d, ne, p = 3, 12, 3
    R = ref(d, ne, p, assemble=False)
    b = np.random.Generator(np.random.PCG64(5)).standard_normal(R.N)
    with _problem(d, ne, p, "fp64tc") as P:
        z0 = P.precond_apply(torch.zeros(R.N, dtype=torch.float64, device="cuda"))
        assert torch.count_nonzero(z0).item() == 0
        z1 = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
        z2 = P.precond_apply(torch.from_numpy(b * 2.0 ** 40).cuda()).cpu().numpy()
        z3 = P.precond_apply(torch.from_numpy(b * 2.0 ** -70).cuda()).cpu().numpy()
    assert np.array_equal(z2, z1 * 2.0 ** 40)
    assert np.array_equal(z3, z1 * 2.0 ** -70)


@pytest.mark.parametrize("d,ne,p,geo", [(2, 32, 3, "annulus"), (2, 70, 5, "annulus"),
                                         (3, 10, 3, "annulus"), (3, 8, 4, "revolved")])
def test_f64tc_gmres_takes_the_fp64_steps(d, ne, p, geo):
    R = ref(d, ne, p, geo)
    b = R.manufactured_rhs(0.0) if geo == "annulus" else \
        np.random.Generator(np.random.PCG64(11)).standard_normal(R.N)
    o = R.gmres(b, tol=1e-8, max_iter=300)
    bt = torch.from_numpy(b).cuda()
    with _problem(d, ne, p, "fp64tc", geo) as P:
        x, info = P.solve(bt, tol=1e-8, max_iter=300)
        x = x.cpu().numpy()
    with _problem(d, ne, p, "fp64", geo) as P:
        x64, info64 = P.solve(bt, tol=1e-8, max_iter=300)
        x64 = x64.cpu().numpy()
    relres = np.linalg.norm(b - R.A @ x) / np.linalg.norm(b)
    assert info["status"] == 0 and relres <= 1.05e-8, relres
    assert abs(info["iters"] - o["iters"]) <= 1
    assert info["iters"] == info64["iters"]
    assert np.allclose(info["hist"], info64["hist"], rtol=1e-9, atol=0)
    assert _rel(x, x64) <= 1e-10


def test_f64tc_multi_rhs_bitwise_equals_single():
    R = ref(2, 30, 3)
    B = np.random.Generator(np.random.PCG64(17)).standard_normal((3, R.N))
    B[1] *= 1e-3
    with _problem(2, 30, 3, "fp64tc") as P:
        X, info = P.solve_multi(torch.from_numpy(B).cuda(), tol=1e-8, max_iter=200)
        X = X.cpu().numpy()
        for r in range(3):
            x1, i1 = P.solve(torch.from_numpy(B[r]).cuda(), tol=1e-8, max_iter=200)
            assert i1["iters"] == info["iters"][r]
            assert np.array_equal(x1.cpu().numpy(), X[r])


def test_f64tc_rejects_what_it_does_not_cover():
    from paper_1705_04384_gb300 import IgaError
    with pytest.raises(IgaError) as e:
        _problem(2, 148, 3, "fp64tc")  # n = 149: G_6 could round
    assert e.value.status == 8  # IGA_ERR_UNSUPPORTED
    from paper_1705_04384_gb300.api import Problem
    with pytest.raises(IgaError):
        Problem(2, 10, 3, wind=(1.0, 1.0), precision="fp64tc")


def test_f64tc_device_error_word():
    """A bounded wait that runs out is reported through the device error word (set from the
    host here; no wait is made to run out)."""
    from paper_1705_04384_gb300 import IgaError
    with _problem(2, 24, 3, "fp64tc") as P:
        b = torch.from_numpy(np.random.default_rng(3).standard_normal(P.N)).cuda()
        x0, i0 = P.solve(b, tol=1e-8, max_iter=100)
        x0 = x0.clone()
        P.test_set_device_error(13)
        with pytest.raises(IgaError) as e:
            P.solve(b, tol=1e-8, max_iter=100)
        assert e.value.status == 6
        x1, i1 = P.solve(b, tol=1e-8, max_iter=100)
        assert i1["iters"] == i0["iters"] and torch.equal(x1, x0)


def test_f64tc_full_size_3d_ne128():
    """The bench configuration (3D extruded annulus, 128 elements, p = 4, N = 2.197e6): the
    FP64_TC form against the FP64 form -- the same step count, solutions within 1e-10 --
    and the oracle's collocation rows at sampled points."""
    import workload as W
    R = ref(3, 128, 4, assemble=False)
    b = W.config_rhs("3d_annulus_ne128", R.points, p_index=0)
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([[0, R.N - 1], rng.integers(0, R.N, 24)]))
    rows = R.rows(idx)
    bt = torch.from_numpy(b).cuda()
    with _problem(3, 128, 4, "fp64tc") as P:
        x, info = P.solve(bt, tol=1e-8, max_iter=200)
        x = x.cpu().numpy()
    with _problem(3, 128, 4, "fp64") as P:
        x64, info64 = P.solve(bt, tol=1e-8, max_iter=200)
        x64 = x64.cpu().numpy()
    print(f"ne128 p=4 fp64tc: iters {info['iters']} (fp64 {info64['iters']}), "
          f"|x - x_fp64|/|x_fp64| = {_rel(x, x64):.2e}")
    assert info["status"] == 0 and info["relres_true"] <= 1.05e-8
    assert np.max(np.abs(b[idx] - rows @ x)) <= 1.05e-8 * np.linalg.norm(b)
    assert info["iters"] == info64["iters"]
    assert _rel(x, x64) <= 1e-10
