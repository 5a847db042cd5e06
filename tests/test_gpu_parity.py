"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances, each derived from the arithmetic it covers:
* 1D factors, points: exact up to a few ulps (same formulas, different code);
* operator: max |A_gpu u - A_oracle u| <= 1e-13 max |A_oracle u| (FP64 sums of <= 9
  terms of W products; reordering error ~ 1e-15, margin for cancellation);
* FD solve: ||s_gpu - s_oracle|| <= 1e-11 ||s_oracle|| (cond(U) <= 15 amplifies the
  FP64 rounding of 2d mode products);
* GMRES iterate at fixed k: relative difference <= 1e-10;
* GMRES to tol 1e-8: iteration counts within +-1, true residual <= 1e-8.
"""

import os

import numpy as np
import pytest
import torch

from tests.oracle_ref import ref

pytestmark = pytest.mark.gpu

CASES_OP = [
    (2, 40, 3, "annulus"), (2, 23, 2, "annulus"), (2, 17, 5, "annulus"), (2, 30, 6, "annulus"),
    (2, 19, 4, "identity"), (3, 8, 4, "annulus"), (3, 9, 3, "annulus"), (3, 6, 3, "revolved"),
    (3, 7, 5, "identity"), (3, 11, 2, "annulus"), (3, 5, 6, "revolved"),
]


def _problem(d, ne, p, geometry="annulus", precision="fp64", r0=1.0, r1=2.0):
    from paper_1705_04384_gb300.api import Problem
    return Problem(d, ne, p, geometry=geometry, r_inner=r0, r_outer=r1, precision=precision)


def _rand(N, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(N)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_factors_match_oracle(p):
    R = ref(2, 21, p, assemble=False)
    with _problem(2, 21, p) as P:
        s = R.spaces[0]
        assert np.max(np.abs(P.factor("tau") - s.tau)) <= 2e-16
        assert np.max(np.abs(P.factor("M") - s.M)) <= 1e-14
        assert np.max(np.abs(P.factor("B1") - s.B[1])) <= 1e-12
        assert np.max(np.abs(P.factor("K") - s.K)) <= 1e-10 * np.max(np.abs(s.K))
        lam = P.factor("lambda")
        assert np.max(np.abs(lam - R.fd.lam[0]) / np.abs(R.fd.lam[0])) <= 1e-9
        U, Uo, Vt = P.factor("U"), R.fd.U[0], P.factor("Vt")
        # eq. (eigendecomposition) holds for the GPU factors, and V^T = (M U)^{-1}
        assert np.max(np.abs(s.K @ U - s.M @ U * lam)) <= 1e-10 * np.max(np.abs(s.K))
        assert np.max(np.abs(Vt @ (s.M @ U) - np.eye(R.n))) <= 1e-10
        # columns agree with LAPACK's up to sign where the eigenvalue is well separated;
        # the near-double outlier pair of Remark 1 is fixed only up to ~eps/gap.
        gap = np.array([np.min(np.abs(np.delete(lam, j) - lam[j])) / lam[j] for j in range(R.n)])
        sign = np.sign(np.sum(U * Uo, axis=0))
        ok = gap > 1e-4
        assert np.max(np.abs(U * sign - Uo)[:, ok]) <= 1e-8
        assert np.max(np.abs(Vt * sign[:, None] - R.fd.V[0].T)[ok, :]) <= 1e-8 * np.max(np.abs(Vt))


@pytest.mark.parametrize("d,ne,p,geo", [(2, 12, 3, "annulus"), (3, 5, 4, "annulus"),
                                         (3, 4, 3, "revolved"), (2, 9, 2, "identity")])
def test_collocation_points_match_oracle(d, ne, p, geo):
    R = ref(d, ne, p, geo, assemble=False)
    with _problem(d, ne, p, geo) as P:
        assert np.max(np.abs(P.collocation_points() - R.points)) <= 1e-14


@pytest.mark.parametrize("d,ne,p,geo", CASES_OP)
def test_operator_matches_oracle(d, ne, p, geo):
    R = ref(d, ne, p, geo)
    with _problem(d, ne, p, geo) as P:
        for seed in (0, 1):
            u = _rand(R.N, seed)
            got = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
            want = R.A @ u
            assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_operator_ragged_annulus_radii():
    R = ref(2, 37, 4, "annulus", 0.5, 1.5)
    with _problem(2, 37, 4, "annulus", r0=0.5, r1=1.5) as P:
        u = _rand(R.N, 3)
        got = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
        want = R.A @ u
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("d,ne,p", [(2, 40, 3), (2, 95, 5), (2, 150, 2), (3, 9, 3), (3, 14, 6),
                                     (3, 20, 4),
                                     # every branch of the FP64 FD kernel's work split: blocks
                                     # shorter than one k-step (n = 3, 4), a partial last group
                                     # of 4 columns (n = 8), exact 8-column groups (n = 16, 256),
                                     # a 1-column partial group on FMAs (n = 130) and one past the
                                     # FMA length limit, padded (n = 259)
                                     (2, 3, 2), (3, 3, 3), (3, 5, 5), (2, 14, 4), (2, 255, 3),
                                     (2, 130, 2), (2, 258, 3)])
def test_fd_matches_oracle(d, ne, p):
    R = ref(d, ne, p, assemble=False)
    with _problem(d, ne, p) as P:
        b = _rand(R.N, 7)
        got = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
        want = R.fd(b)
        assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)
        assert np.linalg.norm(R.P_apply(got) - b) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("d,ne,p,k", [(2, 24, 3, 1), (2, 24, 3, 4), (2, 24, 3, 12),
                                       (3, 8, 3, 6), (2, 60, 4, 9), (3, 13, 5, 5)])
def test_gmres_iterate_at_fixed_k_matches(d, ne, p, k):
    R = ref(d, ne, p)
    b = R.manufactured_rhs(1e-3, 0)
    o = R.gmres(b, tol=0.0, max_iter=k)
    with _problem(d, ne, p) as P:
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=0.0, max_iter=k)
        x = x.cpu().numpy()
    assert info["iters"] == k == o["iters"]
    assert np.linalg.norm(x - o["x"]) <= 1e-10 * np.linalg.norm(o["x"])
    assert np.max(np.abs(info["hist"] - o["hist"]) / o["hist"]) <= 1e-8


@pytest.mark.parametrize("d,ne,p,geo", [(2, 32, 3, "annulus"), (2, 64, 5, "annulus"),
                                         (3, 10, 3, "annulus"), (3, 8, 4, "revolved")])
def test_gmres_to_tolerance_matches(d, ne, p, geo):
    R = ref(d, ne, p, geo)
    b = R.manufactured_rhs(0.0) if geo == "annulus" else _rand(R.N, 11)
    o = R.gmres(b, tol=1e-8, max_iter=300)
    with _problem(d, ne, p, geo) as P:
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=300)
        x = x.cpu().numpy()
    assert abs(info["iters"] - o["iters"]) <= 1
    relres = np.linalg.norm(b - R.A @ x) / np.linalg.norm(b)
    assert relres <= 1.05e-8
    assert abs(relres - info["relres_true"]) <= 1e-12
    assert np.linalg.norm(x - o["x"]) <= 1e-6 * np.linalg.norm(o["x"])
    assert np.all(np.diff(info["hist"]) <= 1e-15)


def test_unpreconditioned_matches_oracle():
    R = ref(2, 32, 3)
    b = R.manufactured_rhs(0.0)
    o = R.gmres(b, M=None, tol=1e-8, max_iter=1000)
    with _problem(2, 32, 3, precision="none") as P:
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=1000)
        x = x.cpu().numpy()
    assert abs(info["iters"] - o["iters"]) <= 2
    assert np.linalg.norm(b - R.A @ x) / np.linalg.norm(b) <= 1.05e-8
    # FD preconditioning cuts the count (Table 2 behaviour)
    with _problem(2, 32, 3) as P:
        _, info_fd = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=300)
    assert info_fd["iters"] < info["iters"] / 3


def test_initial_guess_paths():
    R = ref(2, 30, 3)
    b = R.manufactured_rhs(0.0)
    o = R.gmres(b, tol=1e-12, max_iter=300)
    with _problem(2, 30, 3) as P:
        bt = torch.from_numpy(b).cuda()
        x, info = P.solve(bt, x0=torch.from_numpy(o["x"]).cuda(), tol=1e-8, max_iter=50)
        assert info["iters"] == 0
        assert np.array_equal(x.cpu().numpy(), o["x"])
        x0 = _rand(R.N, 4)
        x, info = P.solve(bt, x0=torch.from_numpy(x0).cuda(), tol=1e-8, max_iter=200)
        x = x.cpu().numpy()
        assert np.linalg.norm(b - R.A @ x) / np.linalg.norm(b) <= 1.05e-8


def test_zero_and_nan_rhs():
    from paper_1705_04384_gb300 import IgaError
    with _problem(2, 12, 3) as P:
        z = torch.zeros(P.N, dtype=torch.float64, device="cuda")
        x, info = P.solve(z, tol=1e-8, max_iter=20)
        assert info["iters"] == 0 and torch.count_nonzero(x).item() == 0
        bad = torch.ones(P.N, dtype=torch.float64, device="cuda")
        bad[5] = float("nan")
        with pytest.raises(IgaError) as ei:
            P.solve(bad, tol=1e-8, max_iter=20)
        assert ei.value.status == 7
        # the handle stays usable
        x, info = P.solve(torch.ones_like(bad), tol=1e-8, max_iter=60)
        assert info["relres_true"] <= 1.05e-8


def test_max_iter_reports_no_convergence():
    from paper_1705_04384_gb300 import IgaError
    with _problem(2, 40, 3, precision="none") as P:
        b = torch.ones(P.N, dtype=torch.float64, device="cuda")
        with pytest.raises(IgaError) as ei:
            P.solve(b, tol=1e-8, max_iter=5, allow_no_convergence=False)
        assert ei.value.status == 5


def test_graph_and_eager_bitwise_equal_and_deterministic():
    R = ref(3, 9, 4, assemble=False)
    b = torch.from_numpy(_rand(R.N, 21)).cuda()
    with _problem(3, 9, 4) as P:
        x1, i1 = P.solve(b, tol=1e-9, max_iter=100)
        x2, i2 = P.solve(b, tol=1e-9, max_iter=100)
        os.environ["IGA_EAGER"] = "1"
        try:
            x3, i3 = P.solve(b, tol=1e-9, max_iter=100)
        finally:
            del os.environ["IGA_EAGER"]
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert i1["iters"] == i2["iters"] == i3["iters"]
    assert np.array_equal(i1["hist"], i3["hist"])


def test_host_buffer_solve_matches_device_solve():
    R = ref(2, 33, 4, assemble=False)
    b = _rand(R.N, 5)
    with _problem(2, 33, 4) as P:
        xd, infod = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=100)
        xh = np.zeros(R.N)
        infoh = P.solve_host(np.ascontiguousarray(b), xh, tol=1e-8, max_iter=100)
    assert infoh["iters"] == infod["iters"]
    assert np.array_equal(xh, xd.cpu().numpy())


@pytest.mark.parametrize("p", [3, 4, 5])
def test_full_size_3d_ne64(p):
    """The bench workload (3D extruded annulus, 64 elements, manufactured f with the
    seeded 1e-3 perturbation): sampled oracle rows of A_C, the full FD against the
    oracle's FD, and the residual of the converged solution on sampled rows."""
    import workload as W
    R = ref(3, 64, p, assemble=False)
    b = W.config_rhs("3d_annulus_ne64", R.points, p_index=p - 3)
    rng = np.random.default_rng(p)
    idx = np.unique(np.concatenate([[0, R.N - 1, R.N // 2],
                                    rng.integers(0, R.N, 24)]))
    rows = R.rows(idx)
    with _problem(3, 64, p) as P:
        u = _rand(R.N, 8)
        Au = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
        want = rows @ u
        assert np.max(np.abs(Au[idx] - want)) <= 1e-13 * np.max(np.abs(want))
        s = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
        s_ref = R.fd(b)
        assert np.linalg.norm(s - s_ref) <= 1e-11 * np.linalg.norm(s_ref)
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=200)
        x = x.cpu().numpy()
    assert info["status"] == 0 and info["relres_true"] <= 1e-8 * 1.05
    assert info["iters"] <= 60
    r = b[idx] - rows @ x
    assert np.max(np.abs(r)) <= 1.05e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("ne,p", [(64, 3), (32, 5)])
def test_full_size_3d_revolved(ne, p):
    """Sec. 5's 3D domain (the revolved quarter ring, all nine coefficient fields live) at
    the bench size: sampled oracle rows of A_C, the full FD against the oracle's FD, and
    the residual of the converged solution on sampled rows."""
    import workload as W
    R = ref(3, ne, p, geometry="revolved", assemble=False)
    b = W.config_rhs("3d_revolved_ne64", R.points, p_index=0)
    rng = np.random.default_rng(ne + p)
    idx = np.unique(np.concatenate([[0, R.N - 1, R.N // 2], rng.integers(0, R.N, 24)]))
    rows = R.rows(idx)
    with _problem(3, ne, p, "revolved") as P:
        u = _rand(R.N, 9)
        Au = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
        want = rows @ u
        assert np.max(np.abs(Au[idx] - want)) <= 1e-13 * np.max(np.abs(want))
        s = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
        s_ref = R.fd(b)
        assert np.linalg.norm(s - s_ref) <= 1e-11 * np.linalg.norm(s_ref)
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=300)
        x = x.cpu().numpy()
    assert info["status"] == 0 and info["relres_true"] <= 1e-8 * 1.05
    r = b[idx] - rows @ x
    assert np.max(np.abs(r)) <= 1.05e-8 * np.linalg.norm(b)


FMA_CHECK = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1705_04384_gb300.api import Problem
from tests.oracle_ref import ref
worst = 0.0
# n odd and even, tiny n, n past one 32-column run, 3D
for d, ne, p in ((2, 3, 2), (2, 14, 4), (2, 40, 3), (2, 130, 2), (2, 97, 5), (3, 3, 3),
                 (3, 8, 4), (3, 13, 6), (3, 20, 3)):
    R = ref(d, ne, p, assemble=False)
    with Problem(d, ne, p, precision="fp64") as P:
        for seed in (7, 8):
            b = np.random.default_rng(seed).standard_normal(R.N)
            got = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
            want = R.fd(b)
            e = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert e <= 1e-11, (d, ne, p, e)
            worst = max(worst, e / 1e-11)
# three right-hand sides in lockstep, GMRES iterate at fixed k against the oracle's
for d, ne, p, k in ((2, 24, 3, 6), (3, 9, 4, 5)):
    R = ref(d, ne, p)
    B = np.stack([R.manufactured_rhs(1e-3, s) for s in range(3)])
    with Problem(d, ne, p, precision="fp64") as P:
        X, info = P.solve_multi(torch.from_numpy(B).cuda(), tol=0.0, max_iter=k)
        X = X.cpu().numpy()
    for r in range(3):
        o = R.gmres(B[r], tol=0.0, max_iter=k)
        e = np.linalg.norm(X[r] - o["x"]) / np.linalg.norm(o["x"])
        assert info["iters"][r] == k and e <= 1e-10, (d, ne, p, r, e)
        worst = max(worst, e / 1e-10)
print("ok", worst)
"""


@pytest.mark.parametrize("kernel", ["fma", "mma"])
def test_fd64_kernels_match_oracle(kernel, tmp_path):
    """Both kernels of the folded FP64 mode products, forced through IGA_FD64 (read once
    per process, hence a child process), against the oracle's FD (1e-11, as above) and
    GMRES iterates (1e-10) with one and three right-hand sides."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fd64.py"
    script.write_text(FMA_CHECK)
    env = dict(os.environ, IGA_FD64=kernel, PYTHONPATH=root)
    r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def test_fd_kernel_choice():
    """iga_fd_kernel names the kernel the FD solve runs: the folded products on mma.sync for
    few rows, on FMAs for many (unless IGA_FD64 forces one), dense products for a wind,
    tensor cores for the precision forms."""
    from paper_1705_04384_gb300.api import Problem
    forced = os.environ.get("IGA_FD64")
    with _problem(3, 8, 3) as P:
        assert P.fd_kernel(1) == ("fold_fma" if forced == "fma" else "fold_mma")
    with _problem(2, 1024, 3) as P:
        assert P.fd_kernel(1) == ("fold_mma" if forced == "mma" else "fold_fma")
    with Problem(2, 16, 3, wind=(2.0, 1.0), precision="fp64") as P:
        assert P.fd_kernel(1) == "dense_mma"
    with _problem(2, 16, 3, precision="tf32") as P:
        assert P.fd_kernel(2) == "tensor_core"


def test_operator_flop_count():
    """iga_operator_flops counts the plan's banded products: the 3D extruded annulus keeps
    4 of 9 fields (2 + 3 + 4 band passes of 2W FLOPs per DOF, 2 per contracted term), the
    2D one 3 of 5 (2 passes along the second direction, 3 contracted terms); a WQ plan on
    the quadrature grid costs more per DOF than the collocation plan of the same mesh."""
    import bench
    from paper_1705_04384_gb300.api import Problem
    for p in (3, 4):
        with _problem(3, 8, p) as P:
            assert P.operator_flops() == bench.operator_flops_per_dof(p + 1, 3) * P.N
    with _problem(2, 12, 3) as P:
        assert P.operator_flops() == P.N * (2 * 4 * (2 + 3) + 2 * 3)
    with Problem(3, 6, 3, geometry="revolved", precision="fp64", scheme="wq") as P:
        fl_wq = P.operator_flops()
    with Problem(3, 6, 3, geometry="revolved", precision="fp64") as P:
        assert fl_wq > 4 * P.operator_flops() > 0


FUSE_RUN = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1705_04384_gb300.api import Problem
out = {}
g = np.random.default_rng(5)
for key, (d, ne, p, geo, prec, R, tol, mi) in enumerate((
        (2, 30, 3, "annulus", "fp64", 1, 1e-8, 200),
        (3, 10, 4, "revolved", "fp64", 1, 0.0, 22),      # 23 basis vectors: the chunked path
        (3, 9, 3, "annulus", "fp64", 3, 1e-8, 200),      # right-hand sides finishing apart
        (3, 12, 3, "annulus", "tf32", 2, 1e-8, 200),
        (2, 40, 5, "annulus", "none", 1, 0.0, 18),
        (2, 20, 3, "annulus", "fp64", 2, 0.0, 30))):   # up to 31 vectors: every pass-2 path
    with Problem(d, ne, p, geometry=geo, precision=prec) as P:
        B = g.standard_normal((R, P.N))
        B[0] *= 1e3  # different scales: different step counts
        if R == 1:
            x, info = P.solve(torch.from_numpy(B[0]).cuda(), tol=tol, max_iter=mi)
            out[f"x{key}"] = x.cpu().numpy()
            out[f"h{key}"] = info["hist"]
        else:
            X, info = P.solve_multi(torch.from_numpy(B).cuda(), tol=tol, max_iter=mi)
            out[f"x{key}"] = X.cpu().numpy()
            for r in range(R):
                out[f"h{key}_{r}"] = info["hist"][r]
np.savez(sys.argv[2], **out)
print("ok")
"""


def test_fused_operator_pass1_is_bitwise_the_unfused_step(tmp_path):
    """The Arnoldi step's fused kernel (the operator's last pass with CGS2 pass 1) does the
    same FP64 operations in the same order as the two kernels it replaces: solutions and
    residual histories are bitwise equal with IGA_FUSE_P1=0 (read once per process, hence
    child processes) -- 2D and 3D, more than 15 basis vectors, right-hand sides that stop at
    different steps, the TF32 form and the unpreconditioned solver."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fuse.py"
    script.write_text(FUSE_RUN)
    res = {}
    for flag in ("1", "0"):
        f = tmp_path / f"r{flag}.npz"
        env = dict(os.environ, IGA_FUSE_P1=flag, PYTHONPATH=root)
        r = subprocess.run([sys.executable, str(script), root, str(f)], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
        res[flag] = dict(np.load(f))
    assert res["1"].keys() == res["0"].keys()
    for k in res["1"]:
        assert np.array_equal(res["1"][k], res["0"][k]), k


def test_stashed_pass2_is_bitwise_the_two_sweep_pass2(tmp_path):
    """CGS2 pass 2 for 16..21 basis vectors keeps the row's entries of V in shared memory
    instead of reading V twice; it does the same FMAs in the same order and forms the same
    partials, so solutions and residual histories are bitwise those of the two-sweep path
    (IGA_P2_STASH=0), for solves that pass through 1..15, 16..21 and 22..31 vectors."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "stash.py"
    script.write_text(FUSE_RUN)
    res = {}
    for flag in ("1", "0"):
        f = tmp_path / f"s{flag}.npz"
        env = dict(os.environ, IGA_P2_STASH=flag, PYTHONPATH=root)
        r = subprocess.run([sys.executable, str(script), root, str(f)], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
        res[flag] = dict(np.load(f))
    assert res["1"].keys() == res["0"].keys()
    for k in res["1"]:
        assert np.array_equal(res["1"][k], res["0"][k]), k
