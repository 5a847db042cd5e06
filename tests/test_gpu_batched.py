"""Batched form: several right-hand sides of one problem in lockstep, and several
problems of uneven size, degree and dimension solved concurrently.

Every reduction runs in a fixed block order per right-hand side and every kernel
computes each entry with the same arithmetic whatever the batch size, so a result
must be bitwise identical alone and in the mix; each must also meet the FP64 true
residual 1e-8 checked with the oracle's A_C.
"""

import numpy as np
import pytest
import torch

from tests.oracle_ref import ref

pytestmark = pytest.mark.gpu


def _problem(d, ne, p, precision="fp64", r0=1.0, r1=2.0, stream=None, grid="latency"):
    from paper_1705_04384_gb300.api import Problem
    return Problem(d, ne, p, r_inner=r0, r_outer=r1, precision=precision, stream=stream,
                   grid=grid)


def _rhs(N, nrhs, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((nrhs, N))


@pytest.mark.parametrize("grid", ["latency", "throughput"])
@pytest.mark.parametrize("prec", ["fp64", "tf32", "bf16", "none", "tf32x3", "fp64tc"])
@pytest.mark.parametrize("d,ne,p", [(2, 30, 3), (3, 9, 4)])
def test_multi_rhs_bitwise_equals_single(prec, d, ne, p, grid):
    R = ref(d, ne, p)
    B = _rhs(R.N, 4, 17)
    B[2] *= 1e-3  # different scales converge at different steps
    maxit = 600 if prec == "none" else 200
    with _problem(d, ne, p, prec, grid=grid) as P:
        X, info = P.solve_multi(torch.from_numpy(B).cuda(), tol=1e-8, max_iter=maxit)
        X = X.cpu().numpy()
        for r in range(4):
            x1, i1 = P.solve(torch.from_numpy(B[r]).cuda(), tol=1e-8, max_iter=maxit)
            assert i1["iters"] == info["iters"][r]
            assert np.array_equal(x1.cpu().numpy(), X[r])
            assert np.array_equal(i1["hist"], info["hist"][r])
    for r in range(4):
        relres = np.linalg.norm(B[r] - R.A @ X[r]) / np.linalg.norm(B[r])
        assert relres <= 1.05e-8
        assert abs(relres - info["relres_true"][r]) <= 1e-12


def test_multi_rhs_zero_nan_and_regular_mix():
    R = ref(2, 24, 3)
    B = _rhs(R.N, 3, 5)
    B[0] = 0.0
    B[1, 7] = np.nan
    with _problem(2, 24, 3) as P:
        from paper_1705_04384_gb300 import IgaError
        with pytest.raises(IgaError) as ei:
            P.solve_multi(torch.from_numpy(B).cuda(), tol=1e-8, max_iter=100)
        assert ei.value.status == 7
        # per-rhs statuses through the raw entry point
        import ctypes
        rhs = torch.from_numpy(B).cuda()
        out = torch.empty_like(rhs)
        iters = np.zeros(3, dtype=np.int32)
        stat = np.zeros(3, dtype=np.int32)
        st = P.lib.iga_solve_multi(P.h, 3, ctypes.c_void_p(rhs.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), 0, 1e-8, 100,
                                   iters.ctypes.data_as(ctypes.c_void_p), None, None,
                                   stat.ctypes.data_as(ctypes.c_void_p))
        assert st == 7
        assert list(stat) == [0, 7, 0]
        assert iters[0] == 0 and torch.count_nonzero(out[0]).item() == 0
        x2 = out[2].cpu().numpy()
        assert np.linalg.norm(B[2] - R.A @ x2) / np.linalg.norm(B[2]) <= 1.05e-8


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_batched_uneven_problems_match_individual_solves(prec):
    from paper_1705_04384_gb300.api import solve_batched
    specs = [(2, 40, 2, 0.7), (2, 57, 5, 1.3), (3, 8, 3, 1.0), (2, 33, 6, 0.5), (3, 10, 4, 1.2)]
    probs, rhs, outs, refs = [], [], [], []
    for q, (d, ne, p, r0) in enumerate(specs):
        s = torch.cuda.Stream()
        P = _problem(d, ne, p, prec, r0=r0, r1=r0 + 1.0, stream=s)
        nr = 1 + q % 3
        B = torch.from_numpy(_rhs(P.N, nr, 100 + q)).cuda()
        probs.append(P)
        rhs.append(B)
        outs.append(torch.empty_like(B))
        refs.append(ref(d, ne, p, "annulus", r0, r0 + 1.0))
    torch.cuda.synchronize()
    res = solve_batched(probs, rhs, outs, tol=1e-8, max_iter=200, history=True)
    torch.cuda.synchronize()
    assert np.all(res["status"] == 0)
    assert res["hist"].shape == (int(res["nrhs"].sum()), 201)
    off = 0
    for P, B, X, R in zip(probs, rhs, outs, refs):
        nr = B.shape[0]
        Xi, info = P.solve_multi(B, tol=1e-8, max_iter=200)
        assert torch.equal(Xi, X)
        assert np.array_equal(info["iters"], res["iters"][off:off + nr])
        for r in range(nr):
            # the batch returns each right-hand side's residual history, bitwise the same as
            # alone, zero past its last iteration
            k = int(info["iters"][r])
            assert np.array_equal(res["hist"][off + r, :k + 1], info["hist"][r])
            assert not np.any(res["hist"][off + r, k + 1:])
        Bn, Xn = B.cpu().numpy(), X.cpu().numpy()
        for r in range(nr):
            assert np.linalg.norm(Bn[r] - R.A @ Xn[r]) / np.linalg.norm(Bn[r]) <= 1.05e-8
        off += nr
    for P in probs:
        P.close()


def test_async_ready_collect_overlap():
    P1 = _problem(2, 64, 3, stream=torch.cuda.Stream())
    P2 = _problem(3, 12, 4, stream=torch.cuda.Stream())
    b1 = torch.from_numpy(_rhs(P1.N, 2, 1)).cuda()
    b2 = torch.from_numpy(_rhs(P2.N, 1, 2)).cuda()
    torch.cuda.synchronize()
    x1, x2 = torch.empty_like(b1), torch.empty_like(b2)
    P1.solve_async(b1, x1)
    P2.solve_async(b2, x2)
    from paper_1705_04384_gb300 import IgaError
    with pytest.raises(IgaError):  # one solve in flight per handle
        P1.solve_async(b1, x1)
    i1 = P1.collect()
    i2 = P2.collect()
    assert P1.ready() and P2.ready()
    y1, j1 = P1.solve_multi(b1)
    y2, j2 = P2.solve_multi(b2)
    assert torch.equal(x1.view_as(y1), y1) and torch.equal(x2.view_as(y2), y2)
    assert np.array_equal(i1["iters"], j1["iters"]) and np.array_equal(i2["iters"], j2["iters"])
    P1.close()
    P2.close()


@pytest.mark.parametrize("d,ne,p", [(2, 200, 3), (3, 40, 4)])
def test_grid_modes_agree(d, ne, p):
    """The two reduction grids partition the rows differently: at a fixed number of
    Arnoldi steps the iterates differ by rounding only."""
    b = torch.from_numpy(_rhs(ref(d, ne, p, assemble=False).N, 1, 5)[0]).cuda()
    xs = []
    for grid in ("latency", "throughput"):
        with _problem(d, ne, p, "fp64", grid=grid) as P:
            x, info = P.solve(b, tol=0.0, max_iter=12)
            assert info["iters"] == 12
            xs.append(x.cpu().numpy())
    assert np.linalg.norm(xs[1] - xs[0]) <= 1e-10 * np.linalg.norm(xs[0])
