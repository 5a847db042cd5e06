"""GPU parity of the weighted-quadrature Galerkin discretization (Sec. 2.3, eq. WQapprox)
against the oracle (oracle/wq.py), through the C ABI.

Tolerances (FP64; the same arguments as the collocation parity tests):
* univariate Galerkin factors M, K: 1e-13 relative (Gauss sums of the same products in a
  different order; K is of size 1/h, its entries agree to ~1e-14 relative);
* operator A_wq u: 1e-12 relative to max |A_wq u| (sums over up to (3p + 2)^d weights times
  (p + 1)^d basis values per output, different order; the weights themselves come from two
  different minimum-norm solvers, agreeing to ~1e-15 relative);
* FD solve of P_wq: 1e-11 (as for collocation);
* load vector: 1e-13;
* GMRES iterate at a fixed number of steps: 1e-10; to 1e-8: iterations within +-1 of the
  oracle's and true residual <= 1.05e-8 with the oracle's A_wq.
"""

import numpy as np
import pytest
import torch

from oracle import fd as F, geometry as Geo, gmres as G, wq as Q

pytestmark = pytest.mark.gpu


def _problem(d, ne, p, geometry="annulus", precision="fp64"):
    from paper_1705_04384_gb300.api import Problem
    return Problem(d, ne, p, geometry=geometry, precision=precision, scheme="wq")


class _Ref:
    def __init__(self, d, ne, p, geometry, assemble=True):
        self.spaces = [Q.WQSpace1D(ne, p) for _ in range(d)]
        self.fmap = Geo.make_map(geometry, d, 1.0, 2.0)
        self.A = Q.assemble_wq(self.spaces, self.fmap) if assemble else None
        self.op = Q.WQOperator(self.spaces, self.fmap)
        self.fd = F.FD(self.spaces)
        self.N = int(np.prod([s.n for s in self.spaces]))


_CACHE = {}


def ref(d, ne, p, geometry="annulus", assemble=True):
    key = (d, ne, p, geometry, assemble)
    if key not in _CACHE:
        _CACHE[key] = _Ref(d, ne, p, geometry, assemble)
    return _CACHE[key]


def _rand(N, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(N)


CASES = [(2, 12, 2, "annulus"), (2, 17, 3, "annulus"), (2, 9, 6, "annulus"),
         (2, 10, 4, "identity"), (3, 5, 3, "annulus"), (3, 6, 2, "revolved"),
         (3, 4, 4, "revolved"), (3, 5, 5, "identity")]


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_galerkin_factors_and_eigenpairs(p):
    R = ref(2, 14, p, assemble=False)
    s = R.spaces[0]
    with _problem(2, 14, p) as P:
        M, K = P.factor("M"), P.factor("K")
        assert np.max(np.abs(M - s.M)) <= 1e-13 * np.max(np.abs(s.M))
        assert np.max(np.abs(K - s.K)) <= 1e-13 * np.max(np.abs(s.K))
        lam, U, Vt = P.factor("lambda"), P.factor("U"), P.factor("Vt")
        assert np.max(np.abs(lam - R.fd.lam[0]) / R.fd.lam[0]) <= 1e-10
        assert np.max(np.abs(s.K @ U - s.M @ U * lam)) <= 1e-10 * np.max(np.abs(s.K))
        assert np.max(np.abs(Vt @ (s.M @ U) - np.eye(s.n))) <= 1e-10


@pytest.mark.parametrize("d,ne,p,geo", CASES)
def test_wq_operator_matches_oracle(d, ne, p, geo):
    R = ref(d, ne, p, geo)
    with _problem(d, ne, p, geo) as P:
        for seed in (0, 1):
            u = _rand(R.N, seed)
            got = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
            want = R.A @ u
            assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), seed


@pytest.mark.parametrize("d,ne,p,geo", [(2, 16, 3, "annulus"), (3, 6, 4, "revolved")])
def test_wq_fd_and_load_match_oracle(d, ne, p, geo):
    R = ref(d, ne, p, geo, assemble=False)
    with _problem(d, ne, p, geo) as P:
        b = _rand(R.N, 3)
        s = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
        want = R.fd(b)
        assert np.linalg.norm(s - want) <= 1e-11 * np.linalg.norm(want)
        nq, Nq = P.quadrature_dims()
        assert nq == R.spaces[0].nq and Nq == nq ** d
        X = P.quadrature_points()
        assert np.max(np.abs(X - Q.quadrature_points_physical(R.spaces, R.fmap))) <= 1e-14
        g = np.sin(X[:, 0]) + X[:, 1] ** 2
        f = P.wq_load(torch.from_numpy(g).cuda()).cpu().numpy()
        fo = Q.wq_load(R.spaces, R.fmap, g)
        assert np.max(np.abs(f - fo)) <= 1e-13 * np.max(np.abs(fo))


def test_collocation_points_rejected_for_wq():
    from paper_1705_04384_gb300 import IgaError
    with _problem(2, 8, 3) as P:
        with pytest.raises(IgaError) as e:
            P.collocation_points()
        assert e.value.status == 8


@pytest.mark.parametrize("d,ne,p,geo", [(2, 20, 3, "annulus"), (3, 6, 3, "revolved")])
def test_wq_gmres_fixed_k_and_to_tolerance(d, ne, p, geo):
    R = ref(d, ne, p, geo)
    b = _rand(R.N, 11)
    with _problem(d, ne, p, geo) as P:
        bd = torch.from_numpy(b).cuda()
        for k in (1, 4, 9):
            o = G.gmres(R.A, b, M=R.fd, tol=0.0, max_iter=k)
            x, info = P.solve(bd, tol=0.0, max_iter=k)
            x = x.cpu().numpy()
            assert info["iters"] == k
            assert np.linalg.norm(x - o["x"]) <= 1e-10 * np.linalg.norm(o["x"]), k
        o = G.gmres(R.A, b, M=R.fd, tol=1e-8, max_iter=200)
        x, info = P.solve(bd, tol=1e-8, max_iter=200)
        x = x.cpu().numpy()
        assert abs(info["iters"] - o["iters"]) <= 1
        assert np.linalg.norm(b - R.A @ x) <= 1.05e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3", "fp64tc"])
def test_wq_precision_form_reaches_fp64_residual(prec):
    R = ref(2, 24, 4, "annulus")
    b = _rand(R.N, 5)
    with _problem(2, 24, 4, "annulus", prec) as P:
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=200)
        x = x.cpu().numpy()
    assert np.linalg.norm(b - R.A @ x) <= 1.05e-8 * np.linalg.norm(b)


def test_wq_bicgstab_matches_oracle_half_steps():
    from oracle import bicgstab as BI
    R = ref(2, 32, 3, "annulus")
    b = Q.galerkin_rhs(R.spaces, R.fmap, lambda x: np.ones(x.shape[0]))
    o = BI.bicgstab(R.A, b, M=R.fd, tol=1e-8, max_iter=200)
    with _problem(2, 32, 3) as P:
        x, info = P.solve_bicgstab(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=200)
        x = x.cpu().numpy()
    assert abs(info["half_steps"] - o["steps"]) <= 2
    assert np.linalg.norm(b - R.A @ x) <= 1.05e-8 * np.linalg.norm(b)


def test_wq_full_size_3d_revolved_ne64():
    """The bench's WQ workload (Sec. 5's revolved ring, 64 elements, p = 3, N = 274,625;
    2.35 M quadrature points): operator against the oracle's matrix-free A_wq, and a solve
    whose true residual the oracle recomputes."""
    R = ref(3, 64, 3, "revolved", assemble=False)
    with _problem(3, 64, 3, "revolved") as P:
        u = _rand(R.N, 2)
        got = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
        want = R.op(u)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
        X = P.quadrature_points()
        g = np.ones(X.shape[0])
        b = P.wq_load(torch.from_numpy(g).cuda())
        x, info = P.solve(b, tol=1e-8, max_iter=200)
        bn, xn = b.cpu().numpy(), x.cpu().numpy()
        assert info["status"] == 0
        assert np.linalg.norm(bn - R.op(xn)) <= 1.05e-8 * np.linalg.norm(bn)


@pytest.mark.parametrize("d,ne,p,geo,prec", [(2, 14, 3, "annulus", "fp64"),
                                              (3, 5, 4, "revolved", "fp64"),
                                              (3, 6, 3, "revolved", "tf32")])
def test_wq_several_rhs_bitwise_alone_and_against_oracle(d, ne, p, geo, prec):
    """Several right-hand sides in lockstep on a WQ problem: every pass of the matrix-free
    operator, the fan-out to Q_ab times each derivative included, addresses each right-hand
    side's slice. Each solution must equal the same right-hand side's solve alone bit for
    bit, and (FP64) the oracle's GMRES iterate at a fixed step count to 1e-10."""
    R = ref(d, ne, p, geo)
    B = np.stack([_rand(R.N, 20 + s) * (10.0 ** s) for s in range(3)])
    with _problem(d, ne, p, geo, prec) as P:
        X, info = P.solve_multi(torch.from_numpy(B).cuda(), tol=0.0, max_iter=7)
        X = X.cpu().numpy()
        for r in range(3):
            x1, i1 = P.solve(torch.from_numpy(B[r]).cuda(), tol=0.0, max_iter=7)
            assert np.array_equal(x1.cpu().numpy(), X[r]), r
            if prec == "fp64":
                o = G.gmres(R.A, B[r], M=R.fd, tol=0.0, max_iter=7)
                assert np.linalg.norm(X[r] - o["x"]) <= 1e-10 * np.linalg.norm(o["x"]), r
