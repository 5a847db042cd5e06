"""Convection-diffusion with a constant wind (Sec. 3.2, collocation form) on the GPU
against the oracle.

Tolerances as for the Poisson operator and FD (test_gpu_parity.py): the operator's
sums gain one first-order term per direction (1e-13); the FD factors of the shifted
pencils are less well conditioned than the Poisson ones (cond(U) about 5 at these
winds, 100 at |w| = 10), so the FD parity is 1e-10; GMRES to 1e-8 as before.
"""

import numpy as np
import pytest
import torch

from oracle import bicgstab as OB, collocation as C, fd as F
from tests.oracle_ref import ref

pytestmark = pytest.mark.gpu


def _problem(d, ne, p, geometry="annulus", wind=None, precision="fp64"):
    from paper_1705_04384_gb300.api import Problem
    return Problem(d, ne, p, geometry=geometry, wind=wind, precision=precision)


def _rand(N, seed):
    return np.random.default_rng(seed).standard_normal(N)


CASES = [(2, 10, 3, "annulus", (3.0, -2.0)), (2, 8, 5, "annulus", (0.0, 4.0)),
         (3, 6, 3, "annulus", (3.0, -2.0, 1.5)), (3, 5, 4, "revolved", (1.0, 2.0, -3.0))]


@pytest.mark.parametrize("d,ne,p,geo,wind", CASES)
def test_operator_fd_and_solve_match_oracle(d, ne, p, geo, wind):
    R = ref(d, ne, p, geo, wind=wind)
    u = _rand(R.N, 1)
    with _problem(d, ne, p, geo, wind) as P:
        Au = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
        want = R.A @ u
        assert np.max(np.abs(Au - want)) <= 1e-13 * np.max(np.abs(want))
        s = P.precond_apply(torch.from_numpy(u).cuda()).cpu().numpy()
        s_ref = R.fd(u)
        assert np.linalg.norm(s - s_ref) <= 1e-10 * np.linalg.norm(s_ref)
        for l in range(d):
            lam = P.factor("lambda", l)
            want_lam = F.eig_factors(C.wind_factor(R.spaces[l], wind[l]), R.spaces[l].M)[0]
            assert np.allclose(lam, want_lam, rtol=1e-10, atol=0)
        b = _rand(R.N, 2)
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=300)
        want_it = R.gmres(b, tol=1e-8, max_iter=300)["iters"]
        assert info["status"] == 0 and abs(info["iters"] - want_it) <= 1
        assert np.linalg.norm(b - R.A @ x.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)
        xb, ib = P.solve_bicgstab(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=300)
        want_b = OB.bicgstab(R.A, b, M=R.fd, tol=1e-8, max_iter=300)
        assert ib["status"] == 0 and abs(ib["half_steps"] - want_b["steps"]) <= 1
        assert np.linalg.norm(b - R.A @ xb.cpu().numpy()) <= 1.05e-8 * np.linalg.norm(b)


def test_identity_map_preconditioner_is_exact():
    wind = (5.0, -3.0, 2.0)
    R = ref(3, 8, 3, "identity", wind=wind)
    b = _rand(R.N, 3)
    with _problem(3, 8, 3, "identity", wind) as P:
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_iter=20)
    assert info["iters"] == 1
    assert np.linalg.norm(b - R.A @ x.cpu().numpy()) <= 1e-11 * np.linalg.norm(b)


def test_zero_wind_is_the_poisson_problem():
    u = torch.from_numpy(_rand(ref(2, 12, 4, assemble=False).N, 4)).cuda()
    with _problem(2, 12, 4) as P0, _problem(2, 12, 4, wind=(0.0, 0.0)) as P1:
        assert torch.equal(P0.apply_operator(u), P1.apply_operator(u))
        assert torch.equal(P0.precond_apply(u), P1.precond_apply(u))


def test_rejected_settings():
    from paper_1705_04384_gb300._lib import IgaError
    with pytest.raises(IgaError):
        _problem(2, 10, 3, wind=(1.0, 1.0), precision="tf32")
    with pytest.raises(IgaError, match="diagonaliz|NOT_DIAG|ill"):
        _problem(2, 64, 3, wind=(60.0, 0.0))


def test_full_size_3d_wind_ne64():
    """The wind bench workload (3D extruded ring, 64 elements, p = 3, w = (5, 5, 5)):
    sampled oracle rows of A_C, the full FD, the converged residual on sampled rows."""
    import workload as W
    wind = W.CONFIGS["3d_wind_ne64"]["wind"]
    R = ref(3, 64, 3, assemble=False, wind=wind)
    b = W.config_rhs("3d_wind_ne64", R.points, p_index=0)
    rng = np.random.default_rng(64)
    idx = np.unique(np.concatenate([[0, R.N - 1, R.N // 2], rng.integers(0, R.N, 24)]))
    rows = R.rows(idx)
    with _problem(3, 64, 3, wind=wind) as P:
        u = _rand(R.N, 5)
        Au = P.apply_operator(torch.from_numpy(u).cuda()).cpu().numpy()
        want = rows @ u
        assert np.max(np.abs(Au[idx] - want)) <= 1e-13 * np.max(np.abs(want))
        s = P.precond_apply(torch.from_numpy(b).cuda()).cpu().numpy()
        s_ref = R.fd(b)
        assert np.linalg.norm(s - s_ref) <= 1e-10 * np.linalg.norm(s_ref)
        x, info = P.solve(torch.from_numpy(b).cuda(), tol=1e-8, max_iter=300)
        x = x.cpu().numpy()
    assert info["status"] == 0 and info["relres_true"] <= 1.05e-8
    r = b[idx] - rows @ x
    assert np.max(np.abs(r)) <= 1.05e-8 * np.linalg.norm(b)
