"""Pins of the BiCGStab oracle (oracle/bicgstab.py, Sec. 5's solver).

* a worked 2 x 2 example computed by hand (first iteration's iterate and residuals,
  and termination at iteration 1.5: BiCG ends in n = 2 steps, so the BiCG half of
  iteration 2 leaves a zero residual);
* agreement with scipy's independent BiCGStab at fixed step counts, with the FD
  preconditioner of a collocation problem as M;
* an exact preconditioner (M = A^-1, or the FD solve for the identity map, where
  A_C = P_C) stops after one half step with the exact solution;
* zero right-hand side, history length and the final true residual.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bicgstab as B, collocation as C, fd as F, geometry as Geo


def test_worked_2x2_example():
    # A = diag(1, 2), b = (1, 1), M = I.  r0 = rhat = b, rho = 2, p = (1, 1),
    # v = A p = (1, 2), alpha = 2 / 3, s = (1/3, -1/3), t = A s = (1/3, -2/3),
    # omega = (t.s)/(t.t) = (3/9)/(5/9) = 3/5, x1 = alpha p + omega s = (13/15, 7/15),
    # r1 = s - omega t = (2/15, 1/15).
    A = np.diag([1.0, 2.0])
    b = np.array([1.0, 1.0])
    one = B.bicgstab(A, b, tol=0.0, max_iter=1)
    assert np.allclose(one["x"], [13 / 15, 7 / 15], rtol=0, atol=1e-15)
    nb = np.sqrt(2.0)
    assert np.allclose(one["hist"], [1.0, (np.sqrt(2) / 3) / nb, (np.sqrt(5) / 15) / nb],
                       rtol=1e-14, atol=0)
    assert one["steps"] == 2 and one["flag"] == 2
    full = B.bicgstab(A, b, tol=1e-12, max_iter=10)
    assert full["steps"] == 3 and full["iters"] == 1.5 and full["flag"] == 0
    assert np.allclose(full["x"], [1.0, 0.5], rtol=0, atol=1e-14)


def _small_problem(d=2, ne=8, p=3, kind="annulus"):
    spaces = [C.Space1D(ne, p) for _ in range(d)]
    fmap = Geo.make_map(kind, d, 1.0, 2.0)
    A = C.assemble_collocation(spaces, fmap)
    return A, F.FD(spaces), spaces


@pytest.mark.parametrize("d,ne,p", [(2, 8, 3), (3, 4, 4)])
def test_matches_scipy_at_fixed_step_counts(d, ne, p):
    A, fd, _ = _small_problem(d, ne, p)
    N = A.shape[0]
    b = np.random.default_rng(d + ne).standard_normal(N)
    M = spla.LinearOperator((N, N), matvec=fd, dtype=np.float64)
    for k in range(1, 7):
        mine = B.bicgstab(A, b, M=fd, tol=0.0, max_iter=k)
        theirs, info = spla.bicgstab(A, b, rtol=0.0, atol=0.0, maxiter=k, M=M)
        assert mine["steps"] == 2 * k
        assert np.linalg.norm(mine["x"] - theirs) <= 1e-10 * np.linalg.norm(theirs), k


def test_exact_preconditioner_stops_after_one_half_step():
    rng = np.random.default_rng(3)
    A = np.eye(20) * 4.0 + rng.standard_normal((20, 20))
    b = rng.standard_normal(20)
    Ainv = np.linalg.inv(A)
    out = B.bicgstab(A, b, M=Ainv, tol=1e-10, max_iter=50)
    assert out["steps"] == 1 and out["iters"] == 0.5 and out["flag"] == 0
    assert np.linalg.norm(out["x"] - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(out["x"])


def test_identity_map_fd_is_the_exact_inverse():
    # for the identity map A_C = P_C (pinned in test_oracle_collocation), so the FD
    # preconditioner is exact and BiCGStab stops after the BiCG half of iteration 1
    A, fd, _ = _small_problem(2, 10, 3, kind="identity")
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    out = B.bicgstab(A, b, M=fd, tol=1e-8, max_iter=50)
    assert out["steps"] == 1 and out["flag"] == 0
    assert out["relres_true"] <= 1e-12


def test_zero_rhs_takes_no_step():
    A, fd, _ = _small_problem(2, 6, 2)
    out = B.bicgstab(A, np.zeros(A.shape[0]), M=fd)
    assert out["steps"] == 0 and out["flag"] == 0 and not np.any(out["x"])


def test_history_and_true_residual_at_tolerance():
    A, fd, _ = _small_problem(2, 16, 4)
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    out = B.bicgstab(A, b, M=fd, tol=1e-8, max_iter=100)
    assert out["flag"] == 0
    assert len(out["hist"]) == out["steps"] + 1
    assert out["hist"][-1] <= 1e-8 and np.all(out["hist"][:-1] > 1e-8)
    assert out["relres_true"] <= 1.05e-8


def _sec5_table():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sec5_bicgstab_iterations.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            dom, hinv, p, its = line.split()
            rows.append((dom, int(hinv), int(p), float(its)))
    return rows


def test_iteration_counts_of_the_sec5_tables():
    """The oracle's BiCGStab + FD on the configurations of Sec. 5's Tables 2 and 4
    (tests/golden/sec5_bicgstab_iterations.txt: h^-1 = 128 and 256 in 2D, 16 and 32 in 3D)
    lands within 2.5 iterations of every
    printed count and within 1.5 on average.  The paper leaves the tolerance and the
    source term open (f = 1 and 1e-6 here), so the counts are compared with a margin;
    a wrong operator, preconditioner or iteration count would miss it by far more."""
    diffs = []
    for dom, hinv, p, paper in _sec5_table():
        d, kind = (2, "annulus") if dom == "quarter" else (3, "revolved")
        spaces = [C.Space1D(hinv, p) for _ in range(d)]
        fmap = Geo.make_map(kind, d, 1.0, 2.0)
        A = C.assemble_collocation(spaces, fmap)
        o = B.bicgstab(A, np.ones(A.shape[0]), M=F.FD(spaces), tol=1e-6, max_iter=200)
        assert o["flag"] == 0
        assert abs(o["iters"] - paper) <= 2.5, (dom, hinv, p, o["iters"], paper)
        diffs.append(abs(o["iters"] - paper))
    assert np.mean(diffs) <= 1.5
