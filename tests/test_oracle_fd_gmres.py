"""Pins for oracle.fd (Sec. 4) and oracle.gmres (Sec. 3 Krylov solver).

FD: the 1D pencil's spectrum against the Dirichlet Laplacian's closed form (k pi)^2,
Remark 1's properties, FD(P b) = b, FD = dense Kronecker solve on tiny n, invariance
under eigenvector scaling, the symmetric special case V = U (Sec. 4).
GMRES: one iteration on the identity map (A_C = P_C), the k-th iterate equals the
brute-force least-squares minimizer over the Krylov space, exactness at k = N,
monotone history, flexible = standard for a fixed preconditioner, and the
qualitative Table 2 behaviour (FD count flat in h, unpreconditioned count growing).
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import workload as W
from oracle import collocation as C, fd as F, geometry as Geo, gmres as G


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_pencil_spectrum_approaches_dirichlet_laplacian(p):
    s = C.Space1D(64, p)
    lam, U, V = F.eig_factors(s.K, s.M)
    for k in (1, 2, 3):
        assert abs(lam[k - 1] / (k * np.pi) ** 2 - 1.0) < 2e-3 * k * k
    assert np.all(lam > 0)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_remark1_outlier_pair_and_conditioning(p):
    s = C.Space1D(32, p)
    lam, U, V = F.eig_factors(s.K, s.M)
    assert abs(lam[-1] - lam[-2]) / lam[-1] < 1e-4  # near-double outlier
    assert np.linalg.cond(U) < 100


@pytest.mark.parametrize("ne,p", [(95, 5), (200, 6), (64, 5), (33, 4)])
def test_outlier_pair_split_by_reflection_is_well_conditioned(ne, p):
    s = C.Space1D(ne, p)
    assert F.is_reflection_symmetric(s.K) and F.is_reflection_symmetric(s.M)
    lam, U, V = F.eig_factors(s.K, s.M)
    assert np.linalg.cond(U) < 50
    # each eigenvector is even or odd under the flip, and solves the pencil
    par = np.sum(U[::-1] * U, axis=0)
    assert np.all(np.abs(np.abs(par) - 1.0) < 1e-12)
    assert np.max(np.abs(s.K @ U - s.M @ U * lam)) <= 1e-11 * np.max(np.abs(s.K))
    assert np.max(np.abs(V.T @ s.M @ U - np.eye(s.n))) < 1e-11


def test_reflection_basis_is_orthogonal():
    for n in (1, 2, 5, 8):
        E, O = F.reflection_basis(n)
        Q = np.hstack([E, O])
        assert np.max(np.abs(Q.T @ Q - np.eye(n))) < 1e-15
        assert np.allclose(E[::-1], E) and np.allclose(O[::-1], -O)


def test_complex_pencil_is_rejected():
    K = np.array([[0.0, -1.0], [1.0, 0.0]])
    with pytest.raises(F.NotDiagonalizable):
        F.eig_factors(K, np.eye(2))


@pytest.mark.parametrize("d,ne,p", [(2, 6, 2), (2, 9, 3), (3, 4, 3), (3, 5, 5)])
def test_fd_inverts_preconditioner(d, ne, p):
    spaces = [C.Space1D(ne, p) for _ in range(d)]
    P = C.assemble_preconditioner(spaces)
    fd = F.FD(spaces)
    b = np.random.default_rng(1).standard_normal(P.shape[0])
    assert np.linalg.norm(fd(P @ b) - b) < 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("d,ne,p", [(2, 5, 3), (3, 3, 3), (3, 4, 2)])
def test_fd_matches_dense_kronecker_solve(d, ne, p):
    spaces = [C.Space1D(ne + l, p) for l in range(d)]  # unequal n per direction
    Pd = np.zeros((1, 1))
    for l in range(d):
        mats = [spaces[j].K if j == l else spaces[j].M for j in range(d)]
        term = np.ones((1, 1))
        for A in mats:
            term = np.kron(A, term)
        Pd = term if l == 0 else Pd + term
    b = np.random.default_rng(2).standard_normal(Pd.shape[0])
    ref = np.linalg.solve(Pd, b)
    got = F.FD(spaces)(b)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


def test_fd_invariant_under_eigenvector_scaling():
    spaces = [C.Space1D(7, 3), C.Space1D(7, 3)]
    fd = F.FD(spaces)
    b = np.random.default_rng(3).standard_normal(fd.D.size)
    s0 = fd(b)
    rng = np.random.default_rng(4)
    for l in range(2):
        scale = rng.uniform(0.5, 2.0, fd.U[l].shape[1]) * rng.choice([-1, 1], fd.U[l].shape[1])
        fd.U[l] = fd.U[l] * scale
        fd.V[l] = np.linalg.inv(spaces[l].M @ fd.U[l]).T
    assert np.linalg.norm(fd(b) - s0) < 1e-13 * np.linalg.norm(s0)


def test_symmetric_pencil_gives_V_equal_U():
    # Sec. 4: for symmetric K and SPD M with M-orthonormal U, V = (M U)^{-T} = U.
    rng = np.random.default_rng(5)
    X = rng.standard_normal((6, 6))
    M = X @ X.T + 6 * np.eye(6)
    Y = rng.standard_normal((6, 6))
    K = Y + Y.T
    lam, U, V = F.eig_factors(K, M, cond_max=1e6)
    Um = U / np.sqrt(np.einsum("ij,ij->j", U, M @ U))
    Vm = np.linalg.inv(M @ Um).T
    assert np.max(np.abs(Vm - Um)) < 1e-12


def test_identity_geometry_converges_in_one_iteration():
    spaces = [C.Space1D(8, 3), C.Space1D(8, 3)]
    A = C.assemble_collocation(spaces, Geo.Identity(2))
    fd = F.FD(spaces)
    b = np.random.default_rng(6).standard_normal(A.shape[0])
    r = G.gmres(A, b, M=fd, tol=1e-8, max_iter=20)
    assert r["iters"] == 1 and r["relres_true"] < 1e-12


def _annulus_system(ne, p, d=2):
    fmap = Geo.QuarterAnnulus(1, 2) if d == 2 else Geo.ExtrudedAnnulus(1, 2)
    spaces = [C.Space1D(ne, p) for _ in range(d)]
    A = C.assemble_collocation(spaces, fmap)
    pts = C.physical_points(fmap, [s.tau for s in spaces])
    return spaces, A, W.manufactured_f(pts)


def test_kth_iterate_is_krylov_least_squares_minimizer():
    spaces, A, b = _annulus_system(6, 3)
    fd = F.FD(spaces)
    Ad = A.toarray()
    for k in (1, 2, 4, 7):
        r = G.gmres(A, b, M=fd, tol=0.0, max_iter=k)
        # brute force: basis of K_k(A M^{-1}, b), minimize ||b - A M^{-1} K y||
        AM = np.column_stack([Ad @ fd(e) for e in np.eye(A.shape[0])])
        Kry = np.column_stack([np.linalg.matrix_power(AM, j) @ b for j in range(k)])
        Q, _ = np.linalg.qr(Kry)
        y, *_ = np.linalg.lstsq(AM @ Q, b, rcond=None)
        x_ref = fd(Q @ y)
        assert np.linalg.norm(r["x"] - x_ref) < 1e-9 * np.linalg.norm(x_ref)


def test_exact_after_N_iterations_and_monotone_history():
    spaces, A, b = _annulus_system(3, 2)
    r = G.gmres(A, b, M=None, tol=0.0, max_iter=A.shape[0])
    x = spl.spsolve(A.tocsc(), b)
    assert np.linalg.norm(r["x"] - x) < 1e-10 * np.linalg.norm(x)
    assert np.all(np.diff(r["hist"]) <= 1e-14)


def test_flexible_matches_standard_for_fixed_preconditioner():
    spaces, A, b = _annulus_system(10, 3)
    fd = F.FD(spaces)
    r1 = G.gmres(A, b, M=fd, tol=1e-10, max_iter=60)
    r2 = G.gmres(A, b, M=fd, tol=1e-10, max_iter=60, flexible=True)
    assert r1["iters"] == r2["iters"]
    assert np.linalg.norm(r1["x"] - r2["x"]) < 1e-10 * np.linalg.norm(r1["x"])


def test_history_is_true_residual_for_right_preconditioning():
    spaces, A, b = _annulus_system(10, 3)
    fd = F.FD(spaces)
    r = G.gmres(A, b, M=fd, tol=1e-8, max_iter=60)
    assert r["relres_true"] < 1.5e-8
    assert abs(r["hist"][-1] - r["relres_true"]) < 1e-9


def test_iteration_counts_flat_in_h_for_fd_and_growing_without():
    its_fd, its_none = [], []
    for ne in (8, 16, 32):
        spaces, A, b = _annulus_system(ne, 3)
        its_fd.append(G.gmres(A, b, M=F.FD(spaces), tol=1e-8, max_iter=200)["iters"])
        its_none.append(G.gmres(A, b, M=None, tol=1e-8, max_iter=2000)["iters"])
    assert max(its_fd) - min(its_fd) <= 4
    assert its_none[2] > 1.5 * its_none[0]
    assert all(f < u for f, u in zip(its_fd, its_none))


def test_preconditioned_spectrum_lies_near_symbol_range():
    # soft check (bound of eq. bound / symbol analysis cited in Sec. 3): the
    # eigenvalues of P^{-1} A_C on the annulus r in [1,2] have real parts in
    # roughly [min(1, 4/(pi^2 r^2)), 1]; report loosely.
    spaces, A, _ = _annulus_system(6, 3)
    P = C.assemble_preconditioner(spaces).toarray()
    ev = np.linalg.eigvals(np.linalg.solve(P, A.toarray()))
    assert ev.real.min() > 0.05 and ev.real.max() < 1.5
