"""Pins for oracle.geometry and oracle.collocation.

* the maps' analytic Jacobian and Hessian against finite differences of F;
* the general pull-back formula against the polar closed form on the annulus;
* A_C = P_C on the identity map (Sec. 2.2, eqs. colloc2D/colloc3D with Sec. 3);
* A_C applied to the exact spline coefficients of a polynomial u_hat equals the
  closed-form -Lap u at F(tau) (catches transposed Kronecker order, wrong signs,
  dropped first-order terms);
* the hand-derived manufactured forcing against a finite-difference Laplacian;
* observed collocation convergence order >= p - 1 (Sec. 2.2 scheme, order reading).
"""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl

import workload as W
from oracle import bspline, collocation as C, geometry as Geo

MAPS = [Geo.QuarterAnnulus(1.0, 2.0), Geo.QuarterAnnulus(0.5, 1.5),
        Geo.ExtrudedAnnulus(1.0, 2.0), Geo.RevolvedAnnulus(1.0, 2.0), Geo.Identity(3)]


@pytest.mark.parametrize("fmap", MAPS, ids=lambda m: type(m).__name__)
def test_jacobian_and_hessian_match_finite_differences(fmap):
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(5):
        xi = rng.uniform(0.1, 0.9, fmap.d)
        J = fmap.J(xi)
        H = fmap.H(xi)
        for a in range(fmap.d):
            e = np.zeros(fmap.d)
            e[a] = h
            fd1 = (fmap.F(xi + e) - fmap.F(xi - e)) / (2 * h)
            assert np.max(np.abs(fd1 - J[:, a])) < 1e-8
            fdJ = (fmap.J(xi + e) - fmap.J(xi - e)) / (2 * h)
            for b in range(fmap.d):
                assert np.max(np.abs(fdJ[:, b] - H[:, b, a])) < 1e-7


@pytest.mark.parametrize("r0,r1", [(1.0, 2.0), (0.5, 1.5), (1.5, 2.5)])
def test_pullback_matches_polar_closed_form(r0, r1):
    fmap = Geo.QuarterAnnulus(r0, r1)
    for xi in np.random.default_rng(0).uniform(0, 1, (20, 2)):
        G, L = Geo.pullback_coefficients(fmap, xi)
        Gc, Lc = Geo.annulus_closed_form(r0, r1, xi)
        assert np.max(np.abs(G - Gc)) < 1e-14
        assert np.max(np.abs(L - Lc)) < 1e-14


def test_extruded_pullback_adds_zz():
    fmap = Geo.ExtrudedAnnulus(1.0, 2.0)
    xi = np.array([0.3, 0.6, 0.2])
    G, L = Geo.pullback_coefficients(fmap, xi)
    Gc, Lc = Geo.annulus_closed_form(1.0, 2.0, xi[:2])
    assert np.max(np.abs(G[:2, :2] - Gc)) < 1e-14
    assert G[2, 2] == 1.0 and np.all(G[2, :2] == 0) and L[2] == 0.0


def test_revolved_pullback_is_laplacian_of_inverse_map():
    # L_c = Lap_x xi_c; check with a finite-difference Laplacian of F^{-1} around a point.
    fmap = Geo.RevolvedAnnulus(1.0, 2.0)
    xi0 = np.array([0.4, 0.3, 0.7])
    G, L = Geo.pullback_coefficients(fmap, xi0)
    x0 = fmap.F(xi0)

    def inv(x, guess):
        xi = guess.copy()
        for _ in range(30):
            xi = xi - np.linalg.solve(fmap.J(xi), fmap.F(xi) - x)
        return xi

    h = 1e-3
    lap = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lap += (inv(x0 + e, xi0) - 2 * xi0 + inv(x0 - e, xi0)) / h**2
    assert np.max(np.abs(lap - L)) < 1e-5
    Ji = np.linalg.inv(fmap.J(xi0))
    assert np.max(np.abs(G - Ji @ Ji.T)) < 1e-14


@pytest.mark.parametrize("d,p", [(2, 2), (2, 3), (2, 5), (3, 3), (3, 4)])
def test_identity_map_A_equals_P(d, p):
    spaces = [C.Space1D(5, p) for _ in range(d)]
    A = C.assemble_collocation(spaces, Geo.Identity(d))
    P = C.assemble_preconditioner(spaces)
    assert abs(A - P).max() <= 1e-13 * abs(P).max()


def _spline_coeffs_1d(space, fun):
    """Interior coefficients of the spline interpolant of ``fun`` at the full Greville
    points (exact when fun is a polynomial of degree <= p vanishing at 0 and 1)."""
    xs = bspline.greville_full(space.t, space.p)
    Bf = np.array([bspline.basis_all(space.t, space.p, x, 0) for x in xs])
    c = sla.solve(Bf, fun(xs))
    assert abs(c[0]) < 1e-12 and abs(c[-1]) < 1e-12
    return c[1:-1]


@pytest.mark.parametrize("p", [2, 3, 4])
def test_operator_on_exact_polynomial_2d(p):
    # u_hat(xi, eta) = a(xi) b(eta), polynomials of degree <= 2 (in the space for p >= 2),
    # deliberately non-symmetric so a transposed Kronecker order fails.
    a = lambda s: s * (1 - s)
    a1 = lambda s: 1 - 2 * s
    a2 = lambda s: -2.0 + 0 * s
    b = lambda s: 3 * s * (1 - s)
    b2 = lambda s: -6.0 + 0 * s
    r0, r1 = 1.0, 2.0
    fmap = Geo.QuarterAnnulus(r0, r1)
    sp1, sp2 = C.Space1D(6, p), C.Space1D(7, p)
    A = C.assemble_collocation([sp1, sp2], fmap)
    coef = np.kron(_spline_coeffs_1d(sp2, b), _spline_coeffs_1d(sp1, a))
    pts = C.tensor_points([sp1.tau, sp2.tau])
    xi, eta = pts[:, 0], pts[:, 1]
    R = r1 - r0
    r = r0 + R * xi
    ref = -(a2(xi) * b(eta)) / R**2 - a1(xi) * b(eta) / (R * r) \
        - 4.0 / (np.pi**2 * r * r) * a(xi) * b2(eta)
    got = A @ coef
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_operator_on_exact_polynomial_3d():
    p = 3
    fa = [lambda s: s * (1 - s), lambda s: s * (1 - s) ** 2, lambda s: s * s * (1 - s)]
    fd1 = lambda s: 1 - 2 * s
    fd2 = [lambda s: -2.0 + 0 * s, lambda s: -4.0 + 6 * s, lambda s: 2.0 - 6 * s]
    fmap = Geo.ExtrudedAnnulus(1.0, 2.0)
    spaces = [C.Space1D(4, p), C.Space1D(5, p), C.Space1D(6, p)]
    A = C.assemble_collocation(spaces, fmap)
    coef = np.kron(_spline_coeffs_1d(spaces[2], fa[2]),
                   np.kron(_spline_coeffs_1d(spaces[1], fa[1]), _spline_coeffs_1d(spaces[0], fa[0])))
    pts = C.tensor_points([s.tau for s in spaces])
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    r = 1.0 + x
    uxx = fd2[0](x) * fa[1](y) * fa[2](z)
    ux = fd1(x) * fa[1](y) * fa[2](z)
    uyy = fa[0](x) * fd2[1](y) * fa[2](z)
    uzz = fa[0](x) * fa[1](y) * fd2[2](z)
    ref = -uxx - ux / r - 4.0 / (np.pi**2 * r * r) * uyy - uzz
    got = A @ coef
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("d", [2, 3])
def test_manufactured_forcing_matches_finite_differences(d):
    rng = np.random.default_rng(5)
    fmap = Geo.QuarterAnnulus(1, 2) if d == 2 else Geo.ExtrudedAnnulus(1, 2)
    pts = np.array([fmap.F(x) for x in rng.uniform(0.05, 0.95, (15, d))])
    h = 1e-4
    lap = np.zeros(len(pts))
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        lap += (W.manufactured_u(pts + e) - 2 * W.manufactured_u(pts) + W.manufactured_u(pts - e)) / h**2
    f = W.manufactured_f(pts)
    assert np.max(np.abs(-lap - f)) < 1e-5 * max(1.0, np.max(np.abs(f)))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_collocation_convergence_order(p):
    fmap = Geo.QuarterAnnulus(1.0, 2.0)
    errs = []
    nes = [8, 16, 32]
    for ne in nes:
        spaces = [C.Space1D(ne, p), C.Space1D(ne, p)]
        A = C.assemble_collocation(spaces, fmap)
        pts = C.physical_points(fmap, [s.tau for s in spaces])
        u = spl.spsolve(A.tocsc(), W.manufactured_f(pts))
        # evaluate the discrete solution at the collocation points: (M2 (x) M1) u
        uh = C.kron_list([spaces[0].M, spaces[1].M]) @ u
        errs.append(np.max(np.abs(uh - W.manufactured_u(pts))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= p - 1 - 0.2, (errs, orders)


@pytest.mark.parametrize("kind,d", [("annulus", 2), ("annulus", 3), ("revolved", 3)])
def test_collocation_rows_match_assembly(kind, d):
    fmap = Geo.make_map(kind, d)
    spaces = [C.Space1D(4, 3) for _ in range(d)]
    A = C.assemble_collocation(spaces, fmap).toarray()
    rows = [0, 5, A.shape[0] - 1, A.shape[0] // 2]
    R = C.collocation_rows(spaces, fmap, rows)
    assert np.max(np.abs(R - A[rows])) < 1e-13 * np.max(np.abs(A))


# ---------------------------------------------------------------- whole-grid evaluation
@pytest.mark.parametrize("kind,d", [("identity", 2), ("identity", 3), ("annulus", 2),
                                    ("annulus", 3), ("revolved", 3)])
def test_many_point_geometry_matches_point_by_point(kind, d):
    """pullback_coefficients_many / wind_coefficients_many / physical_points_grid evaluate
    the same formulas on arrays of points: equal to the single-point functions (which the
    closed-form and finite-difference pins above check)."""
    fmap = Geo.make_map(kind, d, 0.8, 1.9)
    xs = np.random.default_rng(5).uniform(size=(40, d))
    G, L = Geo.pullback_coefficients_many(fmap, xs)
    Wc = Geo.wind_coefficients_many(fmap, xs, [1.5, -2.0, 0.5][:d])
    for i, x in enumerate(xs):
        g, l = Geo.pullback_coefficients(fmap, x)
        assert np.allclose(G[i], g, rtol=1e-13, atol=1e-13)
        assert np.allclose(L[i], l, rtol=1e-13, atol=1e-13)
        assert np.allclose(Wc[i], Geo.wind_coefficients(fmap, x, [1.5, -2.0, 0.5][:d]),
                           rtol=1e-13, atol=1e-13)
    taus = [C.Space1D(4 + l, 2).tau for l in range(d)]
    assert np.array_equal(C.physical_points_grid(fmap, taus), C.physical_points(fmap, taus))


@pytest.mark.parametrize("kind,d,wind", [("annulus", 2, None), ("annulus", 3, None),
                                         ("revolved", 3, None), ("identity", 3, None),
                                         ("annulus", 3, (1.0, -2.0, 3.0))])
def test_matrix_free_operator_equals_assembled(kind, d, wind):
    """CollocationOperator applies the definition of A_C through the Kronecker identity; it
    equals the assembled CSR matrix (pinned above by exact polynomials, the polar form and
    A = P on the identity map) applied to random vectors.  Directions of different sizes
    catch a transposed mode order."""
    spaces = [C.Space1D(5 + l, 3) for l in range(d)]
    fmap = Geo.make_map(kind, d, 1.0, 2.0)
    A = C.assemble_collocation(spaces, fmap, wind)
    op = C.CollocationOperator(spaces, fmap, wind)
    for seed in range(2):
        u = np.random.default_rng(seed).standard_normal(A.shape[0])
        ref_ = A @ u
        assert np.max(np.abs(op(u) - ref_)) <= 1e-13 * np.max(np.abs(ref_))
