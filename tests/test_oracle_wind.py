"""Pins of the convection--diffusion extension of the oracle (Sec. 3.2, collocation form,
constant wind w): L_w = -Lap + w . grad, preconditioner factors K_l + H_l = -B'' + w_l B'.

* the 1D pencil (K + w B', M) has the spectrum of -u'' + w u' with homogeneous Dirichlet
  conditions, lambda_k = (k pi)^2 + w^2 / 4 (closed form; the smallest eigenvalue to 1e-3);
* for the identity map with a constant wind, A_C = P_C (the preconditioner is exact);
* the convective term of A_C applied to a spline against finite differences of the
  composed function u o F^{-1} in physical space (quarter ring, explicit inverse map);
* the FD solve inverts P_C with the wind, and GMRES with it converges in one step on
  the identity map.
"""

import numpy as np
import pytest

from oracle import collocation as C, fd as F, geometry as Geo, gmres as G


@pytest.mark.parametrize("w", [1.0, 5.0, 10.0, -5.0])
def test_1d_spectrum_closed_form(w):
    s = C.Space1D(64, 5)
    lam, U, V = F.eig_factors(C.wind_factor(s, w), s.M)
    assert abs(lam[0] - (np.pi ** 2 + w * w / 4)) <= 1e-3 * lam[0]
    assert abs(lam[1] - (4 * np.pi ** 2 + w * w / 4)) <= 1e-3 * lam[1]


@pytest.mark.parametrize("d", [2, 3])
def test_identity_map_operator_equals_preconditioner(d):
    spaces = [C.Space1D(5, 3) for _ in range(d)]
    wind = [3.0, -2.0, 1.5][:d]
    fmap = Geo.make_map("identity", d)
    A = C.assemble_collocation(spaces, fmap, wind)
    P = C.assemble_preconditioner(spaces, wind)
    assert abs(A - P).max() <= 1e-12 * abs(P).max()
    b = np.random.default_rng(d).standard_normal(A.shape[0])
    fd = F.FD(spaces, wind)
    assert np.linalg.norm(fd(P @ b) - b) <= 1e-10 * np.linalg.norm(b)
    r = G.gmres(A, b, M=fd, tol=1e-10, max_iter=10)
    assert r["iters"] == 1


def test_convective_term_against_finite_differences():
    # spline u_hat with random coefficients on the quarter ring; the difference of A_C
    # with and without wind is the convective term (J^-1 w)_c d_c u_hat at tau_I, which
    # must equal w . grad_x (u_hat o F^-1) computed by central differences in x, y
    r0, r1 = 1.0, 2.0
    spaces = [C.Space1D(6, 3) for _ in range(2)]
    fmap = Geo.make_map("annulus", 2, r0, r1)
    wind = np.array([2.0, -1.0])
    A0 = C.assemble_collocation(spaces, fmap)
    Aw = C.assemble_collocation(spaces, fmap, wind)
    c = np.random.default_rng(7).standard_normal(A0.shape[0])
    conv = (Aw - A0) @ c

    from oracle import bspline

    def u_hat(xi, eta):
        bx = bspline.basis_all(spaces[0].t, 3, xi, 0)[1:-1]
        by = bspline.basis_all(spaces[1].t, 3, eta, 0)[1:-1]
        return np.kron(by, bx) @ c

    def u_phys(x, y):
        r = np.hypot(x, y)
        return u_hat((r - r0) / (r1 - r0), np.arctan2(y, x) * 2 / np.pi)

    pts = C.tensor_points([s.tau for s in spaces])
    h = 1e-6
    for I in [7, 11, 20, 30]:
        X, Y = fmap.F(pts[I])
        gx = (u_phys(X + h, Y) - u_phys(X - h, Y)) / (2 * h)
        gy = (u_phys(X, Y + h) - u_phys(X, Y - h)) / (2 * h)
        want = wind[0] * gx + wind[1] * gy
        assert abs(conv[I] - want) <= 1e-6 * (1 + abs(want)), I
