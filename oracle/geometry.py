"""Single-patch geometry maps F : [0,1]^d -> Omega and the pulled-back operator.

Paper, Sec. 2.1: Omega = F([0,1]^d).  Sec. 2.2: the collocation operator is
L u = -div(K grad u) with K = I (the tests of Sec. 5 set K = I_d); the paper
does not print A_C for a general F ("complicated, we do not report it").

Reading used here (written out in ``pullback_coefficients``): with u = u_hat o F^{-1},
J = dF/dxi (J[k, a] = d F_k / d xi_a) and G = J^{-1} J^{-T},

    -Lap_x u = - sum_{a,b} G^{ab} d_a d_b u_hat  -  sum_c L_c d_c u_hat,
    L_c = Lap_x(xi_c) = - sum_k (J^{-1})_{ck} sum_{a,b} G^{ab} d_a d_b F_k.

(The second line follows from applying Lap_x to the identity x_k = F_k(xi(x)).)

Maps provided, each with an analytic Jacobian and Hessian:
* identity on [0,1]^d (Sec. 2.2 special case: A_C is then eq. colloc2D / colloc3D);
* quarter annulus  x = r cos(pi eta/2), y = r sin(pi eta/2), r = r0 + (r1 - r0) xi
  (Sec. 5 "quarter of ring"; radii r0, r1 are inputs because the figure is lost);
* the extruded thick quarter annulus in 3D (z = zeta);
* the revolved quarter ring of Sec. 5: the 2D ring in the plane z = 0 turned by
  pi/2 * zeta about the axis through (-1,-1,-1) with direction (0,1,0).
"""

import numpy as np


class Map:
    """Analytic map with F(xi), J(xi) (d x d) and Hess(xi) (d x d x d, [k, a, b]).

    ``xi`` may also be an array of shape (d, ...) holding many points; the results then
    carry the same trailing axes (F: (d, ...), J: (d, d, ...), H: (d, d, d, ...)).
    """

    d = 0

    def F(self, xi):
        raise NotImplementedError

    def J(self, xi):
        raise NotImplementedError

    def H(self, xi):
        raise NotImplementedError


class Identity(Map):
    def __init__(self, d):
        self.d = d

    def F(self, xi):
        return np.array(xi, dtype=np.float64)

    def J(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        out = np.zeros((self.d, self.d) + xi.shape[1:])
        for a in range(self.d):
            out[a, a] = 1.0
        return out

    def H(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        return np.zeros((self.d, self.d, self.d) + xi.shape[1:])


class QuarterAnnulus(Map):
    """2D quarter ring r0 <= r <= r1 in the first quadrant; xi radial, eta angular."""

    d = 2

    def __init__(self, r0=1.0, r1=2.0):
        self.r0, self.r1 = float(r0), float(r1)

    def F(self, xi):
        r = self.r0 + (self.r1 - self.r0) * xi[0]
        th = 0.5 * np.pi * xi[1]
        return np.array([r * np.cos(th), r * np.sin(th)])

    def J(self, xi):
        R = self.r1 - self.r0
        r = self.r0 + R * np.asarray(xi[0], dtype=np.float64)
        th = 0.5 * np.pi * np.asarray(xi[1], dtype=np.float64)
        w = 0.5 * np.pi
        return np.array([[R * np.cos(th), -r * w * np.sin(th)],
                         [R * np.sin(th), r * w * np.cos(th)]])

    def H(self, xi):
        R = self.r1 - self.r0
        r = self.r0 + R * np.asarray(xi[0], dtype=np.float64)
        th = 0.5 * np.pi * np.asarray(xi[1], dtype=np.float64)
        w = 0.5 * np.pi
        h = np.zeros((2, 2, 2) + np.shape(th))
        # F_x = r cos(th): d_xi d_eta = -R w sin, d_eta d_eta = -r w^2 cos
        h[0, 0, 1] = h[0, 1, 0] = -R * w * np.sin(th)
        h[0, 1, 1] = -r * w * w * np.cos(th)
        # F_y = r sin(th)
        h[1, 0, 1] = h[1, 1, 0] = R * w * np.cos(th)
        h[1, 1, 1] = -r * w * w * np.sin(th)
        return h


class ExtrudedAnnulus(Map):
    """Quarter annulus times [0,1] in z (z = zeta)."""

    d = 3

    def __init__(self, r0=1.0, r1=2.0):
        self.ring = QuarterAnnulus(r0, r1)

    def F(self, xi):
        xy = self.ring.F(xi[:2])
        return np.array([xy[0], xy[1], np.asarray(xi[2], dtype=np.float64)])

    def J(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        j = np.zeros((3, 3) + xi.shape[1:])
        j[:2, :2] = self.ring.J(xi[:2])
        j[2, 2] = 1.0
        return j

    def H(self, xi):
        xi = np.asarray(xi, dtype=np.float64)
        h = np.zeros((3, 3, 3) + xi.shape[1:])
        h[:2, :2, :2] = self.ring.H(xi[:2])
        return h


class RevolvedAnnulus(Map):
    """Sec. 5: the quarter ring (z = 0 plane) revolved by angle phi = (pi/2) zeta
    about the axis through c = (-1,-1,-1) with direction (0,1,0).

    Rotation about the y-axis through c: with (X, Y) = ring(xi, eta) and
    a = X - c_x, b = 0 - c_z,
        x = c_x + a cos(phi) + b sin(phi),  y = Y,  z = c_z - a sin(phi) + b cos(phi).
    """

    d = 3

    def __init__(self, r0=1.0, r1=2.0, center=(-1.0, -1.0, -1.0)):
        self.ring = QuarterAnnulus(r0, r1)
        self.c = np.array(center, dtype=np.float64)

    def F(self, xi):
        X, Y = self.ring.F(xi[:2])
        phi = 0.5 * np.pi * xi[2]
        a = X - self.c[0]
        b = 0.0 - self.c[2]
        return np.array([self.c[0] + a * np.cos(phi) + b * np.sin(phi),
                         Y * np.ones_like(phi),
                         self.c[2] - a * np.sin(phi) + b * np.cos(phi)])

    def J(self, xi):
        X, _ = self.ring.F(xi[:2])
        jr = self.ring.J(xi[:2])
        phi = 0.5 * np.pi * xi[2]
        w = 0.5 * np.pi
        a = X - self.c[0]
        b = 0.0 - self.c[2]
        c, s = np.cos(phi), np.sin(phi)
        j = np.zeros((3, 3) + np.shape(phi))
        j[0, 0:2] = c * jr[0, :]
        j[1, 0:2] = jr[1, :]
        j[2, 0:2] = -s * jr[0, :]
        j[0, 2] = w * (-a * s + b * c)
        j[1, 2] = 0.0
        j[2, 2] = w * (-a * c - b * s)
        return j

    def H(self, xi):
        X, _ = self.ring.F(xi[:2])
        jr = self.ring.J(xi[:2])
        hr = self.ring.H(xi[:2])
        phi = 0.5 * np.pi * xi[2]
        w = 0.5 * np.pi
        a = X - self.c[0]
        b = 0.0 - self.c[2]
        c, s = np.cos(phi), np.sin(phi)
        h = np.zeros((3, 3, 3) + np.shape(phi))
        h[0, :2, :2] = c * hr[0]
        h[1, :2, :2] = hr[1]
        h[2, :2, :2] = -s * hr[0]
        # mixed (xi_a, zeta): d/dzeta of c*jr[0,a] etc.
        for a_ in range(2):
            h[0, a_, 2] = h[0, 2, a_] = -w * s * jr[0, a_]
            h[2, a_, 2] = h[2, 2, a_] = -w * c * jr[0, a_]
        h[0, 2, 2] = w * w * (-a * c - b * s)
        h[2, 2, 2] = w * w * (a * s - b * c)
        return h


def make_map(kind, d, r0=1.0, r1=2.0):
    """kind: 'identity', 'annulus' (2D quarter ring / 3D extruded), 'revolved' (3D)."""
    if kind == "identity":
        return Identity(d)
    if kind == "annulus":
        return QuarterAnnulus(r0, r1) if d == 2 else ExtrudedAnnulus(r0, r1)
    if kind == "revolved":
        if d != 3:
            raise ValueError("revolved ring is 3D")
        return RevolvedAnnulus(r0, r1)
    raise ValueError(kind)


def pullback_coefficients(fmap, xi):
    """Coefficients of -Lap_x (u_hat o F^{-1}) at the parametric point xi.

    Returns (G, Lvec): G = J^{-1} J^{-T} (symmetric d x d) and
    Lvec[c] = -sum_k (J^{-1})_{ck} sum_{a,b} G^{ab} H[k, a, b], so that
        -Lap_x u = -sum_{a,b} G[a,b] d_a d_b u_hat - sum_c Lvec[c] d_c u_hat.
    """
    J = fmap.J(xi)
    Ji = np.linalg.inv(J)
    G = Ji @ Ji.T
    H = fmap.H(xi)
    lap_F = np.einsum("ab,kab->k", G, H)
    Lvec = -Ji @ lap_F
    return G, Lvec


def wind_coefficients(fmap, xi, wind):
    """Coefficients of the convective term w . grad_x (u_hat o F^{-1}) of eq. (convection)
    (Sec. 3.2) at the parametric point xi, for a constant wind w: grad_x u = J^{-T}
    grad_xi u_hat, so w . grad_x u = sum_c (J^{-1} w)_c d_c u_hat.  Returns J^{-1} w."""
    return np.linalg.solve(fmap.J(xi), np.asarray(wind, dtype=np.float64))


def annulus_closed_form(r0, r1, xi):
    """Polar form of -Lap for the quarter annulus (pin for ``pullback_coefficients``):
    -Lap u = -(1/R^2) u_xixi - 1/(R r) u_xi - 4/(pi^2 r^2) u_etaeta, R = r1 - r0."""
    R = r1 - r0
    r = r0 + R * xi[0]
    G = np.array([[1.0 / R**2, 0.0], [0.0, 4.0 / (np.pi**2 * r * r)]])
    L = np.array([1.0 / (R * r), 0.0])
    return G, L


# ----------------------------------------------------------------- many points at once
# The same formulas as ``pullback_coefficients`` / ``wind_coefficients``, evaluated for an
# array of parametric points (the maps broadcast over trailing axes).  Used to build the
# coefficient fields of large problems in seconds; pinned point by point against the
# single-point functions above.

def pullback_coefficients_many(fmap, xis):
    """xis: (N, d) parametric points.  Returns G (N, d, d) and Lvec (N, d), the same
    quantities as ``pullback_coefficients`` at each point."""
    X = np.asarray(xis, dtype=np.float64).T            # (d, N)
    J = np.moveaxis(fmap.J(X), -1, 0)                 # (N, d, d)
    H = np.moveaxis(fmap.H(X), -1, 0)                 # (N, d, d, d)
    Ji = np.linalg.inv(J)
    G = Ji @ np.swapaxes(Ji, 1, 2)
    lap_F = np.einsum("nab,nkab->nk", G, H)
    Lvec = -np.einsum("nck,nk->nc", Ji, lap_F)
    return G, Lvec


def wind_coefficients_many(fmap, xis, wind):
    """J^{-1} w at each of the points xis (N, d), as ``wind_coefficients``."""
    X = np.asarray(xis, dtype=np.float64).T
    J = np.moveaxis(fmap.J(X), -1, 0)
    w = np.broadcast_to(np.asarray(wind, dtype=np.float64), (J.shape[0], J.shape[1]))
    return np.linalg.solve(J, w[..., None])[..., 0]
