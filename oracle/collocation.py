"""Collocation factors, assembled collocation matrix A_C and preconditioner P_C.

Paper references:
* eq. (univariatecolloc): (M_l)_{ij} = B_j(tau_{l,i}), (K_l)_{ij} = -B''_j(tau_{l,i}),
  i, j = 1..n  (interior basis B_1..B_n, eq. space);
* eq. (collocation) / (collocationsystem): row I of A_C is (L B_J)(F(tau_I));
* eq. (space): scalar index i = 1 + sum_l n^{l-1} (i_l - 1), i.e. i_1 runs fastest,
  so a tensor product "D_d (x) ... (x) D_1" is numpy ``kron(D_d, ..., D_1)``;
* eq. (colloc2D) / (colloc3D) and Sec. 3: P_C = K2 (x) M1 + M2 (x) K1 (2D) and the
  three-term sum in 3D.
* Sec. 3.2 (convection--diffusion, eq. convection / convec_prec_2), restated for
  collocation with a constant wind w: the operator gains + sum_c (J^{-1} w)_c d_c, and
  the preconditioner's factors K_l become K_l + H_l with H_l = w_l B'_l (the collocation
  counterpart of the paper's H_l with the univariate wind approximation w~_l = w_l).
"""

import itertools

import numpy as np
import scipy.sparse as sp

from . import bspline
from .fd import kron_apply
from .geometry import (pullback_coefficients, pullback_coefficients_many, wind_coefficients,
                       wind_coefficients_many)


class Space1D:
    """One parametric direction: knots, Greville points and the three n x n
    collocation matrices B0 = M, B1 = B', B2 = B'' (K = -B2)."""

    def __init__(self, n_elem, p):
        self.n_elem, self.p = n_elem, p
        self.t = bspline.open_uniform_knots(n_elem, p)
        self.m = bspline.num_basis(self.t, p)
        self.n = self.m - 2
        self.tau = bspline.greville_interior(self.t, p)
        full = [np.array([bspline.basis_all(self.t, p, x, r) for x in self.tau])
                for r in range(3)]
        # drop B_0 and B_{m-1} (homogeneous Dirichlet, eq. space)
        self.B = [f[:, 1:self.m - 1].copy() for f in full]

    @property
    def M(self):
        return self.B[0]

    @property
    def K(self):
        return -self.B[2]


def kron_list(mats):
    """mats[l] acts on direction l+1; returns mats[d-1] (x) ... (x) mats[0] (sparse)."""
    out = sp.csr_matrix(mats[-1])
    for A in reversed(mats[:-1]):
        out = sp.kron(out, sp.csr_matrix(A), format="csr")
    return out


def tensor_points(taus):
    """All parametric collocation points tau_I in scalar order (i_1 fastest):
    array of shape (N, d) with column l = tau_{l, i_l}."""
    d = len(taus)
    grids = np.meshgrid(*taus[::-1], indexing="ij")  # slowest first
    pts = np.stack([g.ravel() for g in grids[::-1]], axis=1)
    assert pts.shape[1] == d
    return pts


def physical_points(fmap, taus):
    """F(tau_I) for every collocation point, shape (N, d)."""
    return np.array([fmap.F(x) for x in tensor_points(taus)])


def physical_points_grid(fmap, taus):
    """``physical_points`` with the map evaluated on all points at once."""
    return np.asarray(fmap.F(tensor_points(taus).T), dtype=np.float64).T.copy()


def coefficient_fields(fmap, taus):
    """G^{ab}(tau_I) and L_c(tau_I) at every collocation point: shapes (N,d,d), (N,d)."""
    pts = tensor_points(taus)
    N, d = pts.shape
    G = np.empty((N, d, d))
    L = np.empty((N, d))
    for i, x in enumerate(pts):
        G[i], L[i] = pullback_coefficients(fmap, x)
    return G, L


def assemble_collocation(spaces, fmap, wind=None):
    """A_C in CSR, from the definition: row I = -sum_{a,b} G^{ab}(tau_I) d_a d_b B_J(tau_I)
    - sum_c L_c(tau_I) d_c B_J(tau_I), with tensor-product B_J (eq. multivariatesplines);
    with a constant wind w (Sec. 3.2) also + sum_c (J^{-1} w)_c(tau_I) d_c B_J(tau_I).

    The derivative multi-index (e_1, .., e_d) picks the 1D matrix B[e_l] in direction l.
    """
    d = len(spaces)
    G, L = coefficient_fields(fmap, [s.tau for s in spaces])
    if wind is not None:
        pts = tensor_points([s.tau for s in spaces])
        Wc = np.array([wind_coefficients(fmap, x, wind) for x in pts])
        L = L - Wc  # the first-order term enters with -L_c
    N = G.shape[0]
    A = sp.csr_matrix((N, N))
    for a, b in itertools.product(range(d), range(d)):
        orders = [0] * d
        orders[a] += 1
        orders[b] += 1
        term = kron_list([spaces[l].B[orders[l]] for l in range(d)])
        A = A - sp.diags(G[:, a, b]) @ term
    for c in range(d):
        orders = [0] * d
        orders[c] = 1
        term = kron_list([spaces[l].B[orders[l]] for l in range(d)])
        A = A - sp.diags(L[:, c]) @ term
    A = A.tocsr()
    A.eliminate_zeros()
    return A


def wind_factor(space, w_l):
    """K_l + H_l of Sec. 3.2 in collocation form: -B'' + w_l B' (w_l = 0: K_l)."""
    return space.K + w_l * space.B[1]


def assemble_preconditioner(spaces, wind=None):
    """P_C from eq. (colloc2D) (d = 2) or eq. (colloc3D) (d = 3): sum over l of the
    Kronecker product with K_l in slot l and M in every other slot; with a wind, K_l is
    K_l + H_l (eq. convec_prec_2)."""
    d = len(spaces)
    w = np.zeros(d) if wind is None else np.asarray(wind, dtype=np.float64)
    P = None
    for l in range(d):
        mats = [wind_factor(spaces[j], w[j]) if j == l else spaces[j].M for j in range(d)]
        term = kron_list(mats)
        P = term if P is None else P + term
    return P.tocsr()


def collocation_rows(spaces, fmap, rows, wind=None):
    """Selected rows of A_C (same definition as ``assemble_collocation``), for
    checking large problems on sampled collocation points.  Returns a dense array
    of shape (len(rows), N)."""
    d = len(spaces)
    ns = [s.n for s in spaces]
    N = int(np.prod(ns))
    out = np.zeros((len(rows), N))
    for r, I in enumerate(rows):
        idx = []
        rem = int(I)
        for l in range(d):
            idx.append(rem % ns[l])
            rem //= ns[l]
        xi = np.array([spaces[l].tau[idx[l]] for l in range(d)])
        G, Lv = pullback_coefficients(fmap, xi)
        if wind is not None:
            Lv = Lv - wind_coefficients(fmap, xi, wind)
        row = np.zeros(N)

        def add(coef, orders):
            vecs = [spaces[l].B[orders[l]][idx[l]] for l in range(d)]
            t = vecs[-1]
            for v in reversed(vecs[:-1]):
                t = np.kron(t, v)
            row[:] -= coef * t

        for a, b in itertools.product(range(d), range(d)):
            orders = [0] * d
            orders[a] += 1
            orders[b] += 1
            add(G[a, b], orders)
        for c in range(d):
            orders = [0] * d
            orders[c] = 1
            add(Lv[c], orders)
        out[r] = row
    return out


class CollocationOperator:
    """A_C applied to a vector without assembling it: the definition used by
    ``assemble_collocation`` (eq. collocation),

        (A_C u)_I = - sum_{a,b} G^{ab}(tau_I) (d_a d_b u_h)(tau_I) - sum_c L_c(tau_I) (d_c u_h)(tau_I),

    where each derivative of u_h = sum_J u_J B_J at the tensor grid of collocation points
    is the Kronecker product of the 1D matrices B[order] (eq. univariatecolloc) applied to
    u, evaluated mode by mode (the Kronecker identity).  With a constant wind (Sec. 3.2)
    the first-order coefficients gain + (J^{-1} w)_c.  For problems whose CSR matrix
    is too large to assemble in reasonable time."""

    def __init__(self, spaces, fmap, wind=None):
        self.spaces = spaces
        self.d = len(spaces)
        self.shape = tuple(s.n for s in spaces)[::-1]
        pts = tensor_points([s.tau for s in spaces])
        G, L = pullback_coefficients_many(fmap, pts)
        if wind is not None:
            L = L - wind_coefficients_many(fmap, pts, wind)
        self.terms = []
        for a, b in itertools.product(range(self.d), range(self.d)):
            orders = [0] * self.d
            orders[a] += 1
            orders[b] += 1
            self.terms.append((G[:, a, b].copy(), orders))
        for c in range(self.d):
            orders = [0] * self.d
            orders[c] = 1
            self.terms.append((L[:, c].copy(), orders))

    def __call__(self, u):
        u = np.asarray(u, dtype=np.float64)
        out = np.zeros_like(u)
        for coef, orders in self.terms:
            mats = [self.spaces[l].B[orders[l]] for l in range(self.d)]
            out -= coef * kron_apply(mats, u, self.shape)
        return out
