"""Weighted-quadrature (WQ) Galerkin discretization of the Poisson problem (Sec. 2.3).

Paper references:
* Galerkin stiffness matrix on the parameter domain (Sec. 2.3):
      (A_G)_{IJ} = sum_{a,b} int_{[0,1]^d} c_ab(xi) d_a B_I(xi) d_b B_J(xi) dxi,
  with the coefficient matrix of eq. (Q), Q = det(J) J^{-1} K J^{-T}, K = I here;
* eq. (WQapprox): A_wq replaces each integral by a quadrature whose weights w^{ab}_{I q}
  absorb the test function's derivative d_a B_I:
      (A_wq)_{IJ} = sum_{a,b} sum_q c_ab(x_q) w^{ab}_{Iq} d_b B_J(x_q);
  the weights are fixed by exactness when the c_ab are constant, so that A_wq = A_G then
  (the paper defers the construction to Calabro, Sangalli, Tani 2017);
* eq. (wq2D) / (wq3D), eq. (univariateWQ): on the identity map A_wq = K2 (x) M1 + M2 (x) K1
  (three terms in 3D) with the univariate Galerkin matrices M_ij = int B_i B_j and
  K_ij = int B_i' B_j', which are symmetric positive definite; the preconditioner P_wq is
  that matrix (Sec. 3, P_wq = P_G), solved by the symmetric FD of Sec. 4.

Readings of what the paper leaves to the cited work (each one written out below):
* the rule is a tensor product of univariate rules, w^{ab}_{Iq} = prod_l w^{(a_l, b_l)}_{i_l q_l}
  with a_l = [l == a], b_l = [l == b]; a univariate rule w^{(s,t)}_{i,q} is exact on the
  spline space: sum_q w^{(s,t)}_{i,q} B_j^{(t)}(x_q) = int_0^1 B_i^{(s)} B_j^{(t)} for every
  basis function B_j (of the full basis) whose support meets that of B_i;
* the weights of row i live on the quadrature points inside the support of B_i and are the
  minimum 2-norm solution of those exactness conditions;
* quadrature points (per direction): every element end point and every element midpoint,
  and in the first and last element p equispaced interior points instead of the midpoint,
  so that each boundary test function has at least as many points as conditions.
"""

import itertools

import numpy as np
import scipy.sparse as sp

from . import bspline
from .collocation import kron_list, tensor_points


def gauss_legendre(k, a, b):
    """k-point Gauss--Legendre nodes and weights on [a, b] (exact for degree 2k - 1)."""
    x, w = np.polynomial.legendre.leggauss(k)
    return 0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w


def element_breaks(n_elem):
    return np.arange(n_elem + 1, dtype=np.float64) / n_elem


def quadrature_points(n_elem, p):
    """WQ quadrature points on [0, 1] (reading above), ascending."""
    br = element_breaks(n_elem)
    pts = list(br)
    for e in range(n_elem):
        a, b = br[e], br[e + 1]
        if e == 0 or e == n_elem - 1:
            pts += list(a + (b - a) * np.arange(1, p + 1) / (p + 1))
        else:
            pts.append(0.5 * (a + b))
    return np.unique(np.array(pts))


class WQSpace1D:
    """One parametric direction of the WQ discretization: knots, the univariate Galerkin
    integrals of the full basis, the quadrature points, the basis (and derivatives) at
    them and the four univariate weight sets W[(s, t)] (rows: interior test functions
    B_1..B_n of eq. space; columns: quadrature points)."""

    def __init__(self, n_elem, p):
        self.n_elem, self.p = n_elem, p
        self.t = bspline.open_uniform_knots(n_elem, p)
        self.m = bspline.num_basis(self.t, p)
        self.n = self.m - 2
        self.xq = quadrature_points(n_elem, p)
        self.nq = self.xq.shape[0]
        # full-basis values and first derivatives at the quadrature points: (nq, m)
        self.Bq_full = [np.array([bspline.basis_all(self.t, p, x, r) for x in self.xq])
                        for r in range(2)]
        # interior trial functions (homogeneous Dirichlet, eq. space): (nq, n)
        self.Bq = [b[:, 1:self.m - 1].copy() for b in self.Bq_full]
        self.G = {(s, t): self.galerkin_full(s, t) for s in (0, 1) for t in (0, 1)}
        self.W = {(s, t): self.weights(s, t) for s in (0, 1) for t in (0, 1)}

    def support(self, j):
        """Closed support [t_j, t_{j+p+1}] of B_j."""
        return self.t[j], self.t[j + self.p + 1]

    def galerkin_full(self, s, t):
        """int_0^1 B_i^{(s)} B_j^{(t)} dx for the full basis (m x m), by Gauss--Legendre with
        p + 1 points per element (the integrand is a polynomial of degree <= 2p there)."""
        br = element_breaks(self.n_elem)
        G = np.zeros((self.m, self.m))
        for e in range(self.n_elem):
            xg, wg = gauss_legendre(self.p + 1, br[e], br[e + 1])
            for x, w in zip(xg, wg):
                bs = bspline.basis_all(self.t, self.p, x, s)
                bt = bspline.basis_all(self.t, self.p, x, t)
                G += w * np.outer(bs, bt)
        return G

    def weights(self, s, t):
        """Univariate weights w^{(s,t)}_{i,q} for the interior test functions i = 1..n
        (full-basis index), minimum-norm exact on every overlapping B_j^{(t)}."""
        W = np.zeros((self.n, self.nq))
        for r, i in enumerate(range(1, self.m - 1)):
            lo, hi = self.support(i)
            q = np.nonzero((self.xq >= lo) & (self.xq <= hi))[0]
            js = [j for j in range(self.m)
                  if self.support(j)[0] < hi and self.support(j)[1] > lo]
            E = self.Bq_full[t][np.ix_(q, js)].T          # conditions x points
            rhs = self.G[(s, t)][i, js]
            w, *_ = np.linalg.lstsq(E, rhs, rcond=None)  # minimum-norm solution
            W[r, q] = w
        return W

    def galerkin(self, s, t):
        """The interior block (n x n) of the univariate Galerkin matrix."""
        return self.G[(s, t)][1:self.m - 1, 1:self.m - 1].copy()

    @property
    def M(self):
        """(M^wq)_ij = int B_i B_j (eq. univariateWQ)."""
        return self.galerkin(0, 0)

    @property
    def K(self):
        """(K^wq)_ij = int B_i' B_j' (eq. univariateWQ)."""
        return self.galerkin(1, 1)


def q_coefficients_many(fmap, xis):
    """Q = det(J) J^{-1} J^{-T} (eq. Q with K = I) at the parametric points xis (N, d):
    shape (N, d, d)."""
    X = np.asarray(xis, dtype=np.float64).T
    J = np.moveaxis(fmap.J(X), -1, 0)
    Ji = np.linalg.inv(J)
    return np.linalg.det(J)[:, None, None] * (Ji @ np.swapaxes(Ji, 1, 2))


def _orders(d, a):
    o = [0] * d
    if a is not None:
        o[a] = 1
    return o


def assemble_wq(spaces, fmap):
    """A_wq in CSR from eq. (WQapprox) with tensor-product weights:
    A_wq = sum_{a,b} (W^{(a_d,b_d)}_d (x) .. (x) W^{(a_1,b_1)}_1) diag(c_ab(x_q))
                     (B^{(b_d)}_d (x) .. (x) B^{(b_1)}_1),  a_l = [l == a], b_l = [l == b]."""
    d = len(spaces)
    pts = tensor_points([s.xq for s in spaces])
    Q = q_coefficients_many(fmap, pts)
    A = None
    for a, b in itertools.product(range(d), range(d)):
        oa, ob = _orders(d, a), _orders(d, b)
        Wk = kron_list([spaces[l].W[(oa[l], ob[l])] for l in range(d)])
        Bk = kron_list([spaces[l].Bq[ob[l]] for l in range(d)])
        term = Wk @ sp.diags(Q[:, a, b]) @ Bk
        A = term if A is None else A + term
    A = A.tocsr()
    A.eliminate_zeros()
    return A


def assemble_galerkin(spaces, fmap, k_extra=2):
    """The exact-integration Galerkin matrix A_G (Sec. 2.3) up to quadrature error:
    tensor Gauss--Legendre with p + 1 + k_extra points per element (exact when Q is a
    polynomial of degree <= 2 k_extra - 1 per element, e.g. constant Q)."""
    d = len(spaces)
    grids, wts, vals = [], [], []
    for s in spaces:
        br = element_breaks(s.n_elem)
        xs, ws = [], []
        for e in range(s.n_elem):
            x, w = gauss_legendre(s.p + 1 + k_extra, br[e], br[e + 1])
            xs.append(x)
            ws.append(w)
        x = np.concatenate(xs)
        grids.append(x)
        wts.append(np.concatenate(ws))
        vals.append([np.array([bspline.basis_all(s.t, s.p, xx, r) for xx in x])[:, 1:s.m - 1]
                     for r in range(2)])
    pts = tensor_points(grids)
    Q = q_coefficients_many(fmap, pts)
    wq = wts[-1]
    for w in reversed(wts[:-1]):
        wq = np.kron(wq, w)
    A = None
    for a, b in itertools.product(range(d), range(d)):
        oa, ob = _orders(d, a), _orders(d, b)
        Ba = kron_list([vals[l][oa[l]] for l in range(d)])
        Bb = kron_list([vals[l][ob[l]] for l in range(d)])
        term = Ba.T @ sp.diags(wq * Q[:, a, b]) @ Bb
        A = term if A is None else A + term
    return A.tocsr()


def galerkin_rhs(spaces, fmap, f, k_extra=2):
    """f_I = int f(F(xi)) B_I(xi) |det J(xi)| dxi by tensor Gauss--Legendre (Sec. 2.3: the
    right-hand side may come from any quadrature); f is a callable on (N, d) points."""
    grids, wts, vals = [], [], []
    for s in spaces:
        br = element_breaks(s.n_elem)
        xs, ws = [], []
        for e in range(s.n_elem):
            x, w = gauss_legendre(s.p + 1 + k_extra, br[e], br[e + 1])
            xs.append(x)
            ws.append(w)
        x = np.concatenate(xs)
        grids.append(x)
        wts.append(np.concatenate(ws))
        vals.append(np.array([bspline.basis_all(s.t, s.p, xx, 0) for xx in x])[:, 1:s.m - 1])
    pts = tensor_points(grids)
    X = pts.T
    detJ = np.abs(np.linalg.det(np.moveaxis(fmap.J(X), -1, 0)))
    phys = np.asarray(fmap.F(X), dtype=np.float64).T
    wq = wts[-1]
    for w in reversed(wts[:-1]):
        wq = np.kron(wq, w)
    Bk = kron_list(vals)
    return Bk.T @ (wq * detJ * f(phys))


def assemble_preconditioner_wq(spaces):
    """P_wq = P_G: eq. (wq2D) / (wq3D) with the univariate Galerkin factors."""
    d = len(spaces)
    P = None
    for l in range(d):
        term = kron_list([spaces[j].K if j == l else spaces[j].M for j in range(d)])
        P = term if P is None else P + term
    return P.tocsr()


def quadrature_points_physical(spaces, fmap):
    """F(x_q) on the tensor grid of WQ quadrature points (direction 1 fastest): (Nq, d)."""
    return np.asarray(fmap.F(tensor_points([s.xq for s in spaces]).T), dtype=np.float64).T.copy()


def wq_load(spaces, fmap, g):
    """The WQ load vector (Sec. 2.3, the right-hand side 'by using again the WQ approach'):
    f_I = sum_q w^{00}_{I q} |det J(x_q)| g_q for source values g at the quadrature points,
    the tensor-product rule applied mode by mode (the Kronecker identity)."""
    from .fd import kron_apply
    pts = tensor_points([s.xq for s in spaces])
    detJ = np.abs(np.linalg.det(np.moveaxis(fmap.J(pts.T), -1, 0)))
    shape_q = tuple(s.nq for s in spaces)[::-1]
    return kron_apply([s.W[(0, 0)] for s in spaces], detJ * np.asarray(g, dtype=np.float64),
                      shape_q)


class WQOperator:
    """A_wq applied without assembling it: the sum of eq. (WQapprox) written as
    W_ab diag(Q_ab) B_b u per term (a, b), each tensor product applied mode by mode
    (the Kronecker identity), for problems too large to assemble quickly."""

    def __init__(self, spaces, fmap):
        from .fd import kron_apply
        self._kron_apply = kron_apply
        self.spaces = spaces
        self.d = len(spaces)
        self.shape_n = tuple(s.n for s in spaces)[::-1]
        self.shape_q = tuple(s.nq for s in spaces)[::-1]
        pts = tensor_points([s.xq for s in spaces])
        self.Q = q_coefficients_many(fmap, pts)

    def __call__(self, u):
        u = np.asarray(u, dtype=np.float64)
        out = np.zeros_like(u)
        d = self.d
        for a, b in itertools.product(range(d), range(d)):
            oa, ob = _orders(d, a), _orders(d, b)
            y = self._kron_apply([self.spaces[l].Bq[ob[l]] for l in range(d)], u, self.shape_n)
            y = self.Q[:, a, b] * y
            out += self._kron_apply([self.spaces[l].W[(oa[l], ob[l])] for l in range(d)], y,
                                    self.shape_q)
        return out
