"""Fast diagonalization (FD) solve of the preconditioner system P s = b (Sec. 4).

* eq. (eigendecomposition): M_l^{-1} K_l U_l = U_l D_l, computed here as the
  generalized problem K_l u = lambda M_l u with LAPACK (scipy.linalg.eig);
* V_l := (M_l U_l)^{-T}  (Sec. 4, definition after eq. eigendecomposition);
* eq. (FD2D) / (FD3D): s = (U_d (x) .. (x) U_1) (sum_l I (x) D_l (x) I)^{-1}
  (V_d (x) .. (x) V_1)^T b.
* Remark 1: the factorization is assumed to exist with real eigenvalues and a
  well-conditioned U; ``eig_factors`` checks both and raises otherwise.

Normalization reading (the paper leaves it free): columns of U have unit 2-norm and
are sorted by ascending eigenvalue.  The FD result does not depend on either choice.

Reflection reading (Remark 1's double "outlier" eigenvalue): on uniform knots the
factors commute with the flip R (i -> n-1-i): R M R = M, R K R = K.  The pencil then
splits exactly into an even part (v = R v) and an odd part (v = -R v), each solved
by LAPACK on its own; the two outlier eigenvectors fall one in each part, so U stays
well conditioned even though the two eigenvalues agree to rounding.  Pencils without
this symmetry use one generalized eigensolve of the whole pencil.
"""

import numpy as np
import scipy.linalg as sla


class NotDiagonalizable(RuntimeError):
    pass


def reflection_basis(n):
    """Orthonormal E (even: v[i] = v[n-1-i]) and O (odd: v[i] = -v[n-1-i]) with [E O]
    an orthogonal n x n matrix."""
    h = n // 2
    E = np.zeros((n, h + n % 2))
    O = np.zeros((n, h))
    c = 1.0 / np.sqrt(2.0)
    for i in range(h):
        E[i, i] = E[n - 1 - i, i] = c
        O[i, i] = c
        O[n - 1 - i, i] = -c
    if n % 2:
        E[h, h] = 1.0
    return E, O


def is_reflection_symmetric(A, rtol=1e-12):
    return np.max(np.abs(A[::-1, ::-1] - A)) <= rtol * np.max(np.abs(A))


def _eig_real(K, M, imag_tol):
    w, U = sla.eig(K, M)
    if np.any(~np.isfinite(w)):
        raise NotDiagonalizable("infinite generalized eigenvalue")
    if np.max(np.abs(w.imag) / np.maximum(np.abs(w), 1e-300)) > imag_tol:
        raise NotDiagonalizable("complex eigenvalues")
    return w.real, U.real


def eig_factors(K, M, imag_tol=1e-10, cond_max=1e3):
    """Return (lam, U, V) with K U = M U diag(lam), unit-norm ascending columns and
    V = (M U)^{-T}.  Raises NotDiagonalizable when Remark 1's assumptions fail."""
    if is_reflection_symmetric(K) and is_reflection_symmetric(M):
        lams, Us = [], []
        for Q in reflection_basis(K.shape[0]):
            if Q.shape[1] == 0:
                continue
            w, Uq = _eig_real(Q.T @ K @ Q, Q.T @ M @ Q, imag_tol)
            lams.append(w)
            Us.append(Q @ Uq)
        lam = np.concatenate(lams)
        U = np.hstack(Us)
    else:
        lam, U = _eig_real(K, M, imag_tol)
    order = np.argsort(lam, kind="stable")
    lam = lam[order]
    U = U[:, order]
    U = U / np.linalg.norm(U, axis=0, keepdims=True)
    if np.linalg.cond(U) > cond_max:
        raise NotDiagonalizable("ill-conditioned eigenvector matrix")
    V = np.linalg.inv(M @ U).T
    return lam, U, V


def mode_product(T, A, l):
    """Apply matrix A (n_l x n_l) along direction l (0-based) of the tensor T.

    T is stored in numpy C order with axes (i_d, .., i_1), so direction l is axis
    d-1-l.  Result[.., i, ..] = sum_j A[i, j] T[.., j, ..].
    """
    d = T.ndim
    ax = d - 1 - l
    out = np.tensordot(A, T, axes=([1], [ax]))  # new axis 0
    return np.moveaxis(out, 0, ax)


def kron_apply(mats, b, shape):
    """(mats[d-1] (x) .. (x) mats[0]) b via mode products (Kronecker property)."""
    T = b.reshape(shape)
    for l, A in enumerate(mats):
        T = mode_product(T, A, l)
    return T.reshape(-1)


class FD:
    """The FD preconditioner for P = sum_l M (x) .. K_l .. (x) M (with a constant wind w:
    K_l + H_l = -B''_l + w_l B'_l, Sec. 3.2, eq. convec_prec_2)."""

    def __init__(self, spaces, wind=None):
        self.d = len(spaces)
        self.n = [s.n for s in spaces]
        self.shape = tuple(self.n[::-1])
        self.lam, self.U, self.V = [], [], []
        w = np.zeros(self.d) if wind is None else np.asarray(wind, dtype=np.float64)
        for l, s in enumerate(spaces):
            K = s.K if w[l] == 0.0 else s.K + w[l] * s.B[1]
            lam, U, V = eig_factors(K, s.M)
            self.lam.append(lam)
            self.U.append(U)
            self.V.append(V)
        # diagonal of sum_l I (x) D_l (x) I in tensor shape (i_d, .., i_1)
        D = np.zeros(self.shape)
        for l in range(self.d):
            sh = [1] * self.d
            sh[self.d - 1 - l] = self.n[l]
            D = D + self.lam[l].reshape(sh)
        self.D = D

    def apply(self, b):
        """s = P^{-1} b by eq. (FD2D) / (FD3D)."""
        y = kron_apply([V.T for V in self.V], np.asarray(b, dtype=np.float64), self.shape)
        y = y / self.D.reshape(-1)
        return kron_apply(self.U, y, self.shape)

    __call__ = apply
