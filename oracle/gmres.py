"""Unrestarted right-preconditioned GMRES (Saad & Schultz 1986, cited in Sec. 3).

Readings (the paper names GMRES as an option but runs BiCGStab; it states no
tolerance, norm, initial guess or preconditioning side):
* right preconditioning, A M^{-1} y = b, x = x0 + M^{-1} V_k y_k, so the monitored
  residual |g_{k+1}| is the true residual norm in exact arithmetic;
* relative criterion |g_{k+1}| <= tol * ||b||, tol = 1e-8;
* Arnoldi with modified Gram--Schmidt, Hessenberg least squares with Givens rotations;
* the flexible variant (``flexible=True``) keeps Z_k = [M^{-1} v_1 ..] and returns
  x = x0 + Z_k y_k, valid for a preconditioner that changes between calls.
"""

import numpy as np


def givens(a, b):
    """(c, s) with [c s; -s c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    if abs(b) > abs(a):
        t = a / b
        s = 1.0 / np.sqrt(1.0 + t * t)
        return s * t, s
    t = b / a
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, c * t


def gmres(A, b, M=None, x0=None, tol=1e-8, max_iter=200, flexible=False):
    """Solve A x = b.  ``A`` and ``M`` (preconditioner inverse) are callables or
    matrices; returns dict(x, iters, hist, relres_true, H, V).

    hist[j] = |g_{j+1}| / ||b|| for j = 0..iters (hist[0] = ||r0||/||b||).
    """
    Aop = A if callable(A) else (lambda v: A @ v)
    Mop = (lambda v: v) if M is None else (M if callable(M) else (lambda v: M @ v))
    b = np.asarray(b, dtype=np.float64)
    N = b.shape[0]
    x0 = np.zeros(N) if x0 is None else np.asarray(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r0 = b - Aop(x0)
    beta = np.linalg.norm(r0)
    hist = [beta / bnorm if bnorm > 0 else 0.0]
    if beta == 0.0 or max_iter == 0:
        return dict(x=x0.copy(), iters=0, hist=np.array(hist), relres_true=hist[0],
                    H=np.zeros((1, 0)), V=r0[:, None])
    V = np.zeros((N, max_iter + 1))
    Z = np.zeros((N, max_iter)) if flexible else None
    H = np.zeros((max_iter + 1, max_iter))
    cs = np.zeros(max_iter)
    sn = np.zeros(max_iter)
    g = np.zeros(max_iter + 1)
    g[0] = beta
    V[:, 0] = r0 / beta
    k = 0
    for j in range(max_iter):
        z = Mop(V[:, j])
        if flexible:
            Z[:, j] = z
        w = Aop(z)
        for i in range(j + 1):  # modified Gram--Schmidt
            H[i, j] = np.dot(w, V[:, i])
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0.0:
            V[:, j + 1] = w / H[j + 1, j]
        # rotate the new column by the previous rotations, then make a new one
        col = H[:j + 2, j].copy()
        for i in range(j):
            a, c_ = col[i], col[i + 1]
            col[i] = cs[i] * a + sn[i] * c_
            col[i + 1] = -sn[i] * a + cs[i] * c_
        cs[j], sn[j] = givens(col[j], col[j + 1])
        col[j] = cs[j] * col[j] + sn[j] * col[j + 1]
        col[j + 1] = 0.0
        H_rot_col = col
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        if j == 0:
            R = np.zeros((max_iter, max_iter))
        R[:j + 1, j] = H_rot_col[:j + 1]
        k = j + 1
        hist.append(abs(g[j + 1]) / bnorm)
        if abs(g[j + 1]) <= tol * bnorm or H[j + 1, j] == 0.0:
            break
    y = np.linalg.solve(np.triu(R[:k, :k]), g[:k])
    if flexible:
        x = x0 + Z[:, :k] @ y
    else:
        x = x0 + Mop(V[:, :k] @ y)
    relres = np.linalg.norm(b - Aop(x)) / bnorm
    return dict(x=x, iters=k, hist=np.array(hist), relres_true=relres,
                H=H[:k + 1, :k], V=V[:, :k + 1])
