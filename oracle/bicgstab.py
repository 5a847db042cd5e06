"""Right-preconditioned BiCGStab (van der Vorst 1992, the solver of Sec. 5).

TEST INFRASTRUCTURE ONLY: the oracle the CUDA path is checked against.

Sec. 5 runs BiCGStab with the FD preconditioner and counts iterations in halves:
one iteration is a BiCG step followed by one GMRES(1) step, and a solve that
stops after the BiCG step of iteration k is reported as k - 0.5.  Readings (the
paper states neither): the preconditioner is applied on the right (x is updated
with M^{-1} p and M^{-1} s, as Matlab's ``bicgstab`` does), the shadow residual is
the initial residual, and the stop test ||r|| <= tol ||b|| is made after each half
step on the recursively updated residual (s after the BiCG half, r after the
GMRES half).
"""

import numpy as np


def bicgstab(A, b, M=None, x0=None, tol=1e-8, max_iter=200):
    """Solve A x = b.  ``A`` and ``M`` (preconditioner inverse) are callables or
    matrices.  Returns dict(x, steps, iters, hist, relres_true, flag):

    steps  number of half steps taken (2k after a full iteration k, 2k - 1 when the
           BiCG half of iteration k met the tolerance);
    iters  steps / 2, the paper's count (k or k - 0.5);
    hist   ||residual|| / ||b|| before the first step and after every half step;
    flag   0 converged, 2 max_iter reached, 3 breakdown (rho or omega zero),
           4 non-finite values.
    """
    Aop = A if callable(A) else (lambda v: A @ v)
    Mop = (lambda v: v) if M is None else (M if callable(M) else (lambda v: M @ v))
    b = np.asarray(b, dtype=np.float64)
    N = b.shape[0]
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - Aop(x)
    rhat = r.copy()
    hist = [np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0]
    steps, flag = 0, 2
    if not np.isfinite(hist[0]):
        flag = 4
    elif np.linalg.norm(r) <= tol * bnorm:
        flag = 0
    else:
        rho_prev = alpha = omega = 1.0
        p = np.zeros(N)
        v = np.zeros(N)
        for k in range(1, max_iter + 1):
            rho = np.dot(rhat, r)
            if rho == 0.0 or omega == 0.0:
                flag = 3
                break
            beta = (rho / rho_prev) * (alpha / omega)
            p = r + beta * (p - omega * v)           # first iteration: p = r
            phat = Mop(p)
            v = Aop(phat)
            alpha = rho / np.dot(rhat, v)
            s = r - alpha * v
            snorm = np.linalg.norm(s)
            steps = 2 * k - 1
            hist.append(snorm / bnorm)
            if not np.isfinite(snorm):
                flag = 4
                break
            if snorm <= tol * bnorm:                 # converged halfway: k - 0.5
                x = x + alpha * phat
                flag = 0
                break
            shat = Mop(s)
            t = Aop(shat)
            omega = np.dot(t, s) / np.dot(t, t)
            x = x + alpha * phat + omega * shat
            r = s - omega * t
            rnorm = np.linalg.norm(r)
            steps = 2 * k
            hist.append(rnorm / bnorm)
            if not np.isfinite(rnorm):
                flag = 4
                break
            if rnorm <= tol * bnorm:
                flag = 0
                break
            rho_prev = rho
    relres_true = np.linalg.norm(b - Aop(x)) / bnorm if bnorm > 0 else 0.0
    return dict(x=x, steps=steps, iters=steps / 2.0, hist=np.array(hist),
                relres_true=relres_true, flag=flag)
