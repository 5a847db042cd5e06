"""Univariate B-splines: knots, Cox--de Boor evaluation, Greville points.

Paper, Sec. 2.1: open knot vector Xi = {xi_1..xi_{m+p+1}} with p+1 repeated end
knots; B-spline basis B_i, i = 0..m-1, of degree p.  Sec. 2.2, eq. (greville):
tau_i = (1/p) * sum_{j=1..p} xi_{i+j+1}, i = 1..n, n = m - 2 (eq. space).

Indices in this module are 0-based on the knot array ``t`` (t[k] = xi_{k+1}) and
on the basis (B_0..B_{m-1}), exactly like the paper's basis indices.
"""

import numpy as np


def open_uniform_knots(n_elem, p):
    """Open knot vector on [0,1] with n_elem uniform elements, simple interior knots.

    Sec. 2.1: 0 = xi_1 = .. = xi_{p+1} < xi_{p+2} <= .. <= xi_m < xi_{m+1} = .. = 1.
    Maximum regularity C^{p-1}: every interior knot has multiplicity 1, so
    m = n_elem + p basis functions.
    """
    if n_elem < 1 or p < 1:
        raise ValueError("need n_elem >= 1 and p >= 1")
    interior = np.arange(1, n_elem, dtype=np.float64) / n_elem
    return np.concatenate([np.zeros(p + 1), interior, np.ones(p + 1)])


def num_basis(t, p):
    """m = (number of knots) - p - 1."""
    return len(t) - p - 1


def _degree0(t, x):
    """B_{k,0}(x) for every k = 0..len(t)-2 (half-open spans; the last non-empty
    span is closed at its right end so that x = t[-1] is covered)."""
    nk = len(t) - 1
    out = np.zeros(nk)
    last = max(k for k in range(nk) if t[k] < t[k + 1])
    for k in range(nk):
        if t[k] <= x < t[k + 1]:
            out[k] = 1.0
    if x == t[-1]:
        out[:] = 0.0
        out[last] = 1.0
    return out


def basis_all(t, p, x, deriv=0):
    """Value of d^deriv/dx^deriv of all m basis functions B_{i,p} at the point x.

    Cox--de Boor recursion written out on the whole table (slow, O(m p) per point):
        B_{k,q}(x)  = w1 * B_{k,q-1}(x) + w2 * B_{k+1,q-1}(x),
        w1 = (x - t_k) / (t_{k+q} - t_k),  w2 = (t_{k+q+1} - x) / (t_{k+q+1} - t_{k+1}),
    and for derivatives the standard identity
        B^{(r)}_{k,q} = q * ( B^{(r-1)}_{k,q-1} / (t_{k+q} - t_k)
                            - B^{(r-1)}_{k+1,q-1} / (t_{k+q+1} - t_{k+1}) ),
    with 0/0 := 0 for repeated knots.
    """
    m = num_basis(t, p)

    def table(q, r):
        # returns the r-th derivative of B_{k,q} for k = 0..len(t)-q-2
        if r > q:
            return np.zeros(len(t) - q - 1)
        if q == 0:
            return _degree0(t, x)
        low = table(q - 1, r - 1) if r > 0 else table(q - 1, 0)
        out = np.zeros(len(t) - q - 1)
        for k in range(len(t) - q - 1):
            d1 = t[k + q] - t[k]
            d2 = t[k + q + 1] - t[k + 1]
            if r == 0:
                a = (x - t[k]) / d1 * low[k] if d1 > 0 else 0.0
                b = (t[k + q + 1] - x) / d2 * low[k + 1] if d2 > 0 else 0.0
            else:
                a = q * low[k] / d1 if d1 > 0 else 0.0
                b = q * low[k + 1] / d2 if d2 > 0 else 0.0
                b = -b
            out[k] = a + b
        return out

    vals = table(p, deriv)
    assert len(vals) == m
    return vals


def greville_full(t, p):
    """Greville abscissae of all m basis functions: xi*_k = mean(t[k+1 .. k+p])."""
    m = num_basis(t, p)
    return np.array([np.mean(t[k + 1:k + p + 1]) for k in range(m)])


def greville_interior(t, p):
    """Collocation points of eq. (greville): tau_i = (1/p) sum_{j=1..p} xi_{i+j+1},
    i = 1..n (1-based knots), i.e. the Greville abscissae of B_1..B_n."""
    m = num_basis(t, p)
    n = m - 2
    tau = np.empty(n)
    for i in range(1, n + 1):
        # xi_{i+j+1} (1-based) == t[i+j] (0-based), j = 1..p
        tau[i - 1] = sum(t[i + j] for j in range(1, p + 1)) / p
    return tau
