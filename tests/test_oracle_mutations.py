"""Plant plausible mistakes in the oracle (CPU only) and check that a pin catches each.

Each mutation is applied with monkeypatch to a copy of the oracle's behaviour; the
corresponding pin from the other test files is re-run inline and must fail.
"""

import numpy as np
import pytest

from oracle import bspline, collocation as C, fd as F, geometry as Geo
import tests.test_oracle_collocation as TC


def test_dropped_first_order_term_is_caught(monkeypatch):
    orig = Geo.pullback_coefficients

    def no_L(fmap, xi):
        G, L = orig(fmap, xi)
        return G, 0.0 * L

    monkeypatch.setattr(C, "pullback_coefficients", no_L)
    with pytest.raises(AssertionError):
        TC.test_operator_on_exact_polynomial_2d(3)


def test_transposed_kronecker_order_is_caught(monkeypatch):
    def wrong_kron(mats):
        out = C.sp.csr_matrix(mats[0])
        for A in mats[1:]:
            out = C.sp.kron(out, C.sp.csr_matrix(A), format="csr")
        return out

    monkeypatch.setattr(C, "kron_list", wrong_kron)
    with pytest.raises(AssertionError):
        TC.test_operator_on_exact_polynomial_2d(3)


def test_wrong_sign_of_K_is_caught():
    s = C.Space1D(64, 3)
    lam, _, _ = F.eig_factors(s.B[2], s.M)  # K = +B'' instead of -B''
    assert not abs(lam[0] / np.pi**2 - 1.0) < 2e-3


def test_off_by_one_greville_is_caught():
    t = bspline.open_uniform_knots(4, 3)
    wrong = np.array([np.mean(t[i + 2:i + 5]) for i in range(1, 6)])  # shifted knot window
    ref = np.array([1 / 12, 0.25, 0.5, 0.75, 11 / 12])
    assert np.max(np.abs(wrong - ref)) > 1e-3


def test_transposed_V_in_fd_is_caught():
    spaces = [C.Space1D(6, 3), C.Space1D(6, 3)]
    P = C.assemble_preconditioner(spaces)
    fd = F.FD(spaces)
    fd.V = [V.T for V in fd.V]
    b = np.random.default_rng(1).standard_normal(P.shape[0])
    assert np.linalg.norm(fd(P @ b) - b) > 1e-6 * np.linalg.norm(b)


def _bicgstab_with(monkeypatch, old, new):
    """Re-build the oracle's BiCGStab with one source line changed."""
    import inspect
    from oracle import bicgstab as B
    src = inspect.getsource(B.bicgstab)
    assert old in src
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    monkeypatch.setattr(B, "bicgstab", ns["bicgstab"])


@pytest.mark.parametrize("old,new", [
    ("p = r + beta * (p - omega * v)", "p = r + beta * p"),           # dropped omega v
    ("omega = np.dot(t, s) / np.dot(t, t)", "omega = np.dot(t, s) / np.dot(s, s)"),
    ("r = s - omega * t", "r = s + omega * t"),                        # wrong sign
    ("x = x + alpha * phat + omega * shat", "x = x + alpha * phat + omega * s"),  # M skipped
])
def test_bicgstab_mistakes_are_caught(monkeypatch, old, new):
    import tests.test_oracle_bicgstab as TB
    _bicgstab_with(monkeypatch, old, new)
    with pytest.raises(AssertionError):
        TB.test_matches_scipy_at_fixed_step_counts(2, 8, 3)


def test_wrong_sign_or_transpose_of_wind_term_is_caught(monkeypatch):
    import tests.test_oracle_wind as TW
    orig = Geo.wind_coefficients
    monkeypatch.setattr(C, "wind_coefficients", lambda fmap, xi, w: -orig(fmap, xi, w))
    with pytest.raises(AssertionError):
        TW.test_convective_term_against_finite_differences()
    # J^{-T} w instead of J^{-1} w
    monkeypatch.setattr(C, "wind_coefficients",
                        lambda fmap, xi, w: np.linalg.solve(fmap.J(xi).T, np.asarray(w)))
    with pytest.raises(AssertionError):
        TW.test_convective_term_against_finite_differences()


def test_swapped_mixed_wq_weights_are_caught(monkeypatch):
    """Weighted quadrature (Sec. 2.3): using the (0, 1) rule where the (1, 0) rule belongs
    breaks exactness for constant coefficients with off-diagonal Q."""
    from oracle import wq as Q
    import tests.test_oracle_wq as TW
    orig = Q.WQSpace1D.weights

    def swapped(self, s, t):
        if (s, t) in ((0, 1), (1, 0)):
            return orig(self, t, s)
        return orig(self, s, t)

    monkeypatch.setattr(Q.WQSpace1D, "weights", swapped)
    with pytest.raises(AssertionError):
        TW.test_constant_coefficients_are_integrated_exactly(2, [[1.3, 0.4], [-0.2, 0.9]])


def test_wq_weights_outside_the_support_are_caught(monkeypatch):
    """A rule spread over every quadrature point (still exact) is not a weighted quadrature of
    the test function: the support pin fails."""
    from oracle import wq as Q
    import tests.test_oracle_wq as TW

    def global_rule(self, s, t):
        W = np.zeros((self.n, self.nq))
        for r, i in enumerate(range(1, self.m - 1)):
            E = self.Bq_full[t].T
            W[r], *_ = np.linalg.lstsq(E, self.G[(s, t)][i], rcond=None)
        return W

    monkeypatch.setattr(Q.WQSpace1D, "weights", global_rule)
    with pytest.raises(AssertionError):
        TW.test_univariate_rules_are_exact_on_the_spline_space(8, 3)
