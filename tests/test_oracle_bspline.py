"""Pins for oracle.bspline (Sec. 2.1 basis, Sec. 2.2 eq. greville).

Pinned against: partition of unity and its derivatives, Marsden linear precision,
scipy.interpolate.BSpline (an independent library implementation), and hand-worked
fixtures in tests/golden/.
"""

import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import bspline
from oracle.collocation import Space1D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n_elem", [1, 3, 8])
def test_partition_of_unity_and_derivatives(p, n_elem):
    t = bspline.open_uniform_knots(n_elem, p)
    rng = np.random.default_rng(p * 100 + n_elem)
    for x in np.concatenate([rng.uniform(0, 1, 7), [0.0, 1.0]]):
        assert abs(bspline.basis_all(t, p, x, 0).sum() - 1.0) < 1e-13
        for r in (1, 2):
            if r <= p:
                assert abs(bspline.basis_all(t, p, x, r).sum()) < 1e-9 * n_elem ** r


@pytest.mark.parametrize("p", [2, 3, 5])
def test_marsden_linear_precision(p):
    t = bspline.open_uniform_knots(7, p)
    xs = bspline.greville_full(t, p)
    for x in np.linspace(0, 1, 23):
        assert abs(np.dot(xs, bspline.basis_all(t, p, x, 0)) - x) < 1e-13


@pytest.mark.parametrize("p", [2, 3, 4, 6])
@pytest.mark.parametrize("deriv", [0, 1, 2])
def test_matches_scipy_bspline(p, deriv):
    n_elem = 9
    t = bspline.open_uniform_knots(n_elem, p)
    m = bspline.num_basis(t, p)
    rng = np.random.default_rng(7 + p)
    xs = rng.uniform(0, 1, 11)
    for j in range(m):
        c = np.zeros(m)
        c[j] = 1.0
        ref = BSpline(t, c, p, extrapolate=False).derivative(deriv) if deriv else \
            BSpline(t, c, p, extrapolate=False)
        for x in xs:
            mine = bspline.basis_all(t, p, x, deriv)[j]
            assert abs(mine - ref(x)) < 1e-11 * max(1.0, n_elem ** deriv)


@pytest.mark.parametrize("fname,n_elem,p", [("greville_ne4_p3.txt", 4, 3),
                                             ("greville_ne3_p2.txt", 3, 2)])
def test_greville_hand_fixture(fname, n_elem, p):
    ref = np.array([float(v) for v in _read_golden(fname)])
    t = bspline.open_uniform_knots(n_elem, p)
    tau = bspline.greville_interior(t, p)
    assert tau.shape == ref.shape
    assert np.max(np.abs(tau - ref)) < 1e-15


def test_collocation_1d_hand_fixture():
    rows = _read_golden("collocation_1d_ne2_p2.txt")
    ref = {"M": [], "D1": [], "K": []}
    for r in rows:
        key, *vals = r.split()
        ref[key].append([float(v) for v in vals])
    s = Space1D(2, 2)
    assert np.allclose(s.tau, [0.25, 0.75], atol=0, rtol=0)
    assert np.max(np.abs(s.M - np.array(ref["M"]))) < 1e-15
    assert np.max(np.abs(s.B[1] - np.array(ref["D1"]))) < 1e-14
    assert np.max(np.abs(s.K - np.array(ref["K"]))) < 1e-13


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_greville_interior_are_full_greville_minus_ends(p):
    t = bspline.open_uniform_knots(10, p)
    full = bspline.greville_full(t, p)
    tau = bspline.greville_interior(t, p)
    assert np.array_equal(tau, full[1:-1])
    assert np.all(np.diff(tau) > 0) and tau[0] > 0 and tau[-1] < 1


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_factor_bandwidth(p):
    s = Space1D(12, p)
    for B in s.B:
        nnz = (np.abs(B) > 0).sum(axis=1)
        assert nnz.max() <= p + 1
