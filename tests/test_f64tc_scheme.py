"""Host checks of the arithmetic the FP64_TC form's kernels rely on (kernels_fd_f64tc.cu),
written out with Python integers and fractions -- the error-free splitting of Ozaki, Ogita,
Oishi and Rump (2012) as the kernels use it: a power of two per row (per factor column),
eight signed base-2^7 digits per value, the 36 digit-slice pairs with s + t <= 7 summed per
weight w = s + t, and the recombination 2^{e + f - 63} sum_w G_w 2^{7 (7 - w)}.

Pinned here, without a GPU:
  * every G_w is an integer below 2^24 for K <= 130 (exact in FP32 accumulation), and up to
    K = 148 (the form's limit) only G_7 can exceed it; at K = 149 G_6 can;
  * the split is exact up to the digit tail: |x - 2^e sum_s d_s 2^{-7(s+1)}| < 2^{e - 56};
  * one product entry is within 13 K 2^{-56} of its scale 2^{e + f} of the exact dot product
    (worst-case digits included): the dropped pairs (s + t = 8: 7 of at most K 127^2 2^{-70},
    the rest 2^-7 smaller) give 7.05 K, the digit tails 2 K, and the final rounding of a result
    of up to K times the scale 4 K; the recombination of H 2^28 + L is exact before that one
    rounding;
  * a planted mistake (a dropped pair) breaks the bound.
"""

import struct
from fractions import Fraction

import numpy as np
import pytest


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _row_exp(v):
    mx = max(_bits(x) & 0x7FFFFFFFFFFFFFFF for x in v)
    emax = mx >> 52
    return emax - 1022 if emax else -1022


def _digits(x, e):
    """Eight signed base-2^7 digits of x / 2^e (truncated, sign carried by every digit)."""
    b = _bits(x)
    ex, m = (b >> 52) & 0x7FF, b & ((1 << 52) - 1)
    if ex:
        m |= 1 << 52
    else:
        ex = 1
    sh = ex - e - 1019
    F = m << sh if sh >= 0 else (0 if -sh >= 64 else m >> (-sh))
    assert F < 1 << 56
    ds = [(F >> (7 * (7 - s))) & 127 for s in range(8)]
    return [-d for d in ds] if b >> 63 else ds


def _groups(a, b, drop=None):
    ea, eb = _row_exp(a), _row_exp(b)
    da = [_digits(x, ea) for x in a]
    db = [_digits(x, eb) for x in b]
    G = [0] * 8
    for s in range(8):
        for t in range(8 - s):
            if drop == (s, t):
                continue
            G[s + t] += sum(da[k][s] * db[k][t] for k in range(len(a)))
    return G, ea, eb


def _recombine(G, E):
    H = L = 0
    for w in range(4):
        H = (H << 7) + G[w]
        L = (L << 7) + G[w + 4]
    T = H * 2 ** 28 + L
    assert T == sum(G[w] << (7 * (7 - w)) for w in range(8))
    return float(Fraction(T) * Fraction(2) ** E) if T else 0.0


def test_split_is_exact_up_to_the_digit_tail():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.standard_normal(40) * 10.0 ** rng.uniform(-8, 8, 40),
                        [0.0, -0.0, 5e-324, -2.5e-310, 1.0, -1.0, 2.0 ** 60]])
    e = _row_exp(v)
    for x in v:
        d = _digits(x, e)
        assert all(abs(q) <= 127 for q in d)
        approx = sum(Fraction(q) * Fraction(2) ** (-7 * (s + 1)) for s, q in enumerate(d))
        assert abs(Fraction(float(x)) - approx * Fraction(2) ** e) < Fraction(2) ** (e - 56)


@pytest.mark.parametrize("K", [1, 64, 130, 132, 148, 149])
def test_group_sums_fit_fp32_exactly(K):
    # worst case: the largest digits (values just below the row scale, same sign: digits
    # 0..6 are 127, the last 120)
    a = [np.nextafter(1.0, 0.0)] * K
    b = [np.nextafter(1.0, 0.0)] * K
    G, _, _ = _groups(a, b)
    for w, g in enumerate(G):
        assert g <= (w + 1) * K * 127 ** 2
        if K <= 130 or (K <= 148 and w < 7):
            assert abs(g) < 2 ** 24, (K, w, g)
    if K == 149:
        assert G[6] >= 2 ** 24  # why the form stops at n = 148


@pytest.mark.parametrize("K", [5, 65, 130])
def test_product_entry_within_the_bound_of_its_scale(K):
    rng = np.random.default_rng(K)
    worst = 0.0
    for trial in range(6):
        a = rng.standard_normal(K) * np.exp(rng.uniform(-4, 4))
        b = rng.standard_normal(K)
        if trial == 0:
            a[::3] = 0.0
        if trial == 1:
            a = np.full(K, np.nextafter(1.0, 0.0))
            b = np.full(K, -np.nextafter(1.0, 0.0))
        G, ea, eb = _groups(a, b)
        got = _recombine(G, ea + eb - 63)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        err = abs(Fraction(got) - exact) / Fraction(2) ** (ea + eb)
        assert err <= Fraction(13 * K, 2 ** 56), (trial, float(err))
        worst = max(worst, float(err))
    assert worst < 13 * K * 2.0 ** -56


def test_a_dropped_pair_breaks_the_bound():
    rng = np.random.default_rng(3)
    K = 64
    a, b = rng.standard_normal(K), rng.standard_normal(K)
    G, ea, eb = _groups(a, b, drop=(1, 2))  # w = 3: weight 2^-35 of the scale
    got = _recombine(G, ea + eb - 63)
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    err = abs(Fraction(got) - exact) / Fraction(2) ** (ea + eb)
    assert err > Fraction(13 * K, 2 ** 56)
