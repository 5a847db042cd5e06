"""Host checks of the arithmetic the error-compensated TF32 form (TF32X3) relies on
(kernels_fd_tc.cu, tc_gemm_kernel<2>), written out with numpy: every operand x is held as
hi = tf32(x) and lo = tf32(x - hi), and a product accumulates A_hi B_lo + A_lo B_hi +
A_hi B_hi in FP32 (a TF32 x TF32 product has at most 22 significant bits and is exact in
FP32; the sums round in FP32).

Pinned here, without a GPU:
  * the split keeps |x - hi - lo| <= 2^-22 |x| (and hi alone only 2^-11 |x|);
  * a compensated dot product of length K is within ~2^-20 sum |a||b| of the exact one, three
    orders of magnitude closer than the plain TF32 product, which is what moves the FD from
    ~1e-3 to ~1e-6 of the oracle's (the GPU tests bound it by 1e-4);
  * dropping a correction term (a planted mistake) falls back to plain TF32's error.
"""

import numpy as np
import pytest


def tf32(x):
    """Round FP32 values to TF32 (10 explicit mantissa bits), to nearest with ties away from
    zero, as the device's cvt.rna.tf32.f32 does."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = np.where(finite, (u + 0x1000) & 0xFFFFE000, u)
    return r.astype(np.uint32).view(np.float32)


def split(x):
    xf = np.asarray(x, dtype=np.float32)
    hi = tf32(xf)
    lo = tf32(xf - hi)  # xf - hi is exact in FP32
    return hi, lo


def fp32_dot(a, b):
    """Sum of exact products (as FP64, then to FP32: a TF32 product fits FP32 exactly) in
    FP32, in order."""
    s = np.float32(0.0)
    for x, y in zip(a, b):
        p = np.float32(np.float64(x) * np.float64(y))
        s = np.float32(s + p)
    return s


def test_split_error_bound():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-10, 10, 20000)).astype(np.float32)
    hi, lo = split(x)
    r = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(r <= 2.0 ** -22 * np.abs(x.astype(np.float64)))
    assert np.max(np.abs(x - hi) / np.abs(x)) <= 2.0 ** -11
    assert np.max(np.abs(x - hi) / np.abs(x)) > 2.0 ** -13  # hi alone really is TF32


@pytest.mark.parametrize("K", [8, 65, 130])
def test_compensated_dot_product(K):
    rng = np.random.default_rng(K)
    worst_x3, worst_tf32 = 0.0, 0.0
    for _ in range(200):
        a = rng.standard_normal(K).astype(np.float32)
        b = rng.standard_normal(K).astype(np.float32)
        exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        scale = float(np.dot(np.abs(a).astype(np.float64), np.abs(b).astype(np.float64)))
        ah, al = split(a)
        bh, bl = split(b)
        acc = np.float32(0.0)  # the three terms into one accumulator, in order
        for i in range(K):
            for p in (np.float64(ah[i]) * bl[i], np.float64(al[i]) * bh[i],
                      np.float64(ah[i]) * bh[i]):
                acc = np.float32(acc + np.float32(p))
        x3 = float(acc)
        t = float(fp32_dot(ah, bh))
        worst_x3 = max(worst_x3, abs(x3 - exact) / scale)
        worst_tf32 = max(worst_tf32, abs(t - exact) / scale)
    assert worst_x3 <= 2.0 ** -20, worst_x3
    assert worst_tf32 >= 2.0 ** -13, worst_tf32
    assert worst_tf32 / worst_x3 > 100


def test_a_dropped_correction_term_loses_the_gain():
    rng = np.random.default_rng(4)
    K = 130
    worst = 0.0
    for _ in range(100):
        a = rng.standard_normal(K).astype(np.float32)
        b = rng.standard_normal(K).astype(np.float32)
        exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        scale = float(np.dot(np.abs(a).astype(np.float64), np.abs(b).astype(np.float64)))
        ah, al = split(a)
        bh, _ = split(b)
        acc = np.float32(0.0)
        for i in range(K):  # A_lo B_hi + A_hi B_hi only: B's correction dropped
            for p in (np.float64(al[i]) * bh[i], np.float64(ah[i]) * bh[i]):
                acc = np.float32(acc + np.float32(p))
        worst = max(worst, abs(float(acc) - exact) / scale)
    assert worst > 2.0 ** -14
