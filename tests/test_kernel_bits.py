"""The integer-pipe format changes of the stage kernels, checked bit for bit.

The kernels (csrc/weno_device.cuh) move values between FP64 and FP32 with
integer operations on the bit patterns instead of conversion instructions
(which issue to the FP64 pipe on this GPU).  This test restates each of those
bit manipulations in Python integers, step for step, and checks it against
numpy's IEEE conversions and against the error bounds the kernels rely on.
Like test_kernel_algebra.py it shows the arithmetic is right; the GPU parity
tests show the CUDA code computes it.
"""
import math
import struct

import numpy as np


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def bdbl(b):
    return struct.unpack("<d", struct.pack("<Q", b & (2 ** 64 - 1)))[0]


def fbits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def bflt(b):
    return struct.unpack("<f", struct.pack("<I", b & 0xFFFFFFFF))[0]


def hi(x):
    v = dbits(x) >> 32
    return v - 2 ** 32 if v >= 2 ** 31 else v


def lo(x):
    return dbits(x) & 0xFFFFFFFF


def funnel_r(l, h, sh):  # __funnelshift_r: (hi:lo) >> sh, low 32 bits
    return ((((h & 0xFFFFFFFF) << 32) | (l & 0xFFFFFFFF)) >> sh) & 0xFFFFFFFF


def f32_scaled(x, es):
    h = hi(x)
    fe = ((h >> 20) & 0x7FF) - es + 123
    m = funnel_r(lo(x), h, 29) & 0x7FFFFF
    b = (h & 0x80000000) | ((fe << 23) & 0xFFFFFFFF) | m
    return bflt(b) if (fe > 0 and (h & 0x7FF00000) != 0) else 0.0


def f32_scaled_rn(x, es):
    l = lo(x)
    lr = (l + 0x10000000) & 0xFFFFFFFF
    h = hi(x) + (1 if lr < l else 0)
    fe = ((h >> 20) & 0x7FF) - es + 123
    m = funnel_r(lr, h, 29) & 0x7FFFFF
    b = (h & 0x80000000) | ((fe << 23) & 0xFFFFFFFF) | m
    return bflt(b) if (fe > 0 and (hi(x) & 0x7FF00000) != 0) else 0.0


def f32_rn(x):
    l = lo(x)
    lr = (l + 0x10000000) & 0xFFFFFFFF
    h = hi(x) + (1 if lr < l else 0)
    fe = ((h >> 20) & 0x7FF) - 896
    sg = h & 0x80000000
    m = funnel_r(lr, h, 29) & 0x7FFFFF
    b = sg if fe <= 0 else ((sg | 0x7F800000) if fe >= 255 else (sg | (fe << 23) | m))
    return bflt(b)


def f64_of_f32(y, k):
    b = fbits(y)
    sg, fe = b & 0x80000000, (b >> 23) & 0xFF
    F = fe + 896 + k
    if fe == 0 or F <= 0:
        h, l = sg, 0
    elif fe == 255 or F >= 2047:
        h, l = sg | 0x7FF00000, 0
    else:
        h, l = sg | (((F << 20) + ((b >> 3) & 0xFFFFF)) & 0xFFFFFFFF), (b << 29) & 0xFFFFFFFF
    return bdbl((h << 32) | l)


def f64_of_f32_pos(y, k):
    b = fbits(y)
    return bdbl(((((b >> 3) + ((896 + k) << 20)) & 0xFFFFFFFF) << 32) | ((b << 29) & 0xFFFFFFFF))


RNG = np.random.default_rng(20261204)


def _doubles(n, lo_exp, hi_exp):
    return [float(RNG.standard_normal() * 2.0 ** int(RNG.integers(lo_exp, hi_exp))) for _ in range(n)]


def test_scaled_truncation_and_rounding():
    # x 2^(1019 - es) in FP32: truncated within 2^-23 (never above |x|), or
    # rounded to nearest; 0 below FP32's normal range
    for x in _doubles(20000, -300, 300):
        es = ((hi(x) & 0x7FFFFFFF) >> 20) + int(RNG.integers(0, 40))
        ref = x * 2.0 ** (1019 - es)
        t, r = f32_scaled(x, es), f32_scaled_rn(x, es)
        if abs(ref) >= 2.0 ** -126:
            assert abs(t - ref) <= abs(ref) * 2.0 ** -23 and abs(t) <= abs(ref)
            assert abs(r - ref) <= abs(ref) * 2.0 ** -24 * (1 + 1e-12)
        else:
            assert t == 0.0


def test_round_to_fp32():
    for z in _doubles(20000, -140, 140):
        r = f32_rn(z)
        if 2.0 ** -126 <= abs(z) < 3.0e38:
            assert r == float(np.float32(z)) or abs(r - z) <= abs(z) * 2.0 ** -24 * (1 + 1e-12)
        elif abs(z) < 2.0 ** -126:
            assert r == 0.0 or abs(r) == 2.0 ** -126  # flushed, or rounded up to the smallest normal


def test_fp32_to_fp64_with_exponent():
    for _ in range(20000):
        y = float(np.float32(RNG.standard_normal() * 2.0 ** int(RNG.integers(-120, 120))))
        k = int(RNG.integers(-900, 900))
        exact = y * 2.0 ** k
        if abs(y) < 2.0 ** -126 or not (2.0 ** -1022 <= abs(exact) < 1.7e308):
            continue
        assert f64_of_f32(np.float32(y), k) == exact
        if y > 0:
            assert f64_of_f32_pos(np.float32(y), k) == exact
    assert f64_of_f32(np.float32(0.0), 5) == 0.0
    assert f64_of_f32(np.float32(1e-40), 5) == 0.0  # subnormal FP32: flushed
    assert f64_of_f32(np.float32(1.0), 2000) == math.inf


def test_reciprocal_and_rsqrt_seeds():
    # rcp_pos: seed 1/m' (m' = m truncated to FP32) made FP64 times 2^(1023 - ex);
    # one cubic step then gives 1/x to about an ulp.  rsqrt_pos: m' in [1, 4)
    # by the exponent's parity, seed times 2^((1023 + odd - ex) / 2), one
    # third-order step.  (np.float32 1/x and 1/sqrt stand in for the
    # special-function unit's approximations, which are within 2^-22.)
    worst_rcp = worst_rsq = 0.0
    for _ in range(20000):
        x = abs(float(RNG.standard_normal())) * 2.0 ** int(RNG.integers(-1000, 1000)) + 1e-300
        h = hi(x)
        ex = (h >> 20) & 0x7FF
        mf = bflt(0x3F800000 | (funnel_r(lo(x), h, 29) & 0x7FFFFF))
        r = f64_of_f32_pos(np.float32(1.0) / np.float32(mf), 1023 - ex)
        e = 1 - x * r
        worst_rcp = max(worst_rcp, abs(e))
        odd = (ex & 1) ^ 1
        mq = bflt(((127 + odd) << 23) | (funnel_r(lo(x), h, 29) & 0x7FFFFF))
        q = f64_of_f32_pos(np.float32(1.0 / math.sqrt(float(mq))), (1023 + odd - ex) // 2)
        worst_rsq = max(worst_rsq, abs(q * math.sqrt(x) - 1))
    assert worst_rcp < 2.0 ** -22      # so the cubic step leaves < 2^-66
    assert worst_rsq < 2.0 ** -22      # so the third-order step leaves < 2^-64


def test_sensitivity_term_from_fp32_product():
    # sens_term's fast path: with the differences scaled by 2^(1019 - es) and
    # the deviation sum devf = mdf 2^edf in FP32, 4 eps mu^2 = me^2 dev^2
    # (me^2 = eps / 9) is y 2^(eme + 2 edf + 2 (es - 1019)), y = mef mdf^2;
    # within ~1e-6 of (me dev + mo)^2 whenever dev / 6 >= 2^30 scale mu0.
    f32 = np.float32
    worst = 0.0
    for _ in range(5000):
        eps, mu0, k = 10.0 ** RNG.uniform(-60, -20), 10.0 ** RNG.uniform(-60, -20), 4.0
        d = [float(v) * 2.0 ** int(RNG.integers(-200, 200)) for v in RNG.standard_normal(5)]
        es = max(hi(x) & 0x7FFFFFFF for x in d) >> 20
        f = [f32(f32_scaled(x, es)) for x in d]
        a = [-(f[0] + f[1]), -f[1], f32(0), f[2], f[2] + f[3], f[2] + f[3] + f[4]]
        fm = f32(((a[0] + a[1]) + (a[3] + a[4]) + a[5]) * f32(1 / 6))
        devf = f32(sum(abs(v - fm) for v in a))
        me2 = eps / 9.0
        eme = ((hi(me2) >> 20) & 0x7FF) - 1023
        mef = bflt(0x3F800000 | (funnel_r(lo(me2), hi(me2), 29) & 0x7FFFFF))
        db = fbits(devf)
        edf = (db >> 23) - 127
        mdf = bflt((db & 0x7FFFFF) | 0x3F800000)
        y = f32(mef) * (f32(mdf) * f32(mdf))
        kk = eme + 2 * (edf + es - 1019)
        lthr = 1019 + (((hi(6 * k * mu0) >> 20) & 0x7FF) - 1023) + 31
        if not (edf + es >= lthr and 0 < (fbits(y) >> 23) + 896 + kk < 2047):
            continue  # the kernel takes the FP64 branch
        e = f64_of_f32_pos(y, kk)
        av = [-(d[0] + d[1]), -d[1], 0.0, d[2], d[2] + d[3], d[2] + d[3] + d[4]]
        m = sum(av) / 6
        dev = sum(abs(v - m) for v in av)
        exact = (math.sqrt(4 * eps) / 6 * dev + math.sqrt(4 * eps) * k * mu0) ** 2
        worst = max(worst, abs(e - exact) / exact)
    assert 0 < worst < 2e-6
