"""The FP64-accurate re-scoring's accumulation scheme, emulated in numpy
(test infrastructure, no GPU): each lane adds a*bh + a*bl + c*dh + c*dl per
row in double-float form -- FP32 products with their exact FMA residuals,
two-sum into (hi, lo) -- and every 256 rows the lanes' pairs are added in
FP64.  Against the exactly rounded sum of the same terms the result stays
within a few FP64 ulps of the terms' magnitude, for chunks far longer than
one flush (a chunk may hold 65536 rows, 2048 per lane)."""
import math

import numpy as np
import pytest

f32 = np.float32


def _fma32(a, b, c):
    # a * b + c rounded once to FP32: the product of two FP32 numbers is exact
    # in FP64, and so is its sum with an FP32 number of similar size
    return f32(float(a) * float(b) + float(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def _acc_dot2(hi, lo, a, bh, bl, c, dh, dl):
    p1 = f32(a * bh)
    e1 = _fma32(a, bh, -p1)
    p2 = f32(c * dh)
    e2 = _fma32(c, dh, -p2)
    s, e3 = _two_sum(p1, p2)
    small = _fma32(a, bl, _fma32(c, dl, f32(f32(e1 + e2) + e3)))
    h2, e4 = _two_sum(hi, s)
    return h2, f32(lo + f32(e4 + small))


def _lane_sum(vr, vi, zh, zl, wh, wl, flush=256):
    """One lane's component sum with FP64 flushes every `flush` rows."""
    tot = 0.0
    hi = lo = f32(0.0)
    for k in range(len(vr)):
        hi, lo = _acc_dot2(hi, lo, vr[k], zh[k], zl[k], vi[k], wh[k], wl[k])
        if (k + 1) % flush == 0:
            tot += float(hi) + float(lo)
            hi = lo = f32(0.0)
    return tot + (float(hi) + float(lo))


@pytest.mark.parametrize("rows,seed", [(256, 1), (2048, 2), (2048, 3)])
def test_double_float_accumulation_is_fp64_accurate(rows, seed):
    rng = np.random.default_rng(seed)
    vr = rng.standard_normal(rows).astype(f32)
    vi = rng.standard_normal(rows).astype(f32)
    k = rng.integers(0, 7, rows)
    z = np.exp(2j * np.pi * k / 7)  # the chosen roots of unity, FP64
    zh = z.real.astype(f32)
    zl = (z.real - zh.astype(np.float64)).astype(f32)
    wh = z.imag.astype(f32)
    wl = (z.imag - wh.astype(np.float64)).astype(f32)
    got = _lane_sum(vr, vi, zh, zl, wh, wl)
    terms = []
    for t in range(rows):  # the same terms, exactly: FP32 x FP32 is exact in FP64
        terms += [float(vr[t]) * float(zh[t]), float(vr[t]) * float(zl[t]),
                  float(vi[t]) * float(wh[t]), float(vi[t]) * float(wl[t])]
    exact = math.fsum(terms)
    scale = math.fsum(abs(x) for x in terms)
    assert abs(got - exact) <= 64 * 2.0 ** -53 * scale


def test_flushes_are_needed_for_long_chunks():
    # the same 2048 rows without the FP64 flushes: the FP32 low part's own
    # rounding errors pile up past the bound above
    rng = np.random.default_rng(3)
    rows = 2048
    vr = rng.standard_normal(rows).astype(f32)
    vi = rng.standard_normal(rows).astype(f32)
    k = rng.integers(0, 7, rows)
    z = np.exp(2j * np.pi * k / 7)
    zh = z.real.astype(f32)
    zl = (z.real - zh.astype(np.float64)).astype(f32)
    wh = z.imag.astype(f32)
    wl = (z.imag - wh.astype(np.float64)).astype(f32)
    terms = []
    for t in range(rows):
        terms += [float(vr[t]) * float(zh[t]), float(vr[t]) * float(zl[t]),
                  float(vi[t]) * float(wh[t]), float(vi[t]) * float(wl[t])]
    exact = math.fsum(terms)
    scale = math.fsum(abs(x) for x in terms)
    flushed = _lane_sum(vr, vi, zh, zl, wh, wl, flush=256)
    unflushed = _lane_sum(vr, vi, zh, zl, wh, wl, flush=rows + 1)
    assert abs(flushed - exact) <= 64 * 2.0 ** -53 * scale < abs(unflushed - exact)
