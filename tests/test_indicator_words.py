"""The tensor-core mode's rounding, bit by bit, against the nearest-root rule.

Test infrastructure (plain numpy, no GPU).  The scoring kernel turns F16
boundary projections into FP8 indicator words with two instructions whose
behaviour the PTX ISA documents: `prmt.b32` (byte permute; a selector nibble
with bit 3 set fills the result byte with the sign of the selected byte) and a
three-input logic op.  Here both are emulated from that documentation, the
words are built the way the kernel builds them, and the class they encode is
compared with the nearest K-th root of unity in angle (Sec. 3, Eq. 9) computed
directly in FP64 from the same projections.  For even K the kernel uses signs
instead of indicators, z = sum_m beta_m sign(p_m) with
beta_m = (w^{m+1} - w^m) / 2; that identity is checked against w^k too.
"""
import numpy as np
import pytest


def prmt(a, b, sel):
    """prmt.b32 d, a, b, sel (default mode): bytes 0-3 of a, 4-7 of b; for
    each result byte a selector nibble picks a source byte (low 3 bits) and,
    with bit 3 set, replicates that byte's sign bit into all 8 bits."""
    a = np.asarray(a, dtype=np.uint32)
    b = np.asarray(b, dtype=np.uint32)
    src = [(a >> (8 * i)) & 0xFF for i in range(4)] + [(b >> (8 * i)) & 0xFF for i in range(4)]
    out = np.zeros_like(a)
    for i in range(4):
        nib = (sel >> (4 * i)) & 0xF
        byte = src[nib & 7]
        if nib & 8:
            byte = np.where(byte & 0x80, 0xFF, 0x00).astype(np.uint32)
        out |= byte.astype(np.uint32) << (8 * i)
    return out


def pack_f16(lo, hi):
    """Two F16 values in one 32-bit register (lo in bits 0-15), as a packed
    tensor-memory load delivers two adjacent columns."""
    lo = np.asarray(lo, dtype=np.float16).view(np.uint16).astype(np.uint32)
    hi = np.asarray(hi, dtype=np.float16).view(np.uint16).astype(np.uint32)
    return lo | (hi << 16)


def hadd2(x, y):
    """add.f16x2: two F16 additions, each rounded to F16."""
    xl = (x & 0xFFFF).astype(np.uint16).view(np.float16).astype(np.float32)
    xh = (x >> 16).astype(np.uint16).view(np.float16).astype(np.float32)
    yl = (y & 0xFFFF).astype(np.uint16).view(np.float16).astype(np.float32)
    yh = (y >> 16).astype(np.uint16).view(np.float16).astype(np.float32)
    return pack_f16((xl + yl).astype(np.float16), (xh + yh).astype(np.float16))


SEL = 0xFDB9  # sign-replicated high bytes of the four F16 halves of (a, b)


def nearest_root(w, K):
    """Eq. 9: the index k of the K-th root of unity nearest to w in angle."""
    return np.mod(np.rint(np.angle(w) / (2 * np.pi / K)).astype(np.int64), K)


def projections(w, K):
    """p_m = Im(exp(-i theta_m) w), theta_m = pi (2m + 1) / K, in F16 (the
    tensor-core mode's GEMM1 output type)."""
    m = np.arange(K)
    th = np.pi * (2 * m + 1) / K
    return (np.exp(-1j * th)[None, :] * w[:, None]).imag.astype(np.float16)


def away_from_boundaries(w, K, margin):
    """Points whose angle is farther than `margin` (radians) from every
    decision boundary pi (2m + 1) / K, and whose F16 projections are not 0."""
    ang = np.mod(np.angle(w), 2 * np.pi)
    th = np.mod(np.pi * (2 * np.arange(K) + 1) / K, 2 * np.pi)
    d = np.abs(ang[:, None] - th[None, :])
    d = np.minimum(d, 2 * np.pi - d)
    return d.min(axis=1) > margin


def _points(seed, n):
    rng = np.random.default_rng(seed)
    mag = np.exp(rng.uniform(-8, 8, n))  # magnitudes over many binades
    return mag * np.exp(1j * rng.uniform(-np.pi, np.pi, n))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_k3_indicator_words_encode_the_nearest_root(seed):
    # the kernel projects lines 0 and 2 only; p_1 = -(p_0 + p_2) because the
    # three boundary directions sum to zero, so p_1 < 0 exactly where
    # p_0 + p_2 > 0; the class-1 word is ~n_0 & n_1 & mag, the class-2 word
    # ~n_1 & n_2 & mag, with n_m the sign mask of p_m and n_1 = ~sign(p_0 + p_2)
    K = 3
    w = _points(seed, 4 * 4000)
    w = w[away_from_boundaries(w, K, 2e-2)]
    w = w[: (len(w) // 4) * 4]
    p = projections(w, K)
    mag = np.uint32(0x38383838)  # E4M3 1.0 in every byte
    p0 = p[:, 0].reshape(-1, 4)
    p2 = p[:, 2].reshape(-1, 4)
    a0, b0 = pack_f16(p0[:, 0], p0[:, 1]), pack_f16(p0[:, 2], p0[:, 3])
    a2, b2 = pack_f16(p2[:, 0], p2[:, 1]), pack_f16(p2[:, 2], p2[:, 3])
    sum_neg = prmt(hadd2(a0, a2), hadd2(b0, b2), SEL)
    n0 = prmt(a0, b0, SEL)
    n1 = ~sum_neg & np.uint32(0xFFFFFFFF)
    n2 = prmt(a2, b2, SEL)
    w1 = ~n0 & n1 & mag
    w2 = ~n1 & n2 & mag
    k = nearest_root(w, K).reshape(-1, 4)
    for j in range(4):
        c1 = ((w1 >> (8 * j)) & 0xFF) == 0x38
        c2 = ((w2 >> (8 * j)) & 0xFF) == 0x38
        assert not np.any(c1 & c2)
        got = np.where(c1, 1, np.where(c2, 2, 0))
        np.testing.assert_array_equal(got, k[:, j])
        # a byte is either the magnitude or zero
        assert np.all(np.isin((w1 >> (8 * j)) & 0xFF, [0, 0x38]))


@pytest.mark.parametrize("K", [5, 7])
def test_odd_k_indicator_words_encode_the_nearest_root(K):
    # every boundary line projected: class k (1 <= k < K) where p_{k-1} > 0 and p_k < 0
    w = _points(10 + K, 4 * 3000)
    w = w[away_from_boundaries(w, K, 2e-2)]
    w = w[: (len(w) // 4) * 4]
    p = projections(w, K).reshape(-1, 4, K)
    nm = [prmt(pack_f16(p[:, 0, m], p[:, 1, m]), pack_f16(p[:, 2, m], p[:, 3, m]), SEL) for m in range(K)]
    mag = np.uint32(0x38383838)
    words = [~nm[k - 1] & nm[k] & mag for k in range(1, K)]
    kk = nearest_root(w, K).reshape(-1, 4)
    for j in range(4):
        hits = np.stack([((wd >> (8 * j)) & 0xFF) == 0x38 for wd in words], axis=1)
        assert np.all(hits.sum(axis=1) <= 1)
        got = np.where(hits.any(axis=1), hits.argmax(axis=1) + 1, 0)
        np.testing.assert_array_equal(got, kk[:, j])


@pytest.mark.parametrize("K", [2, 4, 6, 8])
def test_even_k_signs_sum_to_the_nearest_root(K):
    # even K: the B_K = K/2 lines through the origin; the kernel stores
    # (n_m & 0x80808080) | mag, i.e. -mag where p_m < 0 and +mag elsewhere,
    # and z = sum_m beta_m sign(p_m), beta_m = (w^{m+1} - w^m) / 2
    w = _points(20 + K, 4000)
    w = w[away_from_boundaries(w, K, 2e-2)]
    p = projections(w, K)[:, : K // 2]
    om = np.exp(2j * np.pi / K)
    beta = (om ** (np.arange(K // 2) + 1) - om ** np.arange(K // 2)) / 2
    a = pack_f16(p[:, 0], p[:, 0])
    byte = (prmt(a, a, SEL) & 0x80) | 0x38  # sign byte of coordinate 0, as stored
    assert np.all(np.isin(byte & 0xFF, [0x38, 0xB8]))
    s = np.where(p < 0, -1.0, 1.0)
    z = (s * beta[None, :]).sum(axis=1)
    np.testing.assert_allclose(z, om ** nearest_root(w, K), atol=1e-12)


def test_prmt_emulation_known_values():
    # bytes 1 and 3 of a, then of b, sign-replicated; plain byte moves with
    # bit 3 clear (selector 0x3210 is the identity on a)
    a = np.array([0x80FF7F01], dtype=np.uint32)
    b = np.array([0x0080FF00], dtype=np.uint32)
    assert prmt(a, b, 0x3210)[0] == 0x80FF7F01
    assert prmt(a, b, 0x7654)[0] == 0x0080FF00
    # a: byte1 = 0x7F (positive), byte3 = 0x80 (negative); b: byte1 = 0xFF, byte3 = 0x00
    assert prmt(a, b, SEL)[0] == 0x00FFFF00
