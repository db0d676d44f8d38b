"""A numpy emulation of the tensor-core scoring mode's arithmetic.

Test infrastructure (plain numpy, no GPU): it checks the error bound that the
GPU parity tests use for the tensor-core mode against an arithmetic model of
that mode, written from its description rather than from the CUDA code:

* GEMM1: the augmented rows [Im(rho_m V_i), Re(rho_m V_i)] (FP32) of a
  coordinate are scaled by one power of two (its largest V component into
  [1, 2)), every direction [Re c, Im c] by its own, and both rounded to
  F16; a projection is the F16 sum of the 2r products, accumulated one
  product at a time in F16 (the worst order the bound allows);
* decisions from the sign bits of the F16 projections (for K = 3 the middle
  line from the F16 sum p_0 + p_2, p_1 = -(p_0 + p_2));
* GEMM2: the real form of beta_g conj(V_i) (FP32), scaled by 2^e_i, split
  into hi = E4M3(x) and lo = E4M3(x - hi); the indicator is 2^(g - e_i) (an
  E4M3 power of two); products summed in FP32 per output column; hi and lo
  columns added and divided by 2^g in FP64;
* odd K: V^H z = T + sum_k (w^k - 1) P_k with T in FP64; even K:
  z = sum_m beta_m sign(p_m).
"""
from __future__ import annotations

import numpy as np


def e4m3(x):
    """Round to the nearest FP8 E4M3 value (ties to even, saturating at 448)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    q = np.where(a >= 2.0 ** -6, 2.0 ** (e - 3), 2.0 ** -9)  # quantum: 3 significand bits / subnormal step
    r = np.rint(a / q) * q
    r = np.minimum(r, 448.0)
    return np.copysign(r, x)


def _pow2_scale(m):
    """2^-ilogb(m): brings the largest magnitude m into [1, 2); 1 for m = 0."""
    m = np.asarray(m, dtype=np.float64)
    with np.errstate(divide="ignore"):
        lg = np.floor(np.log2(np.where(m > 0, m, 1.0)))
    return 2.0 ** (-lg)


def _ilogb(m):
    return np.floor(np.log2(m)).astype(np.int64)


def _f16_dot(a, c):
    """F16 operands a (rows x k), c (cols x k): F16 accumulation, product by product."""
    acc = np.zeros((a.shape[0], c.shape[0]), dtype=np.float16)
    for k in range(a.shape[1]):
        prod = (a[:, k:k + 1].astype(np.float32) * c[None, :, k].astype(np.float32))
        acc = (acc.astype(np.float32) + prod).astype(np.float16)
    return acc


def score(V, K: int, C, per_line_scale=False):
    """Emulated tensor-core scores f for directions C (S x r) on V (n x r).

    per_line_scale=True scales each augmented row by its own power of two
    instead of one per coordinate: then the K = 3 middle line, read from the
    F16 sum p_0 + p_2 of two differently scaled projections, is wrong."""
    V = np.asarray(V, dtype=np.complex64)
    C = np.asarray(C, dtype=np.complex64)
    n, r = V.shape
    S = C.shape[0]
    BK = K if K % 2 else K // 2
    lines = [0, 2] if K == 3 else list(range(BK))
    th = np.pi * (2 * np.arange(BK) + 1) / K
    bc_all, bs_all = np.cos(th).astype(np.float32), np.sin(th).astype(np.float32)
    # directions, F16 after a power-of-two scale each
    ct = np.concatenate([C.real, C.imag], axis=1).astype(np.float32)
    c16 = (ct * _pow2_scale(np.abs(ct).max(axis=1))[:, None].astype(np.float32)).astype(np.float16)
    # one power-of-two scale per coordinate, from its largest V component, for
    # all of its lines (so that projections of one coordinate can be added)
    vr, vi = V.real.astype(np.float32), V.imag.astype(np.float32)
    vscale = _pow2_scale(np.maximum(np.abs(vr), np.abs(vi)).max(axis=1)).astype(np.float32)[:, None]
    proj = {}
    for m in lines:
        bc, bs = bc_all[m], bs_all[m]  # rho_m = bc - i bs
        rows = np.concatenate([bc * vi - bs * vr, bc * vr + bs * vi], axis=1).astype(np.float32)  # Im, Re
        sc = _pow2_scale(np.abs(rows).max(axis=1)).astype(np.float32)[:, None] if per_line_scale else vscale
        a16 = (rows * sc).astype(np.float16)
        proj[m] = _f16_dot(a16, c16)  # n x S, F16
    neg = {m: np.signbit(proj[m]) for m in lines}
    if K == 3:
        neg[1] = ~np.signbit((proj[0].astype(np.float32) + proj[2].astype(np.float32)).astype(np.float16))
    # GEMM2 scales
    comp = np.maximum(np.abs(V.real), np.abs(V.imag)).astype(np.float32)
    m_i = comp.max(axis=1)
    amax = comp.max()
    g = 5 - (int(_ilogb(amax)) if amax > 0 else 5)
    e_i = np.where(m_i > 0, 5 - _ilogb(np.where(m_i > 0, m_i, 1.0)), g)
    e_i = np.clip(e_i, g, g + 9)
    ind_mag = 2.0 ** (g - e_i)  # exact E4M3 powers of two, 2^-9 .. 1
    w = np.exp(2j * np.pi * np.arange(K) / K)
    if K % 2:
        betas = [w[k] - 1 for k in range(1, K)]
        indic = [(~neg[k - 1]) & neg[k] for k in range(1, K)]  # n x S booleans
        signs = [ind.astype(np.float64) for ind in indic]
    else:
        betas = [(w[(m + 1) % K] - w[m]) / 2 for m in range(BK)]
        signs = [np.where(neg[m], -1.0, 1.0) for m in range(BK)]
    acc = np.zeros((S, r), dtype=np.complex128)
    for beta, sg in zip(betas, signs):
        br, bi = np.float32(beta.real), np.float32(beta.imag)
        re = (br * V.real + bi * V.imag).astype(np.float32)
        im = (bi * V.real - br * V.imag).astype(np.float32)
        out = []
        for x in (re, im):
            xs = (x.astype(np.float64) * (2.0 ** e_i)[:, None]).astype(np.float32)
            hi = e4m3(xs)
            lo = e4m3(xs.astype(np.float64) - hi)
            wgt = (sg * ind_mag[:, None]).astype(np.float32)  # n x S
            # FP32 sums over the coordinates, hi and lo columns apart
            s_hi = np.zeros((S, r), dtype=np.float32)
            s_lo = np.zeros((S, r), dtype=np.float32)
            for i in range(n):
                s_hi = (s_hi + wgt[i][:, None] * hi[i][None, :].astype(np.float32)).astype(np.float32)
                s_lo = (s_lo + wgt[i][:, None] * lo[i][None, :].astype(np.float32)).astype(np.float32)
            out.append((s_hi.astype(np.float64) + s_lo.astype(np.float64)) * 2.0 ** (-g))
        acc += out[0] + 1j * out[1]
    if K % 2:
        acc += np.conj(V.astype(np.complex128)).sum(axis=0)[None, :]
    return (np.abs(acc) ** 2).sum(axis=1)
