"""Seeded synthetic inputs for the low-rank candidate-scoring path.

This module only draws random numbers and builds test instances.  It holds
none of the method's arithmetic (no rounding rule, no scoring, no
truncation), so both the CUDA path and the FP64 oracle may take their inputs
from it.  Every generator is a pure function of its seed.

Workload shapes follow the paper's synthetic families:

* i.i.d. complex Gaussian factors V ~ CN(0, 1) (Sec. 4, "Gaussian noise"
  definition: Re, Im ~ N(0, 1/2)), optionally with per-column scales;
* directions drawn uniformly on the complex unit sphere (Sec. 4.2, Lemma
  "innerIsBeta": c = Z / ||Z||, Z ~ CN(0, I_r)) -- the random numbers the
  sampling method draws, passed in as inputs;
* graph families of the Max-3-Cut experiments (Sec. 5, App. G): stochastic
  block model, toroidal lattice.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def complex_gaussian(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """i.i.d. CN(0, 1): real and imaginary parts N(0, 1/2)."""
    g = rng(seed)
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return ((re + 1j * im) / np.sqrt(2.0)).astype(dtype)


def factor(n: int, r: int, seed: int, scales=None, dtype=np.complex128) -> np.ndarray:
    """V in C^{n x r}, CN(0,1) entries times optional column scales."""
    V = complex_gaussian((n, r), seed, np.complex128)
    if scales is not None:
        V = V * np.asarray(scales, dtype=np.float64)[None, :]
    return V.astype(dtype)


def directions(S: int, r: int, seed: int, dtype=np.complex64) -> np.ndarray:
    """S directions uniform on the unit sphere of C^r (rows)."""
    Z = complex_gaussian((S, r), seed, np.complex128)
    Z = Z / np.linalg.norm(Z, axis=1, keepdims=True)
    return Z.astype(dtype)


def planted_rank1(n: int, r: int, K: int, seed: int, dtype=np.complex64):
    """V_i = a_i * omega^{k_i} * u^T with a_i > 0, k_i uniform, unit u.

    Returns (V, a, k, u) where V is exactly representable in `dtype` up to
    the rounding of its entries (a, k, u are returned in FP64 for the
    closed-form checks; V is rounded once)."""
    g = rng(seed)
    a = 0.5 + g.random(n)
    k = g.integers(0, K, n)
    u = g.standard_normal(r) + 1j * g.standard_normal(r)
    u = u / np.linalg.norm(u)
    omega = np.exp(2j * np.pi * k / K)
    V = (a * omega)[:, None] * u[None, :]
    return V.astype(dtype), a, k, u


def hermitian_gaussian(n: int, seed: int) -> np.ndarray:
    """H = (G + G^H) / 2 with G i.i.d. CN(0, 1) (a GUE-like Hermitian matrix)."""
    G = complex_gaussian((n, n), seed, np.complex128)
    return 0.5 * (G + G.conj().T)


def _csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray):
    """Symmetric CSR (int32) from an undirected edge list without duplicates."""
    rows = np.concatenate([src, dst]).astype(np.int64)
    cols = np.concatenate([dst, src]).astype(np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for int32 CSR")
    return rowptr.astype(np.int32), cols.astype(np.int32)


def torus_graph(k1: int, k2: int):
    """k1 x k2 toroidal lattice (4-regular for k1, k2 >= 3), symmetric CSR."""
    if k1 < 3 or k2 < 3:
        raise ValueError("torus sides must be >= 3 to avoid multi-edges")
    idx = np.arange(k1 * k2).reshape(k1, k2)
    right = np.roll(idx, -1, axis=1)
    down = np.roll(idx, -1, axis=0)
    src = np.concatenate([idx.ravel(), idx.ravel()])
    dst = np.concatenate([right.ravel(), down.ravel()])
    return _csr_from_edges(k1 * k2, src, dst)


def sbm_graph(n: int, p_in_n: float, p_out_n: float, seed: int, blocks: int = 3):
    """Stochastic block model with `blocks` balanced communities.

    Edge probability p_in = p_in_n / n inside a block and p_out = p_out_n / n
    between blocks.  Sampled in O(m): a binomial edge count per block pair,
    then uniform endpoint pairs; self loops and duplicates are rejected and
    redrawn.  Returns (rowptr, colidx, labels)."""
    g = rng(seed)
    labels = np.arange(n) % blocks
    members = [np.flatnonzero(labels == b) for b in range(blocks)]
    src_all, dst_all = [], []
    for a in range(blocks):
        for b in range(a, blocks):
            na, nb = len(members[a]), len(members[b])
            if a == b:
                pairs = na * (na - 1) // 2
                p = p_in_n / n
            else:
                pairs = na * nb
                p = p_out_n / n
            m = int(g.binomial(pairs, min(p, 1.0)))
            keys = np.empty(0, dtype=np.int64)
            while len(keys) < m:
                need = int((m - len(keys)) * 1.1) + 16
                s = members[a][g.integers(0, na, need)]
                d = members[b][g.integers(0, nb, need)]
                lo, hi = np.minimum(s, d), np.maximum(s, d)
                keep = lo != hi
                keys = np.unique(np.concatenate([keys, lo[keep] * n + hi[keep]]))
            if len(keys) > m:
                keys = np.sort(g.permutation(keys)[:m])
            got_s, got_d = keys // n, keys % n
            src_all.append(got_s)
            dst_all.append(got_d)
    src = np.concatenate(src_all)
    dst = np.concatenate(dst_all)
    rowptr, colidx = _csr_from_edges(n, src, dst)
    return rowptr, colidx, labels


def batched_shapes(P: int, seed: int, n_lo: int = 64, n_hi: int = 8192,
                   ranks=(2, 3, 4, 5, 6), alphabets=(2, 3, 4, 8)):
    """Per-problem (n, r, K) for a batch of uneven instances: n log-uniform in
    [n_lo, n_hi], r and K uniform over the given sets."""
    g = rng(seed)
    n = np.floor(np.exp(g.uniform(np.log(n_lo), np.log(n_hi), P))).astype(np.int64)
    r = g.choice(np.asarray(ranks), P)
    K = g.choice(np.asarray(alphabets), P)
    return n, r, K
