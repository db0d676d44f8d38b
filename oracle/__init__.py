"""FP64 CPU oracle for the low-rank method of arXiv 2602.20376.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  The product path (the CUDA library and its Python binding) never
imports it, and the two share no code.

Pieces and the passages they follow:

* ``lrq_oracle.c`` (plain C, FP64): decision rule (Sec. 3, Eq. 9), sampled
  objective f(c) = ||V^H z(c)||^2 (Sec. 4.2, Eq. 10), objective ||V^H z||^2
  (Sec. 2.2, Eq. 3), brute force over A_K^n (Eq. 1), exact rank-1 sweep
  (Sec. 2.5, Algorithm 1), Max-K-Cut count and Laplacian quadratic form
  (Sec. 1), Philox4x32-10 + Box-Muller sphere sampler (Sec. 4.2, App. E
  Lemma "innerIsBeta").
* ``enumerate_vertices`` (numpy): vertex enumeration of the hyperplane
  arrangement (Sec. 3, Algorithm 2, with the augmented matrix of Eq. 6), in
  the superset reading described in its docstring; SVD is the library step
  that yields each null vector.
* ``rank1_sweep_states`` / ``rank1_sweep_cut`` (numpy): the n + 1 states of
  the rank-1 sweep and their exact cuts; ``greedy_cut`` (numpy): greedy
  local search on the cut from a given partition (the hybrid warm start,
  App. "Hybrid Warm-Start"), in the round reading given in its docstring.
* ``null_directions`` (numpy): the null-vector sampler of Sec. 5 (the
  randomised Algorithm 2), drawing rows with the Philox generator above.
* ``spectral_energy`` (numpy): the spectral energy ratio rho_r (Sec. 5)
  from the full spectrum (LAPACK ``eigvalsh``).
* ``truncate_dense`` / ``truncate_laplacian``: spectral truncation
  (Sec. 4.1, Algorithm 3) through LAPACK ``eigh`` and ARPACK ``eigsh``
  (the paper's own eigen-solver, Sec. 5).

* ``learned.py`` (numpy FP64): the learned proposal, which the paper does
  not have: spectral features with a phase gauge, the 3-layer MLP forward
  and backward, the von Mises-Fisher mixture head on S^7 with its negative
  log-likelihood and gradient, Wood's vMF sampler, the canonical window of
  the K-fold equivalence (Sec. 2.1, 2.3) and Adam.

Parity pins for every function live in ``tests/test_oracle_*.py``.  Parity
unpinned: none of the functions above; the learned-proposal gain over uniform
sampling (an empirical claim no passage of the paper defines) is measured,
not pinned.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lrq_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblrq_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_decide.argtypes = [D, D, I]
        lib.oracle_decide.restype = I
        lib.oracle_decide_array.argtypes = [P, P, I64, I, P]
        lib.oracle_decide_array.restype = None
        lib.oracle_boundary_margin.argtypes = [D, D, I]
        lib.oracle_boundary_margin.restype = D
        lib.oracle_objective.argtypes = [P, I64, I, I, P]
        lib.oracle_objective.restype = D
        lib.oracle_score.argtypes = [P, I64, I, I, P, I64, P, P, I]
        lib.oracle_score.restype = I
        lib.oracle_margins.argtypes = [P, I64, I, I, P, I64, P, P]
        lib.oracle_margins.restype = I
        lib.oracle_bruteforce.argtypes = [P, I64, I, I, P]
        lib.oracle_bruteforce.restype = D
        lib.oracle_quadform.argtypes = [P, I64, I, P]
        lib.oracle_quadform.restype = D
        lib.oracle_quadform_bruteforce.argtypes = [P, I64, I, P]
        lib.oracle_quadform_bruteforce.restype = D
        lib.oracle_cut_count.argtypes = [P, P, I64, P]
        lib.oracle_cut_count.restype = I64
        lib.oracle_laplacian_quadform.argtypes = [P, P, I64, I, P]
        lib.oracle_laplacian_quadform.restype = D
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_sphere_sample.argtypes = [ctypes.c_uint64, I64, I, P]
        lib.oracle_sphere_sample.restype = None
        lib.oracle_rank1_sweep.argtypes = [P, I64, I, P]
        lib.oracle_rank1_sweep.restype = D
        lib.oracle_greedy_sequential.argtypes = [P, P, I64, I, P, I64]
        lib.oracle_greedy_sequential.restype = I64
        _lib = lib
        return lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Decision rule, objective, scoring (Eq. 3, Eq. 9, Eq. 10)
# --------------------------------------------------------------------------
def decide(w, K: int) -> np.ndarray:
    """Codes k = argmax_k Re(conj(omega^k) w) for an array of complex w."""
    w = _c128(w).ravel()
    x = np.ascontiguousarray(w.real)
    y = np.ascontiguousarray(w.imag)
    out = np.empty(w.size, dtype=np.uint8)
    _load().oracle_decide_array(_ptr(x), _ptr(y), w.size, int(K), _ptr(out))
    return out


def objective(V, K: int, z) -> float:
    """||V^H z||^2 for codes z in [0, K)^n."""
    V = _c128(V)
    n, r = V.shape
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint8))
    return float(_load().oracle_objective(_ptr(V), n, r, int(K), _ptr(z)))


def score(V, K: int, C, want_z: bool = False, nthreads: int = 0):
    """f(c_s) = ||V^H z(c_s)||^2 for every row c_s of C (S x r)."""
    V = _c128(V)
    C = _c128(C)
    n, r = V.shape
    S = C.shape[0]
    assert C.shape[1] == r
    f = np.empty(S, dtype=np.float64)
    z = np.empty((S, n), dtype=np.uint8) if want_z else None
    rc = _load().oracle_score(_ptr(V), n, r, int(K), _ptr(C), S, _ptr(f),
                              _ptr(z) if want_z else None, int(nthreads))
    if rc != 0:
        raise ValueError("oracle_score rejected its arguments")
    return (f, z) if want_z else f


def margins(V, K: int, C):
    """Per (s, i): angular distance of arg(V_i c_s) to the nearest decision
    boundary, and |V_i c_s|."""
    V = _c128(V)
    C = _c128(C)
    n, r = V.shape
    S = C.shape[0]
    m = np.empty((S, n), dtype=np.float64)
    a = np.empty((S, n), dtype=np.float64)
    _load().oracle_margins(_ptr(V), n, r, int(K), _ptr(C), S, _ptr(m), _ptr(a))
    return m, a


def bruteforce(V, K: int):
    """max over all K^n assignments of ||V^H z||^2 (the definition of OPT)."""
    V = _c128(V)
    n, r = V.shape
    z = np.empty(n, dtype=np.uint8)
    f = _load().oracle_bruteforce(_ptr(V), n, r, int(K), _ptr(z))
    return float(f), z


def quadform(Q, K: int, z) -> float:
    Q = _c128(Q)
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint8))
    return float(_load().oracle_quadform(_ptr(Q), Q.shape[0], int(K), _ptr(z)))


def quadform_bruteforce(Q, K: int):
    Q = _c128(Q)
    z = np.empty(Q.shape[0], dtype=np.uint8)
    f = _load().oracle_quadform_bruteforce(_ptr(Q), Q.shape[0], int(K), _ptr(z))
    return float(f), z


# --------------------------------------------------------------------------
# Graphs (Sec. 1: Max-3-Cut is K = 3 with a Laplacian objective)
# --------------------------------------------------------------------------
def cut_count(rowptr, colidx, z) -> int:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint8))
    return int(_load().oracle_cut_count(_ptr(rowptr), _ptr(colidx), len(rowptr) - 1, _ptr(z)))


def laplacian_quadform(rowptr, colidx, K: int, z) -> float:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint8))
    return float(_load().oracle_laplacian_quadform(_ptr(rowptr), _ptr(colidx),
                                                   len(rowptr) - 1, int(K), _ptr(z)))


def laplacian_dense(rowptr, colidx, weights=None) -> np.ndarray:
    """Dense L = D - A of a symmetric CSR graph (unit weights unless given);
    self loops cancel in D - A."""
    n = len(rowptr) - 1
    L = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            j = colidx[e]
            if j == i:
                continue
            w = 1.0 if weights is None else float(weights[e])
            L[i, j] -= w
            L[i, i] += w
    return L


# --------------------------------------------------------------------------
# Random directions (Sec. 4.2)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sphere_sample(seed: int, S: int, r: int) -> np.ndarray:
    """Uniform directions on the unit sphere of C^r (FP64), Philox counter
    (s, j) under key `seed`, Box-Muller; see lrq_oracle.c."""
    C = np.empty((S, r), dtype=np.complex128)
    _load().oracle_sphere_sample(ctypes.c_uint64(int(seed)), S, r, _ptr(C))
    return C


# --------------------------------------------------------------------------
# Exact rank-1 sweep (Sec. 2.5, Algorithm 1)
# --------------------------------------------------------------------------
def rank1_sweep(q, K: int):
    q = _c128(q).ravel()
    z = np.empty(q.size, dtype=np.uint8)
    f = _load().oracle_rank1_sweep(_ptr(q), q.size, int(K), _ptr(z))
    return float(f), z


def rank1_sweep_states(q, K: int):
    """The n + 1 states of the rank-1 angular sweep (Sec. 2.5, Algorithm 1):
    state 0 has codes floor(t_i) mod K, t_i = K arg(q_i) / (2 pi); coordinate
    i advances at phi_i = (2 pi / K)(1/2 + floor(t_i) - t_i); state s has
    advanced the first s coordinates in the order (phi_i, i).  Returns
    (codes of state 0, the advancing order)."""
    q = _c128(q).ravel()
    t = K * np.arctan2(q.imag, q.real) / (2 * np.pi)
    fl = np.floor(t)
    phi = (2 * np.pi / K) * (0.5 + fl - t)
    order = np.lexsort((np.arange(q.size), phi))
    return (np.mod(fl, K)).astype(np.uint8), order


def two_eigvec_q(V, lam):
    """Two-eigenvector complex rounding (App. "Two-Eigenvector Complex
    Rounding", Eq. 12): q = u_1 + i u_2 with u_j the real unit eigenvectors,
    here recovered from V = [sqrt(lambda_j) u_j] (0 where lambda_j <= 0)."""
    V = np.asarray(V)
    u = [V[:, j].real / np.sqrt(lam[j]) if lam[j] > 0 else np.zeros(V.shape[0]) for j in (0, 1)]
    return u[0] + 1j * u[1]


def rank1_sweep_cut(q, K: int, rowptr, colidx):
    """Every state of the rank-1 sweep scored on the graph's exact cut
    (Max-K-Cut, Sec. 1); returns (best cut, its codes, all n + 1 cuts), ties
    to the earliest state."""
    z, order = rank1_sweep_states(q, K)
    z = z.copy()
    cuts = [cut_count(rowptr, colidx, z)]
    best, best_z = cuts[0], z.copy()
    for i in order:
        z[i] = (z[i] + 1) % K
        c = cut_count(rowptr, colidx, z)
        cuts.append(c)
        if c > best:
            best, best_z = c, z.copy()
    return best, best_z, np.array(cuts)


# --------------------------------------------------------------------------
# Greedy local search for Max-K-Cut (hybrid warm start, App. "Hybrid
# Warm-Start")
# --------------------------------------------------------------------------
def greedy_cut(rowptr, colidx, K: int, z, max_rounds=None):
    """Greedy hill-climbing on the exact cut from labels z (Sec. 1 objective;
    the hybrid solver runs it from the rank-1 partition).

    Reading of "steepest ascent" for a data-parallel round: with neighbour
    counts n_i(c) (self loops ignored, parallel edges with multiplicity),
    vertex i gains g_i = n_i(z_i) - min_{c != z_i} n_i(c) by moving to the
    smallest label attaining that minimum.  A round moves every vertex with
    g_i > 0 that has no neighbour j with g_j > g_i, or g_j = g_i and j < i.
    Rounds repeat until one moves nothing or max_rounds have run.
    Returns (labels uint8, rounds that moved, vertices moved, converged)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colidx = np.asarray(colidx, dtype=np.int64)
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    keep = colidx != rows
    src, dst = rows[keep], colidx[keep]
    z = np.asarray(z, dtype=np.int64).copy()
    ar = np.arange(n)
    rounds = moves = ran = 0
    converged = False
    while max_rounds is None or ran < max_rounds:
        ran += 1
        cnt = np.zeros((n, K), dtype=np.int64)
        np.add.at(cnt, (src, z[dst]), 1)
        same = cnt[ar, z]
        other = cnt.copy()
        other[ar, z] = np.iinfo(np.int64).max
        best = np.argmin(other, axis=1)          # first minimum: smallest label
        gain = np.maximum(same - other[ar, best], 0)
        gi, gj = gain[src], gain[dst]
        outranked = (gj > gi) | ((gj == gi) & (dst < src))
        blocked = np.bincount(src, weights=outranked, minlength=n) > 0
        mv = (gain > 0) & ~blocked
        if not mv.any():
            converged = True
            break
        z[mv] = best[mv]
        rounds += 1
        moves += int(mv.sum())
    return z.astype(np.uint8), rounds, moves, converged


def greedy_sequential(rowptr, colidx, K: int, z, max_moves=None):
    """Sequential steepest ascent from labels z: one move at a time, always the
    vertex of largest gain (ties to the smaller index), to the smallest label
    attaining its minimum neighbour count, until no vertex gains.  The other
    reading of the appendix's "steepest ascent" (greedy_cut moves, per round,
    every gaining vertex no neighbour outranks).  Returns (labels uint8,
    moves)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.uint8).copy())
    mv = _load().oracle_greedy_sequential(_ptr(rp), _ptr(ci), len(rp) - 1, int(K), _ptr(zz),
                                          -1 if max_moves is None else int(max_moves))
    if mv < 0:
        raise ValueError("oracle_greedy_sequential rejected its arguments")
    return zz, int(mv)


# --------------------------------------------------------------------------
# Exact rank-r vertex enumeration (Sec. 3, Algorithm 2)
# --------------------------------------------------------------------------
def effective_boundaries(K: int) -> int:
    """B_K of Definition 2.1: K/2 for even K, K for odd K."""
    return K // 2 if K % 2 == 0 else K


def augmented_rows(Vd, K: int) -> np.ndarray:
    """Rows of the augmented real matrix (Eq. 6) in interleaved order
    j = i * B_K + m.  Row (i, m) is [Im(rho_m V_i), Re(rho_m V_i)] with
    rho_m = exp(-i pi (2m+1)/K), so that row . [Re c; Im c] equals
    Im(rho_m V_i c): zero exactly when V_i c lies on boundary m."""
    Vd = _c128(Vd)
    n, d = Vd.shape
    BK = effective_boundaries(K)
    rho = np.exp(-1j * np.pi * (2 * np.arange(BK) + 1) / K)
    RV = rho[None, :, None] * Vd[:, None, :]  # n x BK x d
    H = np.concatenate([RV.imag, RV.real], axis=2)
    return H.reshape(n * BK, 2 * d)


def full_rank_by_elimination(H, tol: float = 1e-10) -> bool:
    """Rank test of an m x (m+1) matrix taken in the sampler's precision:
    FP64 Gaussian elimination with full pivoting (first largest entry in
    row-major order), failing when the largest remaining pivot is at or
    below tol * max|H|."""
    A = np.array(H, dtype=np.float64)
    m = A.shape[0]
    scale = np.abs(A).max() if A.size else 0.0
    if scale == 0.0:
        return False
    for k in range(m):
        sub = np.abs(A[k:, k:])
        p = int(np.argmax(sub))
        pr, pc = k + p // sub.shape[1], k + p % sub.shape[1]
        if sub.flat[p] <= tol * scale:
            return False
        A[[k, pr]] = A[[pr, k]]
        A[:, [k, pc]] = A[:, [pc, k]]
        for i in range(k + 1, m):
            A[i, k:] -= (A[i, k] / A[k, k]) * A[k, k:]
    return True


def null_directions(V, K: int, seed: int, S: int, attempts: int = 64):
    """The null-vector sampler (Sec. 5; the randomised form of Algorithm 2):
    each slot draws 2r - 1 distinct rows of the augmented matrix (Eq. 6)
    until they are linearly independent, and returns their unit null vector
    as c = c~[:r] + i c~[r:].  Draw convention (Philox4x32-10, the counter
    layout and the sign rule) as stated for lrq_sample_null_directions; the
    null vector is the last right singular vector (SVD, a library step).
    Returns (C complex128 S x r, draws per slot; 0 rows where a slot failed)."""
    V = _c128(V)
    n, r = V.shape
    rows = augmented_rows(V, K)
    N = rows.shape[0]
    m = 2 * r - 1
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    C = np.zeros((S, r), dtype=np.complex128)
    draws = np.zeros(S, dtype=np.int64)
    for s in range(S):
        for a in range(attempts):
            draws[s] += 1
            idx, neg, ok = [], False, True
            for j in range(m):
                got = False
                for t in range(16):
                    w = philox4x32_10((s & 0xFFFFFFFF, s >> 32, (a << 8) | (j << 4) | t, 0x4E56), key)
                    if j == 0 and t == 0:
                        neg = bool(w[2] & 1)
                    R = (((int(w[0]) << 32) | int(w[1])) * N) >> 64
                    if R not in idx:
                        idx.append(R)
                        got = True
                        break
                if not got:
                    ok = False
                    break
            if not ok:
                continue
            H = rows[idx]
            if not full_rank_by_elimination(H):
                continue
            c = np.linalg.svd(H)[2][-1]
            c = c / np.linalg.norm(c)
            j = int(np.argmax(np.abs(c)))
            if (c[j] < 0) != neg:
                c = -c
            C[s] = c[:r] + 1j * c[r:]
            break
        else:
            C[s] = 0
    return C, draws


def valid_index_sets(n: int, BK: int, size: int) -> np.ndarray:
    """All index sets of `size` hyperplanes with at most two from any
    coordinate group (Sec. 3, 'Structural properties')."""
    out = []
    for I in itertools.combinations(range(n * BK), size):
        g = [j // BK for j in I]
        ok = True
        for a in range(len(g) - 2):
            if g[a] == g[a + 2]:  # sorted => three equal groups are adjacent
                ok = False
                break
        if ok:
            out.append(I)
    return np.asarray(out, dtype=np.int64).reshape(-1, size)


def _objectives_batch(V, K: int, Z: np.ndarray) -> np.ndarray:
    """||V^H z||^2 for every row of the code matrix Z (M x n), FP64."""
    zc = np.exp(2j * np.pi * Z.astype(np.float64) / K)  # M x n
    P = zc @ V.conj()  # M x r : row m is (V^H z_m)^T
    return np.sum(np.abs(P) ** 2, axis=1)


def enumerate_vertices(V, K: int, rank_tol: float = 1e-10, branch_tol: float = 1e-9,
                       levels=None, return_all: bool = False):
    """Exact maximiser of ||V^H z||^2 over A_K^n by vertex enumeration.

    Follows Algorithm 2 level by level, d = r, r-1, ..., 1 (the recursion on
    the leading columns V[:, :d]):

    1. build the augmented rows of V_d (Eq. 6) in interleaved order;
    2. for every valid index set I (|I| = 2d-1, at most two rows per
       coordinate group), take the null vector of the rows in I from the SVD,
       and skip I unless the rows have rank 2d-1 (smallest singular value
       above rank_tol times the largest);
    3. for both signs of the null vector form c = c[:d] + i c[d:] and
       w = V_d c;
    4. per coordinate, collect the codes of every cell that touches the
       vertex: all K codes where w_i = 0 (a coordinate with two rows in I,
       or |w_i| below branch_tol ||V_i||), the two codes on either side of
       the boundary where arg w_i is within branch_tol of one, and the
       decision-rule code (Eq. 9) otherwise;
    5. score every combination on the full-rank V and keep the best.

    Step 4 is the superset reading of the ambiguity resolution (Algorithm 4,
    App. B.3): instead of the fixed-angle solve it tries every code a cell
    adjacent to the vertex can carry, which contains the paper's candidates.

    Returns (best_f, best_z, stats) with stats = dict(index_sets, full_rank,
    candidates); with return_all=True stats also holds every scored value.
    """
    V = _c128(V)
    n, r = V.shape
    BK = effective_boundaries(K)
    levels = list(range(r, 0, -1)) if levels is None else list(levels)
    best_f, best_z = -1.0, None
    n_sets = n_full = n_cand = 0
    all_f = []
    ks = np.arange(K)
    bnd = np.pi * (2 * np.arange(K) + 1) / K  # decision boundaries theta_m
    rownorm = np.linalg.norm(V, axis=1)
    for d in levels:
        Vd = V[:, :d]
        H = augmented_rows(Vd, K)
        sets = valid_index_sets(n, BK, 2 * d - 1)
        n_sets += len(sets)
        if len(sets) == 0:
            continue
        HI = H[sets]  # N x (2d-1) x 2d
        _, sv, vh = np.linalg.svd(HI, full_matrices=True)
        full = sv[:, -1] > rank_tol * sv[:, 0]
        n_full += int(full.sum())
        nulls = vh[full, -1, :]  # N' x 2d
        groups = sets[full] // BK
        for t in range(nulls.shape[0]):
            g, cnt = np.unique(groups[t], return_counts=True)
            doubles = set(g[cnt == 2].tolist())
            for sign in (1.0, -1.0):
                ct = sign * nulls[t]
                c = ct[:d] + 1j * ct[d:]
                w = Vd @ c
                choices = []
                for i in range(n):
                    if i in doubles or abs(w[i]) <= branch_tol * max(rownorm[i], 1e-300):
                        choices.append(ks)
                        continue
                    th = np.angle(w[i])
                    dist = np.abs(np.angle(np.exp(1j * (th - bnd))))
                    m = int(np.argmin(dist))
                    if dist[m] <= branch_tol:
                        choices.append(np.array([m % K, (m + 1) % K]))
                    else:
                        choices.append(decide(w[i:i + 1], K))
                Z = np.array(list(itertools.product(*choices)), dtype=np.uint8)
                fz = _objectives_batch(V, K, Z)
                n_cand += len(Z)
                j = int(np.argmax(fz))
                if return_all:
                    all_f.append(fz)
                if fz[j] > best_f:
                    best_f, best_z = float(fz[j]), Z[j].copy()
    stats = dict(index_sets=n_sets, full_rank=n_full, candidates=n_cand)
    if return_all:
        stats["all_f"] = np.concatenate(all_f) if all_f else np.empty(0)
    return best_f, best_z, stats


def candidate_set_size(n: int, r: int, K: int) -> int:
    """Eq. 8 (Theorem 3.1): |S(V)| for the paper's windowed enumeration."""
    from math import comb
    BK = effective_boundaries(K)
    tot = 0
    for d in range(1, r + 1):
        for i in range(0, d):
            tot += comb(n, i) * comb(n - i, 2 * (d - i) - 1) * BK ** (2 * (d - i) - 2) * (BK - 1) ** i
    return tot


# --------------------------------------------------------------------------
# Spectral energy ratio (Sec. 5, "When does low-rank work?")
# --------------------------------------------------------------------------
def spectral_energy(Q, r: int) -> float:
    """rho_r = 1 - (sum of the r largest positive eigenvalues) / (sum of all
    positive eigenvalues) of a Hermitian Q, from its full spectrum (LAPACK
    eigvalsh); 0 for Q without positive eigenvalues."""
    lam = np.linalg.eigvalsh(0.5 * (np.asarray(Q) + np.asarray(Q).conj().T))
    pos = np.sort(lam[lam > 0])[::-1]
    if pos.size == 0:
        return 0.0
    return float(1.0 - pos[:r].sum() / pos.sum())


# --------------------------------------------------------------------------
# Spectral truncation (Sec. 4.1, Algorithm 3)
# --------------------------------------------------------------------------
def truncate_dense(Q, r: int):
    """Top-r eigenpairs of a Hermitian Q (largest algebraic), V = U sqrt(lam).
    Eigenvalues <= 0 are dropped (their columns are zero): a maximisation
    gains nothing from a negative direction.  Returns (V, lam) with lam
    descending."""
    Q = _c128(Q)
    Q = 0.5 * (Q + Q.conj().T)
    lam, U = np.linalg.eigh(Q)
    order = np.argsort(lam)[::-1][:r]
    lam = lam[order]
    U = U[:, order]
    keep = lam > 0
    V = np.zeros((Q.shape[0], r), dtype=np.complex128)
    V[:, keep] = U[:, keep] * np.sqrt(lam[keep])[None, :]
    return V, lam


def truncate_laplacian(rowptr, colidx, r: int, tol: float = 1e-12, weights=None):
    """Top-r eigenpairs of the graph Laplacian L = D - A (unit weights unless
    given; self loops cancel) via ARPACK (scipy eigsh), the eigen-solver the
    paper uses (Sec. 5)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n = len(rowptr) - 1
    rowptr = np.asarray(rowptr)
    colidx = np.asarray(colidx)
    w = np.ones(len(colidx)) if weights is None else np.asarray(weights, dtype=np.float64)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    w = np.where(colidx == rows, 0.0, w)
    A = sp.csr_matrix((w, colidx, rowptr), shape=(n, n))
    deg = np.asarray(A.sum(axis=1)).ravel()
    L = sp.diags(deg) - A
    # ARPACK may skip a copy of a repeated eigenvalue when asked for exactly
    # r pairs; ask for a few more and keep the top r.
    k = min(n - 1, r + 8)
    lam, U = spla.eigsh(L, k=k, which="LA", tol=tol, ncv=min(n, max(2 * k + 1, 40)))
    order = np.argsort(lam)[::-1][:r]
    lam = lam[order]
    U = U[:, order]
    keep = lam > 0
    V = np.zeros((n, r), dtype=np.complex128)
    V[:, keep] = U[:, keep] * np.sqrt(lam[keep])[None, :]
    return V, lam
