// k_rank1.cu -- exact rank-1 solver by an angular sweep (Sec. 2.5,
// Algorithm 1), and the same sweep scored on a graph's exact cut.
//
// For Q = q q^H the objective of z(c) with c = exp(i phi) is |q^H z|^2.  As
// phi runs over one period 2 pi / K, every coordinate's rounded code
// advances exactly once, at the angle where arg(q_i) + phi crosses a
// decision boundary (Sec. 2.5: the optimum is one of these n + 1 states).
// Convention (shared with the oracle): t_i = K arg(q_i) / (2 pi), the start
// code is floor(t_i) mod K and coordinate i advances at
// phi_i = (2 pi / K)(1/2 + floor(t_i) - t_i); states are the prefixes of the
// coordinates sorted by (phi_i, i).
//
// GPU steps: per-coordinate key (FP64), a bitonic sort of (key, index)
// pairs, the increments conj(q_i) w^{k_i} (w - 1) in sorted order, an FP64
// prefix scan giving q^H z for every state, and the argmax (ties to the
// earliest state).  With a CSR graph every undirected edge adds its change
// of cut to a difference array at the two states where one, then both, of
// its ends have advanced; an int64 prefix scan gives the exact cut of every
// state (Max-K-Cut reading of Sec. 1).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kR1Threads = 256;
constexpr int kR1Local = 2048;  // elements sorted per block in shared memory
constexpr int kR1Scan = 1024;   // elements per block in the scans

struct R1Tables {
  double zr[kMaxK], zi[kMaxK];
};

// order-preserving map of a double to uint64
__device__ __forceinline__ uint64_t r1_key(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void r1_prep_kernel(const double2* __restrict__ q, int64_t n, int64_t npad, int K,
                               uint64_t* __restrict__ key, uint32_t* __restrict__ idx, uint8_t* __restrict__ code0,
                               int32_t* status) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i >= n) {
    key[i] = ~0ull;
    idx[i] = 0xFFFFFFFFu;
    return;
  }
  const double2 v = q[i];
  if (!isfinite(v.x) || !isfinite(v.y)) dev_fail(status, LRQ_EINVAL);
  const double th = atan2(v.y, v.x);
  const double t = static_cast<double>(K) * th / (2.0 * kPi);
  const double fl = floor(t);
  const double phi = (2.0 * kPi / static_cast<double>(K)) * (0.5 + fl - t);
  long long kk = static_cast<long long>(fl) % K;
  if (kk < 0) kk += K;
  key[i] = r1_key(phi);
  idx[i] = static_cast<uint32_t>(i);
  code0[i] = static_cast<uint8_t>(kk);
}

__device__ __forceinline__ bool r1_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// the bitonic stages with partner distance j <= kR1Local / 2 run in shared
// memory: a block owns kR1Local consecutive elements and handles the merge
// sizes k_first..k_last (2..kR1Local in the first pass, one k later)
__global__ void __launch_bounds__(kR1Local / 2) r1_sort_local(uint64_t* __restrict__ key, uint32_t* __restrict__ idx,
                                                              int64_t k_first, int64_t k_last) {
  __shared__ uint64_t sk[kR1Local];
  __shared__ uint32_t si[kR1Local];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kR1Local;
  for (int t = threadIdx.x; t < kR1Local; t += blockDim.x) {
    sk[t] = key[base + t];
    si[t] = idx[base + t];
  }
  __syncthreads();
  for (int64_t k = k_first; k <= k_last; k <<= 1) {
    for (int64_t j = (k >> 1) < (kR1Local >> 1) ? (k >> 1) : (kR1Local >> 1); j > 0; j >>= 1) {
      const int t = threadIdx.x;
      const int a = static_cast<int>((t / j) * 2 * j + (t % j));
      const int b = a + static_cast<int>(j);
      const int64_t ga = base + a;
      const bool up = (ga & k) == 0;
      const bool sw = up ? r1_less(sk[b], si[b], sk[a], si[a]) : r1_less(sk[a], si[a], sk[b], si[b]);
      if (sw) {
        const uint64_t tk = sk[a];
        sk[a] = sk[b];
        sk[b] = tk;
        const uint32_t ti = si[a];
        si[a] = si[b];
        si[b] = ti;
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < kR1Local; t += blockDim.x) {
    key[base + t] = sk[t];
    idx[base + t] = si[t];
  }
}

// one bitonic stage (merge size k, partner distance j >= kR1Local / 2) in
// global memory; a thread per pair
__global__ void r1_sort_global(uint64_t* __restrict__ key, uint32_t* __restrict__ idx, int64_t npad, int64_t k,
                               int64_t j) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= npad / 2) return;
  const int64_t a = (t / j) * 2 * j + (t % j), b = a + j;
  const bool up = (a & k) == 0;
  const uint64_t ka = key[a], kb = key[b];
  const uint32_t ia = idx[a], ib = idx[b];
  const bool sw = up ? r1_less(kb, ib, ka, ia) : r1_less(ka, ia, kb, ib);
  if (sw) {
    key[a] = kb;
    key[b] = ka;
    idx[a] = ib;
    idx[b] = ia;
  }
}

// increments of q^H z in sorted order: d_l = conj(q_i) w^{k_i} (w - 1),
// and the rank of every coordinate
__global__ void r1_delta_kernel(const double2* __restrict__ q, int64_t n, int K, const uint32_t* __restrict__ idx,
                                const uint8_t* __restrict__ code0, const __grid_constant__ R1Tables tb,
                                double2* __restrict__ d, uint32_t* __restrict__ rank) {
  const int64_t l = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const uint32_t i = idx[l];
  rank[i] = static_cast<uint32_t>(l);
  const double2 v = q[i];
  const int c = code0[i], c1 = (c + 1) % K;
  const double dzr = tb.zr[c1] - tb.zr[c], dzi = tb.zi[c1] - tb.zi[c];
  // conj(v) * dz
  d[l] = make_double2(v.x * dzr + v.y * dzi, v.x * dzi - v.y * dzr);
}

// S0 = sum_i conj(q_i) w^{code0_i}, per-block partial sums (fixed order)
__global__ void r1_base_kernel(const double2* __restrict__ q, int64_t n, const uint8_t* __restrict__ code0,
                               const __grid_constant__ R1Tables tb, double2* __restrict__ part) {
  __shared__ double2 red[kR1Threads];
  double2 s = make_double2(0.0, 0.0);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double2 v = q[i];
    const int c = code0[i];
    s.x += v.x * tb.zr[c] + v.y * tb.zi[c];
    s.y += v.x * tb.zi[c] - v.y * tb.zr[c];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[threadIdx.x].x += red[threadIdx.x + h].x;
      red[threadIdx.x].y += red[threadIdx.x + h].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---- inclusive scans in three passes (block sums, scan of block sums, add)
template <typename T>
__device__ __forceinline__ T r1_add(T a, T b);
template <>
__device__ __forceinline__ double2 r1_add<double2>(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
template <>
__device__ __forceinline__ long long r1_add<long long>(long long a, long long b) {
  return a + b;
}
template <typename T>
__device__ __forceinline__ T r1_zero();
template <>
__device__ __forceinline__ double2 r1_zero<double2>() {
  return make_double2(0.0, 0.0);
}
template <>
__device__ __forceinline__ long long r1_zero<long long>() {
  return 0;
}

// in-block inclusive scan of kR1Scan elements (256 threads x 4), writes the
// block total
template <typename T>
__global__ void __launch_bounds__(kR1Threads) r1_scan_block(T* __restrict__ x, int64_t n, T* __restrict__ sums) {
  __shared__ T s[kR1Scan];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kR1Scan;
  for (int t = threadIdx.x; t < kR1Scan; t += blockDim.x) s[t] = (base + t < n) ? x[base + t] : r1_zero<T>();
  __syncthreads();
  // Hillis-Steele over the block (log2 1024 = 10 rounds)
  for (int off = 1; off < kR1Scan; off <<= 1) {
    T v[kR1Scan / kR1Threads];
#pragma unroll
    for (int u = 0; u < kR1Scan / kR1Threads; ++u) {
      const int t = threadIdx.x + u * kR1Threads;
      v[u] = (t >= off) ? r1_add<T>(s[t], s[t - off]) : s[t];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kR1Scan / kR1Threads; ++u) s[threadIdx.x + u * kR1Threads] = v[u];
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kR1Scan; t += blockDim.x)
    if (base + t < n) x[base + t] = s[t];
  if (threadIdx.x == 0) sums[blockIdx.x] = s[kR1Scan - 1];
}

// exclusive offsets of the block sums, sequentially (nb is small)
template <typename T>
__global__ void r1_scan_sums(T* __restrict__ sums, int64_t nb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  T acc = r1_zero<T>();
  for (int64_t b = 0; b < nb; ++b) {
    const T v = sums[b];
    sums[b] = acc;
    acc = r1_add<T>(acc, v);
  }
}

template <typename T>
__global__ void r1_scan_add(T* __restrict__ x, int64_t n, const T* __restrict__ sums) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = r1_add<T>(x[i], sums[i / kR1Scan]);
}

// f of states 1..n (state l+1 = prefix l inclusive) and the argmax over
// states 0..n; one block, fixed order, ties to the earliest state
__global__ void r1_best_kernel(const double2* __restrict__ pref, int64_t n, const double2* __restrict__ base_part,
                               int nbase, int64_t* __restrict__ best_state, double* __restrict__ best_f) {
  __shared__ double bf[kR1Threads];
  __shared__ long long bs[kR1Threads];
  __shared__ double2 s0;
  if (threadIdx.x == 0) {
    double2 a = make_double2(0.0, 0.0);
    for (int b = 0; b < nbase; ++b) {
      a.x += base_part[b].x;
      a.y += base_part[b].y;
    }
    s0 = a;
  }
  __syncthreads();
  double f = s0.x * s0.x + s0.y * s0.y;
  long long st = 0;
  if (threadIdx.x != 0) f = -1.0;
  for (int64_t l = threadIdx.x; l < n; l += blockDim.x) {
    const double2 p = pref[l];
    const double x = s0.x + p.x, y = s0.y + p.y;
    const double g = x * x + y * y;
    if (g > f) {
      f = g;
      st = l + 1;
    }
  }
  bf[threadIdx.x] = f;
  bs[threadIdx.x] = st;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const double o = bf[threadIdx.x + h];
      const long long os = bs[threadIdx.x + h];
      if (o > bf[threadIdx.x] || (o == bf[threadIdx.x] && os < bs[threadIdx.x])) {
        bf[threadIdx.x] = o;
        bs[threadIdx.x] = os;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *best_state = bs[0];
    *best_f = bf[0];
  }
}

// codes of state s: coordinates of rank < s have advanced by one
__global__ void r1_codes_kernel(const uint8_t* __restrict__ code0, const uint32_t* __restrict__ rank, int64_t n,
                                int K, const int64_t* __restrict__ state, uint8_t* __restrict__ z) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t s = *state;
  const int c = code0[i] + (static_cast<int64_t>(rank[i]) < s ? 1 : 0);
  z[i] = static_cast<uint8_t>(c % K);
}

// every undirected edge {i, j} (stored in both rows; j > i counted): its cut
// in state 0 into cut0, and its change at the state where its first end
// advances (undone where the second advances) into the difference array
__global__ void r1_edge_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t n,
                               int64_t nnz, int K, const uint8_t* __restrict__ code0, const uint32_t* __restrict__ rank,
                               long long* __restrict__ diff, unsigned long long* __restrict__ cut0) {
  unsigned long long local = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int ci = code0[i];
    const uint32_t ri = rank[i];
    int64_t e0 = rowptr[i], e1 = rowptr[i + 1];  // bounds-guarded (a malformed CSR reads nothing outside)
    e0 = e0 < 0 ? 0 : (e0 > nnz ? nnz : e0);
    e1 = e1 < e0 ? e0 : (e1 > nnz ? nnz : e1);
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t j = colidx[e];
      if (j <= i || j >= n) continue;
      const int cj = code0[j];
      const uint32_t rj = rank[j];
      const int d0 = ((ci - cj) % K + K) % K;
      // the end with the smaller rank advances first
      const int dm = ri < rj ? (d0 + 1) % K : (d0 + K - 1) % K;
      const int c0 = d0 != 0, cm = dm != 0;
      local += static_cast<unsigned long long>(c0);
      if (cm != c0) {
        const uint32_t lo = ri < rj ? ri : rj, hi = ri < rj ? rj : ri;
        atomicAdd(reinterpret_cast<unsigned long long*>(&diff[lo + 1]), static_cast<unsigned long long>(cm - c0));
        atomicAdd(reinterpret_cast<unsigned long long*>(&diff[hi + 1]), static_cast<unsigned long long>(c0 - cm));
      }
    }
  }
  if (local) atomicAdd(cut0, local);
}

// the best state by cut (ties to the earliest); diff already prefix-summed
__global__ void r1_best_cut_kernel(const long long* __restrict__ pref, int64_t n,
                                   const unsigned long long* __restrict__ cut0, int64_t* __restrict__ best_state,
                                   int64_t* __restrict__ best_cut) {
  __shared__ long long bc[kR1Threads];
  __shared__ long long bs[kR1Threads];
  const long long c0 = static_cast<long long>(*cut0);
  long long c = -1, st = 0;
  for (int64_t s = threadIdx.x; s <= n; s += blockDim.x) {
    const long long v = c0 + pref[s];
    if (v > c) {
      c = v;
      st = s;
    }
  }
  bc[threadIdx.x] = c;
  bs[threadIdx.x] = st;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const long long o = bc[threadIdx.x + h], os = bs[threadIdx.x + h];
      if (o > bc[threadIdx.x] || (o == bc[threadIdx.x] && os < bs[threadIdx.x])) {
        bc[threadIdx.x] = o;
        bs[threadIdx.x] = os;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *best_state = bs[0];
    *best_cut = bc[0];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

int64_t r1_pad(int64_t n) {
  int64_t p = kR1Local;
  while (p < n) p <<= 1;
  return p;
}

struct R1Layout {
  int64_t n, npad, nscan_blocks, nscan_blocks_diff;
  size_t off_key, off_idx, off_code0, off_rank, off_d, off_sums, off_base, off_diff, off_dsums, off_cut0,
      off_state, off_state2, total;
};

R1Layout r1_layout(int64_t n) {
  R1Layout l;
  l.n = n;
  l.npad = r1_pad(n);
  l.nscan_blocks = ceil_div(n, kR1Scan);
  l.nscan_blocks_diff = ceil_div(n + 1, kR1Scan);
  size_t cur = 0;
  auto take = [&](size_t b) {
    size_t o = cur;
    cur = align_up(cur + b, 256);
    return o;
  };
  l.off_key = take(static_cast<size_t>(l.npad) * 8);
  l.off_idx = take(static_cast<size_t>(l.npad) * 4);
  l.off_code0 = take(static_cast<size_t>(n));
  l.off_rank = take(static_cast<size_t>(n) * 4);
  l.off_d = take(static_cast<size_t>(n) * 16);
  l.off_sums = take(static_cast<size_t>(l.nscan_blocks) * 16);
  l.off_base = take(static_cast<size_t>(kR1Threads) * 16);
  l.off_diff = take(static_cast<size_t>(n + 2) * 8);
  l.off_dsums = take(static_cast<size_t>(l.nscan_blocks_diff) * 8);
  l.off_cut0 = take(8);
  l.off_state = take(8);
  l.off_state2 = take(8);
  l.total = cur;
  return l;
}

template <typename T>
void r1_scan(T* x, int64_t n, T* sums, int64_t nb, cudaStream_t st) {
  r1_scan_block<T><<<static_cast<unsigned>(nb), kR1Threads, 0, st>>>(x, n, sums);
  r1_scan_sums<T><<<1, 32, 0, st>>>(sums, nb);
  r1_scan_add<T><<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(x, n, sums);
  count_launch(3);
}

}  // namespace

// two-eigenvector complex rounding vector (App. "Two-Eigenvector Complex
// Rounding", Eq. 12): q_i = u_1(i) + i u_2(i) from the real eigenvectors of
// a real symmetric Q, u_j = V_j / sqrt(lambda_j) (a column with
// lambda_j <= 0 contributes 0)
__global__ void r1_pair_kernel(const double2* __restrict__ V, int64_t n, int r, const double* __restrict__ lambda,
                               double2* __restrict__ q) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l0 = lambda[0], l1 = lambda[1];
  const double s0 = l0 > 0.0 ? 1.0 / sqrt(l0) : 0.0, s1 = l1 > 0.0 ? 1.0 / sqrt(l1) : 0.0;
  q[i] = make_double2(V[i * r].x * s0, V[i * r + 1].x * s1);
}

int launch_two_eigvec_q(const double2* V, int64_t n, int r, const double* lambda, double2* q, cudaStream_t st) {
  r1_pair_kernel<<<static_cast<unsigned>(ceil_div(n, kR1Threads)), kR1Threads, 0, st>>>(V, n, r, lambda, q);
  count_launch();
  return cuda_check(cudaGetLastError(), "r1_pair_kernel");
}

size_t rank1_workspace_bytes(int64_t n) { return r1_layout(n).total; }

int launch_rank1(const double2* q, int64_t n, int K, uint8_t* z_out, double* f_out, const int32_t* rowptr,
                 const int32_t* colidx, int64_t nnz, int64_t* cut_out, uint8_t* zcut_out, void* ws, int32_t* status,
                 cudaStream_t st) {
  const R1Layout L = r1_layout(n);
  uint8_t* w = static_cast<uint8_t*>(ws);
  uint64_t* key = reinterpret_cast<uint64_t*>(w + L.off_key);
  uint32_t* idx = reinterpret_cast<uint32_t*>(w + L.off_idx);
  uint8_t* code0 = w + L.off_code0;
  uint32_t* rank = reinterpret_cast<uint32_t*>(w + L.off_rank);
  double2* d = reinterpret_cast<double2*>(w + L.off_d);
  double2* sums = reinterpret_cast<double2*>(w + L.off_sums);
  double2* base = reinterpret_cast<double2*>(w + L.off_base);
  long long* diff = reinterpret_cast<long long*>(w + L.off_diff);
  long long* dsums = reinterpret_cast<long long*>(w + L.off_dsums);
  unsigned long long* cut0 = reinterpret_cast<unsigned long long*>(w + L.off_cut0);
  int64_t* state = reinterpret_cast<int64_t*>(w + L.off_state);
  int64_t* state2 = reinterpret_cast<int64_t*>(w + L.off_state2);
  R1Tables tb;
  Alphabet a = make_alphabet(K);
  for (int k = 0; k < kMaxK; ++k) {
    tb.zr[k] = k < K ? a.zr64[k] : 0.0;
    tb.zi[k] = k < K ? a.zi64[k] : 0.0;
  }
  r1_prep_kernel<<<static_cast<unsigned>(ceil_div(L.npad, 256)), 256, 0, st>>>(q, n, L.npad, K, key, idx, code0,
                                                                               status);
  count_launch();
  // bitonic sort of the (key, index) pairs
  const unsigned lblocks = static_cast<unsigned>(L.npad / kR1Local);
  r1_sort_local<<<lblocks, kR1Local / 2, 0, st>>>(key, idx, 2, kR1Local);
  count_launch();
  for (int64_t k = 2 * kR1Local; k <= L.npad; k <<= 1) {
    for (int64_t j = k >> 1; j >= kR1Local; j >>= 1) {
      r1_sort_global<<<static_cast<unsigned>(ceil_div(L.npad / 2, 256)), 256, 0, st>>>(key, idx, L.npad, k, j);
      count_launch();
    }
    r1_sort_local<<<lblocks, kR1Local / 2, 0, st>>>(key, idx, k, k);
    count_launch();
  }
  r1_delta_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(q, n, K, idx, code0, tb, d, rank);
  count_launch();
  const int nbase = static_cast<int>(std::min<int64_t>(kR1Threads, std::max<int64_t>(1, ceil_div(n, 4096))));
  r1_base_kernel<<<nbase, kR1Threads, 0, st>>>(q, n, code0, tb, base);
  count_launch();
  r1_scan<double2>(d, n, sums, L.nscan_blocks, st);
  r1_best_kernel<<<1, kR1Threads, 0, st>>>(d, n, base, nbase, state, f_out);
  r1_codes_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(code0, rank, n, K, state, z_out);
  count_launch(2);
  if (rowptr) {
    int e = cuda_check(cudaMemsetAsync(diff, 0, static_cast<size_t>(n + 2) * 8, st), "memset diff");
    if (e) return e;
    if ((e = cuda_check(cudaMemsetAsync(cut0, 0, 8, st), "memset cut0"))) return e;
    const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 152 * 8));
    r1_edge_kernel<<<blocks, 256, 0, st>>>(rowptr, colidx, n, nnz, K, code0, rank, diff, cut0);
    count_launch();
    r1_scan<long long>(diff, n + 1, dsums, L.nscan_blocks_diff, st);
    r1_best_cut_kernel<<<1, kR1Threads, 0, st>>>(diff, n, cut0, state2, cut_out);
    r1_codes_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(code0, rank, n, K, state2, zcut_out);
    count_launch(2);
  }
  return cuda_check(cudaGetLastError(), "rank-1 sweep kernels");
}

}  // namespace lrq
