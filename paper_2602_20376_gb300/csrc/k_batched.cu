// k_batched.cu -- many independent instances of uneven n, r and K scored in
// one persistent launch (the sampling method of Sec. 4.2 applied per
// instance), with per-class tile shapes picked by the library's autotuner.
//
// Work decomposition: an item is (problem p, a tile of T consecutive
// candidates); it scores those T directions against all n_p coordinates, so
// items are independent and need no cross-item reduction.  A block of 256
// threads holds T candidates x (256 / T) row groups; the row groups split the
// coordinates of each shared-memory stage and are combined in FP64 at the end
// of the item.  Items are sorted by cost (n_p T) longest first and pulled by
// the persistent blocks from an atomic counter.
//
// Per problem the launch sequence is: input checks, direction sampling
// (Philox, when the caller passes no directions), the persistent scoring
// kernel (FP32 projections, sector decision by boundary signs, FP32 sums
// flushed to FP64 per stage), then one block per problem selects the top-m
// keys and re-scores them in FP64 (decision and sums in FP64), and keeps
// the best (ties to the smaller candidate index).
//
// Exact sub-batch: a problem given with S = 0 is solved exactly by vertex
// enumeration (Sec. 3, Algorithm 2) in the same persistent launch.  Its
// index sets, levels d = r..1 in turn, are cut into chunks of kBEnumChunk
// consecutive ranks; a chunk is one work item (FP64 null vectors and
// candidate scores, as in the standalone solver), whose best candidate goes
// to the problem's slot for that chunk, and the selection step reduces the
// chunks in the solver's deterministic order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "enum_device.cuh"
#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kBThreads = 256;
constexpr int kBRows = 128;       // V rows per shared-memory stage
constexpr int kBMaxS = 8192;      // candidates per problem
constexpr int kBMaxTopM = 16;
constexpr int kBTiles[3] = {64, 128, 256};
constexpr int kBEnumRanksPerThread = 16;
constexpr int kBEnumChunk = kBThreads * kBEnumRanksPerThread;  // index sets per exact work item
constexpr double kBEnumBudget = 1e10;                            // r n^(2r+1) of one exact problem

struct BProb {
  const float2* V;
  const float2* C;  // directions: the caller's, or the workspace slot when drawn
  int64_t n;
  int r, K, S, tile;
  int gen;          // 1: draw C from seed (+ epoch)
  int exact;        // 1: solved exactly by vertex enumeration (S = 0)
  uint64_t seed;
  int64_t key_off;  // offset of the problem's selection keys
  int64_t eb_off;   // exact: offset of its chunk results
  int nchunks;      // exact: work items
  int pad;
  unsigned long long lvl_total[kEnumMaxD];  // exact: index sets of level d at [d - 1]
};

struct BItem {
  int p;
  int s0;
};

struct BTable {
  float bcos[8], bsin[8];
  float zr[kMaxK], zi[kMaxK];
  double bcos64[8], bsin64[8];
  double zr64[kMaxK], zi64[kMaxK];
};

// decision tables for K = 0..64 (entries below 2 unused), filled once per device
static __device__ BTable g_btab[kMaxK + 1];
// the exact solver's tables for K = 2..8
static __device__ EnumTables g_etab[kMaxTcK + 1];

// ---------------------------------------------------------------------------
// direction sampling and input checks
// ---------------------------------------------------------------------------
__global__ void batched_sample_kernel(const BProb* __restrict__ probs, const int64_t* __restrict__ epoch) {
  const BProb pb = probs[blockIdx.y];
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (!pb.gen || s >= pb.S) return;
  const uint64_t seed = pb.seed + static_cast<uint64_t>(*epoch);
  double a[kMaxRank], b[kMaxRank], nrm2 = 0.0;
#pragma unroll
  for (int j = 0; j < kMaxRank; ++j) {
    if (j < pb.r) {
      sphere_component(seed, s, j, &a[j], &b[j]);
      nrm2 += a[j] * a[j] + b[j] * b[j];
    }
  }
  const double inv = 1.0 / sqrt(nrm2);
  float2* C = const_cast<float2*>(pb.C);
#pragma unroll
  for (int j = 0; j < kMaxRank; ++j)
    if (j < pb.r)
      C[static_cast<int64_t>(s) * pb.r + j] = make_float2(static_cast<float>(a[j] * inv), static_cast<float>(b[j] * inv));
}

__global__ void batched_check_kernel(const BProb* __restrict__ probs, int32_t* status) {
  const BProb pb = probs[blockIdx.y];
  const int64_t nv = 2 * pb.n * pb.r, nc = pb.gen ? 0 : 2 * static_cast<int64_t>(pb.S) * pb.r;
  const float* v = reinterpret_cast<const float*>(pb.V);
  const float* c = reinterpret_cast<const float*>(pb.C);
  bool bad = false;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < nv + nc;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    bad |= !isfinite(t < nv ? v[t] : c[t - nv]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) dev_fail(status, LRQ_EINVAL);
}

// ---------------------------------------------------------------------------
// persistent scoring kernel
// ---------------------------------------------------------------------------
struct BShared {
  float2 vs[kBRows * kMaxRank];
  float2 zt[kMaxK];
  double comb[kBThreads * 2 * kMaxRank];
  int next;
};

// Sector of w = x + i y: boundary signs for K <= 8 (KC = K), the angle for
// larger K (KC = 0).
template <int KC>
__device__ __forceinline__ int b_decide(float x, float y, const float* bc, const float* bs, int K) {
  if constexpr (KC > 0) {
    return decide_fp32<KC>(x, y, bc, bs);
  } else {
    if (K <= 8) {
      const int BK = (K % 2 == 0) ? K / 2 : K;
      uint32_t sb = 0;
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (m < BK) sb |= (fmaf(y, bc[m], -x * bs[m]) > 0.0f ? 1u : 0u) << m;
      if (K % 2 == 0) {
        const int c = __popc(sb);
        return (sb & 1u) ? c : (c == 0 ? 0 : K - c);
      }
      const uint32_t t = sb & ~(sb >> 1) & ((1u << (K - 1)) - 1u);
      return t ? __ffs(t) : 0;
    }
    return decide_fp32_generic(x, y, K);
  }
}

template <int R, int KC>
__device__ void b_score_item(const BProb& pb, int s0, BShared& sh, uint64_t* __restrict__ keys) {
  const int T = pb.tile, RS = kBThreads / T;
  const int tid = threadIdx.x, cl = tid % T, g = tid / T;
  const int s = s0 + cl;
  const bool act = s < pb.S;
  const BTable& tb = g_btab[pb.K];
  float cr[R], ci[R], bc[8], bs[8];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const float2 c = act ? pb.C[static_cast<int64_t>(s) * R + j] : make_float2(0.f, 0.f);
    cr[j] = c.x;
    ci[j] = c.y;
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    bc[m] = tb.bcos[m];
    bs[m] = tb.bsin[m];
  }
  for (int k = tid; k < pb.K; k += kBThreads) sh.zt[k] = make_float2(tb.zr[k], tb.zi[k]);
  double acc64[2 * R];
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) acc64[j] = 0.0;
  for (int64_t b0 = 0; b0 < pb.n; b0 += kBRows) {
    const int rows = static_cast<int>(min(static_cast<int64_t>(kBRows), pb.n - b0));
    __syncthreads();
    for (int t = tid; t < rows * R; t += kBThreads) sh.vs[t] = pb.V[b0 * R + t];
    __syncthreads();
    float acc[2 * R];
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) acc[j] = 0.f;
    for (int i = g; i < rows; i += RS) {
      float vr[R], vi[R], x = 0.f, y = 0.f;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float2 v = sh.vs[i * R + j];
        vr[j] = v.x;
        vi[j] = v.y;
        x = fmaf(vr[j], cr[j], fmaf(-vi[j], ci[j], x));
        y = fmaf(vr[j], ci[j], fmaf(vi[j], cr[j], y));
      }
      const float2 z = sh.zt[b_decide<KC>(x, y, bc, bs, pb.K)];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        acc[2 * j] = fmaf(vr[j], z.x, fmaf(vi[j], z.y, acc[2 * j]));
        acc[2 * j + 1] = fmaf(vr[j], z.y, fmaf(-vi[j], z.x, acc[2 * j + 1]));
      }
    }
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) acc64[j] += static_cast<double>(acc[j]);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) sh.comb[(g * T + cl) * (2 * R) + j] = acc64[j];
  __syncthreads();
  if (g == 0 && act) {
    double f = 0.0;
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) {
      double v = 0.0;
      for (int gg = 0; gg < RS; ++gg) v += sh.comb[(gg * T + cl) * (2 * R) + j];
      f += v * v;
    }
    const uint32_t fb = __float_as_uint(static_cast<float>(f));
    keys[pb.key_off + s] = (static_cast<uint64_t>(fb) << 32) | static_cast<uint64_t>(0xFFFFFFFFu - static_cast<uint32_t>(s));
  }
}

template <int R>
__device__ __forceinline__ void b_dispatch_k(const BProb& pb, int s0, BShared& sh, uint64_t* keys) {
  switch (pb.K) {
    case 2: b_score_item<R, 2>(pb, s0, sh, keys); break;
    case 3: b_score_item<R, 3>(pb, s0, sh, keys); break;
    case 4: b_score_item<R, 4>(pb, s0, sh, keys); break;
    case 8: b_score_item<R, 8>(pb, s0, sh, keys); break;
    default: b_score_item<R, 0>(pb, s0, sh, keys); break;
  }
}

// One exact work item: index sets [chunk kBEnumChunk, (chunk + 1) kBEnumChunk)
// of the problem's levels d = r..1 taken in turn, kBEnumRanksPerThread
// consecutive ranks per thread; the block's best candidate (the solver's
// order) goes to ebest[eb_off + chunk].  Kept out of line so that the
// scoring path keeps its registers.
__device__ __noinline__ void b_enum_item(const BProb& pb, int chunk, BShared& sh, EnumBest* __restrict__ ebest,
                                         int32_t* status) {
  const EnumTables& tb = g_etab[pb.K];
  const EnumV32 va{pb.V, pb.r};
  const int n = static_cast<int>(pb.n);
  const int N = n * tb.BK;
  unsigned long long total = 0;
  for (int d = 1; d <= pb.r; ++d) total += pb.lvl_total[d - 1];
  EnumBest best;
  best.f = -1.0;
  best.level = 0;
  best.sign = 1;
  best.rank = 0;
  best.choice = 0;
  unsigned long long q = static_cast<unsigned long long>(chunk) * kBEnumChunk +
                         static_cast<unsigned long long>(threadIdx.x) * kBEnumRanksPerThread;
  const unsigned long long qend = min(total, q + kBEnumRanksPerThread);
  while (q < qend) {
    int d = pb.r;
    unsigned long long base = 0;
    while (d >= 1 && q >= base + pb.lvl_total[d - 1]) {
      base += pb.lvl_total[d - 1];
      --d;
    }
    if (d < 1) break;
    const int m = 2 * d - 1;
    const unsigned long long l0 = q - base;
    const unsigned long long l1 = min(qend - base, pb.lvl_total[d - 1]);
    int I[kEnumMaxRows];
    unrank(l0, N, m, I);
    for (unsigned long long lr = l0; lr < l1; ++lr) {
      if (lr > l0) next_comb(N, m, I);
      if (!valid_set(I, m, tb.BK)) continue;
      double H[kEnumMaxRows * 2 * kEnumMaxD];
      build_rows(va, pb.r, d, I, m, tb, H);
      double ct[2 * kEnumMaxD];
      if (!null_vector_fp64<kEnumMaxRows>(H, m, ct)) continue;
      eval_vertex(va, n, pb.r, d, I, m, ct, +1, tb, best, lr, -1, nullptr, nullptr, status);
      eval_vertex(va, n, pb.r, d, I, m, ct, -1, tb, best, lr, -1, nullptr, nullptr, status);
    }
    q = base + l1;
  }
  EnumBest* sb = reinterpret_cast<EnumBest*>(sh.comb);
  __syncthreads();
  sb[threadIdx.x] = best;
  __syncthreads();
  for (int h = kBThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h && enum_better(sb[threadIdx.x + h], sb[threadIdx.x])) sb[threadIdx.x] = sb[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) ebest[pb.eb_off + chunk] = sb[0];
  __syncthreads();
}

__global__ void __launch_bounds__(kBThreads) batched_score_kernel(const BProb* __restrict__ probs,
                                                                  const BItem* __restrict__ items, int nitems,
                                                                  int* __restrict__ counter,
                                                                  uint64_t* __restrict__ keys,
                                                                  EnumBest* __restrict__ ebest,
                                                                  int32_t* status) {
  __shared__ BShared sh;
  for (;;) {
    if (threadIdx.x == 0) sh.next = atomicAdd(counter, 1);
    __syncthreads();
    const int it = sh.next;
    __syncthreads();
    if (it >= nitems) break;
    const BItem w = items[it];
    const BProb pb = probs[w.p];
    if (pb.exact) {
      b_enum_item(pb, w.s0, sh, ebest, status);
      continue;
    }
    switch (pb.r) {
      case 1: b_dispatch_k<1>(pb, w.s0, sh, keys); break;
      case 2: b_dispatch_k<2>(pb, w.s0, sh, keys); break;
      case 3: b_dispatch_k<3>(pb, w.s0, sh, keys); break;
      case 4: b_dispatch_k<4>(pb, w.s0, sh, keys); break;
      case 5: b_dispatch_k<5>(pb, w.s0, sh, keys); break;
      case 6: b_dispatch_k<6>(pb, w.s0, sh, keys); break;
      case 7: b_dispatch_k<7>(pb, w.s0, sh, keys); break;
      default: b_dispatch_k<8>(pb, w.s0, sh, keys); break;
    }
  }
}

// ---------------------------------------------------------------------------
// per problem: top-m keys, FP64 re-scoring, winner
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t b_block_max(uint64_t v, uint64_t* red) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    const uint64_t o = __shfl_xor_sync(0xffffffffu, v, m);
    v = o > v ? o : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  uint64_t b = red[0];
  for (int k = 1; k < kBThreads / 32; ++k) b = red[k] > b ? red[k] : b;
  return b;
}

template <int R>
__device__ double b_rescore(const BProb& pb, int s, double* red) {
  double cr[R], ci[R], acc[2 * R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const float2 c = pb.C[static_cast<int64_t>(s) * R + j];
    cr[j] = c.x;
    ci[j] = c.y;
    acc[2 * j] = acc[2 * j + 1] = 0.0;
  }
  const BTable& tb = g_btab[pb.K];
  for (int64_t i = threadIdx.x; i < pb.n; i += kBThreads) {
    double vr[R], vi[R], x = 0.0, y = 0.0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float2 v = pb.V[i * R + j];
      vr[j] = v.x;
      vi[j] = v.y;
      x = fma(vr[j], cr[j], fma(-vi[j], ci[j], x));
      y = fma(vr[j], ci[j], fma(vi[j], cr[j], y));
    }
    const int k = decide_fp64(x, y, pb.K, tb.bcos64, tb.bsin64);
    const double zr = tb.zr64[k], zi = tb.zi64[k];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      acc[2 * j] = fma(vr[j], zr, fma(vi[j], zi, acc[2 * j]));
      acc[2 * j + 1] = fma(vr[j], zi, fma(-vi[j], zr, acc[2 * j + 1]));
    }
  }
  double f = 0.0;
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) {
    double v = acc[j];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < kBThreads / 32; ++k) t += red[k];
    f += t * t;
  }
  return f;
}

// Exact problem: the best of its chunk results, in the solver's order.
__device__ void b_select_exact(const BProb& pb, const EnumBest* __restrict__ ebest, double* best_f, int64_t* best_idx,
                               int32_t* status) {
  __shared__ EnumBest sb[kBThreads];
  EnumBest best;
  best.f = -1.0;
  best.level = 0;
  best.sign = 1;
  best.rank = 0;
  best.choice = 0;
  for (int c = threadIdx.x; c < pb.nchunks; c += kBThreads)
    if (enum_better(ebest[pb.eb_off + c], best)) best = ebest[pb.eb_off + c];
  sb[threadIdx.x] = best;
  __syncthreads();
  for (int h = kBThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h && enum_better(sb[threadIdx.x + h], sb[threadIdx.x])) sb[threadIdx.x] = sb[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // no index set of full rank at any level (V's first column is zero)
    if (sb[0].f < 0.0) dev_fail(status, LRQ_EUNSUPPORTED);
    best_f[blockIdx.x] = sb[0].f;
    best_idx[blockIdx.x] = -1;
  }
}

__global__ void __launch_bounds__(kBThreads) batched_select_kernel(const BProb* __restrict__ probs,
                                                                   const uint64_t* __restrict__ keys, int top_m,
                                                                   const EnumBest* __restrict__ ebest,
                                                                   double* __restrict__ best_f,
                                                                   int64_t* __restrict__ best_idx,
                                                                   int64_t* __restrict__ epoch,
                                                                   int32_t* __restrict__ status) {
  __shared__ uint64_t redk[kBThreads / 32];
  __shared__ double redd[kBThreads / 32];
  const BProb pb = probs[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) *epoch += 1;  // the next call draws fresh directions
  if (pb.exact) {
    b_select_exact(pb, ebest, best_f, best_idx, status);
    return;
  }
  const uint64_t* kp = keys + pb.key_off;
  const int m = min(top_m, pb.S);
  double bf = -1.0;
  int bs = 0;
  uint64_t prev = ~0ull;
  for (int q = 0; q < m; ++q) {
    uint64_t v = 0;
    for (int s = threadIdx.x; s < pb.S; s += kBThreads) {
      const uint64_t k = kp[s];
      if (k < prev && k > v) v = k;
    }
    const uint64_t kmax = b_block_max(v, redk);
    prev = kmax;
    const int s = static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(kmax & 0xFFFFFFFFull));
    if (kmax == 0 || s < 0 || s >= pb.S) break;  // no key left (block-uniform)
    double f;
    switch (pb.r) {
      case 1: f = b_rescore<1>(pb, s, redd); break;
      case 2: f = b_rescore<2>(pb, s, redd); break;
      case 3: f = b_rescore<3>(pb, s, redd); break;
      case 4: f = b_rescore<4>(pb, s, redd); break;
      case 5: f = b_rescore<5>(pb, s, redd); break;
      case 6: f = b_rescore<6>(pb, s, redd); break;
      case 7: f = b_rescore<7>(pb, s, redd); break;
      default: f = b_rescore<8>(pb, s, redd); break;
    }
    if (f > bf || (f == bf && s < bs)) {
      bf = f;
      bs = s;
    }
  }
  if (threadIdx.x == 0) {
    if (bf < 0.0) dev_fail(status, LRQ_EINVAL);
    best_f[blockIdx.x] = bf;
    best_idx[blockIdx.x] = bs;
  }
}

// ---------------------------------------------------------------------------
// host side: plan, workspace, launch sequence, autotuner, graph
// ---------------------------------------------------------------------------
struct lrq_batched_plan_impl {
  std::vector<lrq_problem> probs;
  std::vector<int> tile;
  int top_m = 0;
  int device = 0;
  int grid = 0;
  int64_t nkeys = 0, ncgen = 0;
  size_t off_probs = 0, off_items = 0, off_counter = 0, off_epoch = 0, off_keys = 0, off_C = 0, off_ebest = 0,
         total = 0;
  int64_t nebest = 0;
  int nitems = 0;
  bool prepared = false;
  const void* prepared_ws = nullptr;
};

namespace {

std::mutex g_btab_mu;
bool g_btab_ready[64] = {};
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int, int>, int> g_tile_cache;  // (device, r, K, log2 n) -> tile

int n_bucket(int64_t n) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= n) ++b;
  return b;
}

int ensure_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_btab_mu);
  if (dev < 0 || dev >= 64) return fail(LRQ_EUNSUPPORTED, "device index above 63");
  if (g_btab_ready[dev]) return LRQ_OK;
  std::vector<BTable> t(kMaxK + 1);
  std::memset(t.data(), 0, t.size() * sizeof(BTable));
  for (int K = 2; K <= kMaxK; ++K) {
    Alphabet a = make_alphabet(K);
    for (int m = 0; m < 8; ++m) {
      t[K].bcos[m] = m < a.BK ? a.bcos[m] : 0.f;
      t[K].bsin[m] = m < a.BK ? a.bsin[m] : 0.f;
      t[K].bcos64[m] = m < a.BK ? a.bcos64[m] : 0.0;
      t[K].bsin64[m] = m < a.BK ? a.bsin64[m] : 0.0;
    }
    for (int k = 0; k < K; ++k) {
      t[K].zr[k] = a.zr[k];
      t[K].zi[k] = a.zi[k];
      t[K].zr64[k] = a.zr64[k];
      t[K].zi64[k] = a.zi64[k];
    }
  }
  int e = cuda_check(cudaMemcpyToSymbol(g_btab, t.data(), t.size() * sizeof(BTable)), "upload decision tables");
  if (e) return e;
  std::vector<EnumTables> et(kMaxTcK + 1);
  std::memset(et.data(), 0, et.size() * sizeof(EnumTables));
  for (int K = 2; K <= kMaxTcK; ++K) et[K] = make_enum_tables(K);
  if ((e = cuda_check(cudaMemcpyToSymbol(g_etab, et.data(), et.size() * sizeof(EnumTables)),
                      "upload enumeration tables")))
    return e;
  g_btab_ready[dev] = true;
  return LRQ_OK;
}

// Index sets of an exact problem's levels d = 1..r, and its work items.
void exact_levels(const lrq_problem& q, unsigned long long* lvl) {
  const int BK = (q.K % 2 == 0) ? q.K / 2 : q.K;
  for (int d = 1; d <= kEnumMaxD; ++d) lvl[d - 1] = d <= q.r ? binom(static_cast<int>(q.n) * BK, 2 * d - 1) : 0ull;
}

int64_t exact_chunks(const lrq_problem& q) {
  unsigned long long lvl[kEnumMaxD], total = 0;
  exact_levels(q, lvl);
  for (int d = 0; d < kEnumMaxD; ++d) total += lvl[d];
  return static_cast<int64_t>((total + kBEnumChunk - 1) / kBEnumChunk);
}

void layout(lrq_batched_plan_impl* pl) {
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    size_t o = cur;
    cur = align_up(cur + bytes, 256);
    return o;
  };
  const int P = static_cast<int>(pl->probs.size());
  int64_t nitems = 0;
  pl->nkeys = 0;
  pl->ncgen = 0;
  pl->nebest = 0;
  for (const lrq_problem& q : pl->probs) {
    if (q.S == 0) {  // exact
      const int64_t ch = exact_chunks(q);
      nitems += ch;
      pl->nebest += ch;
      continue;
    }
    nitems += ceil_div(q.S, kBTiles[0]);  // room for the smallest tile
    pl->nkeys += q.S;
    if (!q.C) pl->ncgen += q.S * q.r;
  }
  pl->off_probs = take(static_cast<size_t>(P) * sizeof(BProb));
  pl->off_items = take(static_cast<size_t>(nitems) * sizeof(BItem));
  pl->off_counter = take(sizeof(int));
  pl->off_epoch = take(sizeof(int64_t));
  pl->off_keys = take(static_cast<size_t>(pl->nkeys) * sizeof(uint64_t));
  pl->off_C = take(static_cast<size_t>(pl->ncgen) * sizeof(float2));
  pl->off_ebest = take(static_cast<size_t>(pl->nebest) * sizeof(EnumBest));
  pl->total = cur;
}

// Device descriptors and the item list for the problems in `subset` (all
// when empty), with the plan's current tiles.
int upload(lrq_batched_plan_impl* pl, uint8_t* ws, const std::vector<int>& subset, cudaStream_t st,
           int* nitems_out) {
  const int P = static_cast<int>(pl->probs.size());
  std::vector<BProb> hp(P);
  int64_t key_off = 0, c_off = 0, eb_off = 0;
  float2* Cgen = reinterpret_cast<float2*>(ws + pl->off_C);
  for (int p = 0; p < P; ++p) {
    const lrq_problem& q = pl->probs[p];
    BProb b;
    std::memset(&b, 0, sizeof(b));
    b.V = static_cast<const float2*>(q.V);
    if (q.S == 0) {
      b.exact = 1;
      b.n = q.n;
      b.r = q.r;
      b.K = q.K;
      exact_levels(q, b.lvl_total);
      b.nchunks = static_cast<int>(exact_chunks(q));
      b.eb_off = eb_off;
      eb_off += b.nchunks;
      hp[p] = b;
      continue;
    }
    b.gen = q.C ? 0 : 1;
    b.C = q.C ? static_cast<const float2*>(q.C) : Cgen + c_off;
    if (!q.C) c_off += q.S * q.r;
    b.n = q.n;
    b.r = q.r;
    b.K = q.K;
    b.S = static_cast<int>(q.S);
    b.tile = pl->tile[p];
    b.seed = q.seed;
    b.key_off = key_off;
    key_off += q.S;
    hp[p] = b;
  }
  std::vector<int> which = subset;
  if (which.empty())
    for (int p = 0; p < P; ++p) which.push_back(p);
  std::vector<BItem> items;
  for (int p : which) {
    if (hp[p].exact) {
      for (int c = 0; c < hp[p].nchunks; ++c) items.push_back(BItem{p, c});
      continue;
    }
    for (int s0 = 0; s0 < hp[p].S; s0 += hp[p].tile) items.push_back(BItem{p, s0});
  }
  // longest first: cost ~ n_p * tile * (r_p + 1) FP32 lane operations for a
  // scoring item; an exact item's kBEnumChunk index sets each cost two
  // vertices of about n_p (4 d + 24) FP64 operations, weighted 32x
  auto cost = [&](const BItem& it) {
    const BProb& b = hp[it.p];
    if (b.exact) return static_cast<double>(b.n) * kBEnumChunk * 2.0 * (4.0 * b.r + 24.0) * 32.0 / kBThreads;
    return static_cast<double>(b.n) * b.tile * (b.r + 1);
  };
  std::stable_sort(items.begin(), items.end(), [&](const BItem& a, const BItem& b) { return cost(a) > cost(b); });
  int e = cuda_check(cudaMemcpyAsync(ws + pl->off_probs, hp.data(), hp.size() * sizeof(BProb),
                                     cudaMemcpyHostToDevice, st),
                     "upload problems");
  if (e) return e;
  if (!items.empty() &&
      (e = cuda_check(cudaMemcpyAsync(ws + pl->off_items, items.data(), items.size() * sizeof(BItem),
                                      cudaMemcpyHostToDevice, st),
                      "upload items")))
    return e;
  if ((e = cuda_check(cudaStreamSynchronize(st), "upload sync"))) return e;  // host vectors end here
  *nitems_out = static_cast<int>(items.size());
  return LRQ_OK;
}

int launch_sequence(const lrq_batched_plan_impl* pl, uint8_t* ws, int nitems, bool sample, bool select,
                    double* best_f, int64_t* best_idx, int32_t* status, cudaStream_t st) {
  const int P = static_cast<int>(pl->probs.size());
  const BProb* probs = reinterpret_cast<const BProb*>(ws + pl->off_probs);
  int64_t* epoch = reinterpret_cast<int64_t*>(ws + pl->off_epoch);
  int* counter = reinterpret_cast<int*>(ws + pl->off_counter);
  uint64_t* keys = reinterpret_cast<uint64_t*>(ws + pl->off_keys);
  if (sample) {
    batched_check_kernel<<<dim3(64, P), 256, 0, st>>>(probs, status);
    batched_sample_kernel<<<dim3(kBMaxS / 256, P), 256, 0, st>>>(probs, epoch);
    count_launch(2);
  }
  int e = cuda_check(cudaMemsetAsync(counter, 0, sizeof(int), st), "reset item counter");
  if (e) return e;
  timing_start(st);
  EnumBest* ebest = reinterpret_cast<EnumBest*>(ws + pl->off_ebest);
  batched_score_kernel<<<pl->grid, kBThreads, 0, st>>>(probs, reinterpret_cast<const BItem*>(ws + pl->off_items),
                                                       nitems, counter, keys, ebest, status);
  timing_stop(st);
  count_launch();
  if (select) {
    batched_select_kernel<<<P, kBThreads, 0, st>>>(probs, keys, pl->top_m, ebest, best_f, best_idx, epoch, status);
    count_launch();
  }
  return cuda_check(cudaGetLastError(), "batched kernels");
}

std::mutex g_graph_mu;
std::map<void*, int> g_graph_launches;  // graph exec -> kernels per replay

}  // namespace

}  // namespace lrq

using namespace lrq;

struct lrq_batched_plan : lrq_batched_plan_impl {};

extern "C" {

int lrq_batched_plan_create(const lrq_problem* problems, int P, int top_m, lrq_batched_plan** plan_out) {
  if (!plan_out) return fail(LRQ_EINVAL, "plan_out is NULL");
  *plan_out = nullptr;
  if (!problems || P < 1) return fail(LRQ_EINVAL, "need at least one problem");
  if (P > 65535) return fail(LRQ_EUNSUPPORTED, "at most 65535 problems per plan");
  if (top_m < 1 || top_m > kBMaxTopM) return fail(LRQ_EINVAL, "top_m must be in [1, 16]");
  for (int p = 0; p < P; ++p) {
    const lrq_problem& q = problems[p];
    if (!q.V) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": V is NULL");
    if (q.n < 1 || q.n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": bad n");
    if (q.r < 1 || q.r > kMaxRank) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": r not in [1, 8]");
    if (q.K < 2 || q.K > kMaxK) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": K not in [2, 64]");
    if (q.S == 0) {  // exact sub-batch
      if (q.C) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": exact (S = 0) takes no directions");
      int e = enumerate_check(q.n, q.r, q.K, kBEnumBudget);
      if (e) return fail(e, "problem " + std::to_string(p) + " (exact): " + lrq_last_error());
      if (exact_chunks(q) > (int64_t(1) << 24))
        return fail(LRQ_EUNSUPPORTED, "problem " + std::to_string(p) + ": too many index sets");
      continue;
    }
    if (q.S < 1 || q.S > kBMaxS) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": S not in [0, 8192]");
    if (top_m > q.S) return fail(LRQ_EINVAL, "problem " + std::to_string(p) + ": top_m > S");
  }
  int dev = 0;
  int e = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (e) return e;
  lrq_batched_plan* pl = new lrq_batched_plan();
  pl->probs.assign(problems, problems + P);
  pl->top_m = top_m;
  pl->device = dev;
  pl->tile.resize(P);
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (int p = 0; p < P; ++p) {
      auto it = g_tile_cache.find(std::make_tuple(dev, pl->probs[p].r, pl->probs[p].K, n_bucket(pl->probs[p].n)));
      pl->tile[p] = it != g_tile_cache.end() ? it->second : 128;
    }
  }
  int blocks_per_sm = 1;
  if ((e = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, batched_score_kernel,
                                                                    kBThreads, 0),
                      "occupancy query"))) {
    delete pl;
    return e;
  }
  pl->grid = std::max(1, blocks_per_sm) * num_sms_current();
  layout(pl);
  *plan_out = pl;
  return LRQ_OK;
}

void lrq_batched_plan_destroy(lrq_batched_plan* plan) { delete plan; }

int lrq_batched_workspace_size(const lrq_batched_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return fail(LRQ_EINVAL, "NULL argument");
  *bytes = plan->total;
  return LRQ_OK;
}

int lrq_batched_prepare(lrq_batched_plan* plan, void* ws, size_t ws_bytes, void* stream) {
  if (!plan) return fail(LRQ_EINVAL, "plan is NULL");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < plan->total)
    return fail(LRQ_EWORKSPACE, "workspace missing, misaligned or smaller than lrq_batched_workspace_size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int e = ensure_tables(plan->device);
  if (e) return e;
  uint8_t* w = static_cast<uint8_t*>(ws);
  if ((e = cuda_check(cudaMemsetAsync(w + plan->off_epoch, 0, sizeof(int64_t), st), "reset epoch"))) return e;
  if ((e = upload(plan, w, {}, st, &plan->nitems))) return e;
  plan->prepared = true;
  plan->prepared_ws = ws;
  return LRQ_OK;
}

int lrq_sample_score_batched(const lrq_batched_plan* plan, void* ws, size_t ws_bytes, double* best_f_out,
                             int64_t* best_idx_out, int32_t* dev_status, void* stream) {
  if (!plan || !best_f_out || !best_idx_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  if (!plan->prepared || plan->prepared_ws != ws || ws_bytes < plan->total)
    return fail(LRQ_EINVAL, "call lrq_batched_prepare with this workspace first");
  return launch_sequence(plan, static_cast<uint8_t*>(ws), plan->nitems, true, true, best_f_out, best_idx_out,
                         dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_batched_autotune(lrq_batched_plan* plan, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream) {
  if (!plan || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  if (!plan->prepared || plan->prepared_ws != ws || ws_bytes < plan->total)
    return fail(LRQ_EINVAL, "call lrq_batched_prepare with this workspace first");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const int P = static_cast<int>(plan->probs.size());
  // directions once (the timed runs score them again and again)
  int e = launch_sequence(plan, w, 0, true, false, nullptr, nullptr, dev_status, st);
  if (e) return e;
  if ((e = cuda_check(cudaMemsetAsync(w + plan->off_epoch, 0, sizeof(int64_t), st), "reset epoch"))) return e;
  std::map<std::tuple<int, int, int>, std::vector<int>> classes;
  for (int p = 0; p < P; ++p)
    if (plan->probs[p].S > 0)
      classes[std::make_tuple(plan->probs[p].r, plan->probs[p].K, n_bucket(plan->probs[p].n))].push_back(p);
  cudaEvent_t t0, t1;
  if ((e = cuda_check(cudaEventCreate(&t0), "event"))) return e;
  if ((e = cuda_check(cudaEventCreate(&t1), "event"))) {
    cudaEventDestroy(t0);
    return e;
  }
  for (auto& kv : classes) {
    float best_ms = 0.f;
    int best_tile = 128;
    for (int ti = 0; ti < 3; ++ti) {
      for (int p : kv.second) plan->tile[p] = kBTiles[ti];
      int nit = 0;
      if ((e = upload(plan, w, kv.second, st, &nit))) break;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && !e; ++rep) {
        cudaEventRecord(t0, st);
        e = launch_sequence(plan, w, nit, false, false, nullptr, nullptr, dev_status, st);
        cudaEventRecord(t1, st);
        if (!e) e = cuda_check(cudaEventSynchronize(t1), "autotune sync");
        float x = 0.f;
        cudaEventElapsedTime(&x, t0, t1);
        ms = rep == 0 ? x : std::min(ms, x);
      }
      if (e) break;
      if (ti == 0 || ms < best_ms) {
        best_ms = ms;
        best_tile = kBTiles[ti];
      }
    }
    if (e) break;
    for (int p : kv.second) plan->tile[p] = best_tile;
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_cache[std::make_tuple(plan->device, std::get<0>(kv.first), std::get<1>(kv.first),
                                 std::get<2>(kv.first))] = best_tile;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (e) return e;
  return upload(plan, w, {}, st, &plan->nitems);
}

int lrq_batched_tile(const lrq_batched_plan* plan, int p) {
  if (!plan || p < 0 || p >= static_cast<int>(plan->probs.size())) return -1;
  if (plan->probs[p].S == 0) return 0;  // exact: no candidate tile
  return plan->tile[p];
}

int lrq_batched_graph_create(const lrq_batched_plan* plan, void* ws, size_t ws_bytes, double* best_f_out,
                             int64_t* best_idx_out, int32_t* dev_status, void* stream, void** graph_exec_out) {
  if (!graph_exec_out) return fail(LRQ_EINVAL, "graph_exec_out is NULL");
  *graph_exec_out = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) return fail(LRQ_EINVAL, "graph capture needs a non-default stream");
  int e = cuda_check(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (e) return e;
  const uint64_t before = lrq_kernel_launches();
  int e2 = lrq_sample_score_batched(plan, ws, ws_bytes, best_f_out, best_idx_out, dev_status, stream);
  const int nk = static_cast<int>(lrq_kernel_launches() - before);
  cudaGraph_t g = nullptr;
  e = cuda_check(cudaStreamEndCapture(st, &g), "end capture");
  if (e2 || e) {
    if (g) cudaGraphDestroy(g);
    return e2 ? e2 : e;
  }
  cudaGraphExec_t ex = nullptr;
  e = cuda_check(cudaGraphInstantiate(&ex, g, 0), "instantiate graph");
  cudaGraphDestroy(g);
  if (e) return e;
  // the capture counted its kernels; count them again on every replay instead
  count_launch(-nk);
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graph_launches[ex] = nk;
  }
  *graph_exec_out = ex;
  return LRQ_OK;
}

int lrq_graph_launch(void* graph_exec, void* stream) {
  if (!graph_exec) return fail(LRQ_EINVAL, "graph_exec is NULL");
  int nk = 0;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graph_launches.find(graph_exec);
    if (it == g_graph_launches.end()) return fail(LRQ_EINVAL, "unknown graph");
    nk = it->second;
  }
  int e = cuda_check(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream)),
                     "cudaGraphLaunch");
  if (!e) count_launch(nk);
  return e;
}

int lrq_graph_destroy(void* graph_exec) {
  if (!graph_exec) return LRQ_OK;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graph_launches.erase(graph_exec);
  }
  return cuda_check(cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec)), "cudaGraphExecDestroy");
}

}  // extern "C"
