// k_enum.cu -- exact rank-r solver by vertex enumeration of the hyperplane
// arrangement (Sec. 3, Algorithm 2; Theorem 3.2).
//
// Level d = r, r-1, ..., 1 uses the leading columns V[:, :d] (the recursion of
// Algorithm 2).  The augmented real matrix (Eq. 6) has rows
//   h_(i,m) = [Im(rho_m V_i), Re(rho_m V_i)],  rho_m = exp(-i pi (2m+1)/K),
// m < B_K, so that h . [Re c; Im c] = Im(rho_m V_i c) vanishes exactly when
// V_i c lies on decision boundary m.  For every index set I of 2d-1 rows with
// at most two rows from any coordinate group:
//   1. the null vector c~ of H_I (FP64 Gaussian elimination with full
//      pivoting; I is skipped unless H_I has rank 2d-1);
//   2. for both signs, c = +-(c~[:d] + i c~[d:]) and w = V_d c;
//   3. every coordinate gets the codes of the cells that touch the vertex: all
//      K codes where w_i = 0 (two rows of its group in I), both codes next to
//      the boundary where arg w_i is within 1e-9 of one, else the decision-rule
//      code (Eq. 9);
//   4. every combination is scored on the full V (||V^H z||^2), incrementally
//      from the all-decided base sum.
// Step 3 is a superset of the candidates of the paper's ambiguity resolution
// (Algorithm 4): every cell of the arrangement has a vertex in its closure.
// Each thread walks a contiguous range of combination ranks; the best
// (f, level, rank, sign, choice) is reduced per block, then one thread
// rebuilds the winning assignment.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "enum_device.cuh"
#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kEnumMaxN = 512;
constexpr int kEnumThreads = 128;
constexpr int kEnumRanksPerThread = 64;
constexpr double kEnumDefaultBudget = 1e12;

__global__ void __launch_bounds__(kEnumThreads) enum_kernel(const double2* __restrict__ V, int n, int r, int d,
                                                            unsigned long long total, const __grid_constant__ EnumTables tb,
                                                            const double* __restrict__ rown, EnumBest* __restrict__ block_best,
                                                            unsigned long long* __restrict__ counts, int32_t* status) {
  __shared__ EnumBest sb[kEnumThreads];
  const EnumV64 va{V, r, rown};
  const int m = 2 * d - 1;
  const int N = n * tb.BK;
  EnumBest best;
  best.f = -1.0;
  best.level = 0;
  best.sign = 1;
  best.rank = 0;
  best.choice = 0;
  unsigned long long nfull = 0;
  const unsigned long long per = kEnumRanksPerThread;
  const unsigned long long tid = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x * per;
  for (unsigned long long r0 = tid * per; r0 < total; r0 += stride) {
    int I[kEnumMaxRows];
    unrank(r0, N, m, I);
    const unsigned long long r1 = min(total, r0 + per);
    for (unsigned long long rk = r0; rk < r1; ++rk) {
      if (rk > r0) next_comb(N, m, I);
      if (!valid_set(I, m, tb.BK)) continue;
      double H[kEnumMaxRows * 2 * kEnumMaxD];
      build_rows(va, r, d, I, m, tb, H);
      double ct[2 * kEnumMaxD];
      if (!null_vector_fp64<kEnumMaxRows>(H, m, ct)) continue;
      ++nfull;
      eval_vertex(va, n, r, d, I, m, ct, +1, tb, best, rk, -1, nullptr, nullptr, status);
      eval_vertex(va, n, r, d, I, m, ct, -1, tb, best, rk, -1, nullptr, nullptr, status);
    }
  }
  sb[threadIdx.x] = best;
  atomicAdd(counts, nfull);
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const EnumBest o = sb[threadIdx.x + h];
      if (enum_better(o, sb[threadIdx.x])) sb[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) block_best[blockIdx.x] = sb[0];
}

__global__ void enum_rownorm_kernel(const double2* __restrict__ V, int n, int r, double* __restrict__ rown,
                                    int32_t* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  bool finite = true;
  for (int j = 0; j < r; ++j) {
    double2 v = V[i * r + j];
    finite &= isfinite(v.x) && isfinite(v.y);
    s += v.x * v.x + v.y * v.y;
  }
  rown[i] = s;  // squared row norm
  if (!finite) dev_fail(status, LRQ_EINVAL);
}

// one thread: pick the best over all blocks of all levels, rebuild z
__global__ void enum_final_kernel(const double2* __restrict__ V, int n, int r, const __grid_constant__ EnumTables tb,
                                  const double* __restrict__ rown, const EnumBest* __restrict__ block_best, int nbest,
                                  const unsigned long long* __restrict__ counts, uint8_t* __restrict__ z_out,
                                  double* __restrict__ f_out, int64_t* __restrict__ n_sets_out, int32_t* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  EnumBest best = block_best[0];
  for (int b = 1; b < nbest; ++b) {
    const EnumBest o = block_best[b];
    if (enum_better(o, best)) best = o;
  }
  if (n_sets_out) *n_sets_out = static_cast<int64_t>(*counts);
  if (best.f < 0.0) {
    for (int i = 0; i < n; ++i) z_out[i] = 0;
    if (f_out) *f_out = -1.0;
    return;
  }
  const int d = best.level, m = 2 * d - 1;
  int I[kEnumMaxRows];
  unrank(best.rank, n * tb.BK, m, I);
  double H[kEnumMaxRows * 2 * kEnumMaxD];
  const EnumV64 va{V, r, rown};
  build_rows(va, r, d, I, m, tb, H);
  double ct[2 * kEnumMaxD];
  null_vector_fp64<kEnumMaxRows>(H, m, ct);
  EnumBest dummy = best;
  double f = 0.0;
  eval_vertex(va, n, r, d, I, m, ct, best.sign, tb, dummy, best.rank, static_cast<long long>(best.choice), z_out, &f,
              status);
  if (f_out) *f_out = f;
}

size_t enum_workspace_bytes(int64_t n, int r) {
  // row norms, counts, per-block bests of every level
  (void)r;
  return align_up(static_cast<size_t>(n) * sizeof(double), 256) + 256 +
         static_cast<size_t>(kEnumMaxD) * 4096 * sizeof(EnumBest);
}

static unsigned long long host_binom(int nn, int k) {
  if (k < 0 || k > nn) return 0;
  long double b = 1;
  for (int t = 1; t <= k; ++t) b = b * (nn - k + t) / t;
  return b > 4.0e18L ? ~0ull : static_cast<unsigned long long>(b + 0.5L);
}

int enumerate_check(int64_t n, int r, int K, double budget) {
  if (n < 1) return fail(LRQ_EINVAL, "n must be >= 1");
  if (r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "r must be in [1, 8]");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (n > kEnumMaxN) return fail(LRQ_EUNSUPPORTED, "lrq_enumerate supports n <= 512");
  if (r > kEnumMaxD) return fail(LRQ_EUNSUPPORTED, "lrq_enumerate supports r <= 4");
  if (K > kMaxTcK) return fail(LRQ_EUNSUPPORTED, "lrq_enumerate supports K <= 8");
  const double work = static_cast<double>(r) * std::pow(static_cast<double>(n), 2.0 * r + 1.0);
  if (work > (budget > 0.0 ? budget : kEnumDefaultBudget))
    return fail(LRQ_EUNSUPPORTED, "r * n^(2r+1) exceeds the enumeration budget");
  const int BK = (K % 2 == 0) ? K / 2 : K;
  const int N = static_cast<int>(n) * BK;
  for (int d = r; d >= 1; --d) {
    const unsigned long long t = host_binom(N, 2 * d - 1);
    // the device's incremental binomials multiply by at most N before dividing
    if (t == ~0ull || t > (1ull << 62) / static_cast<unsigned long long>(N))
      return fail(LRQ_EUNSUPPORTED, "too many index sets");
  }
  return LRQ_OK;
}

int launch_enumerate(const double2* V, int64_t n, int r, int K, uint8_t* z_out, double* f_out, int64_t* n_sets_out,
                     void* ws, int32_t* status, cudaStream_t st) {
  const EnumTables tb = make_enum_tables(K);
  uint8_t* w = static_cast<uint8_t*>(ws);
  double* rown = reinterpret_cast<double*>(w);
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(w + align_up(n * sizeof(double), 256));
  EnumBest* bests = reinterpret_cast<EnumBest*>(w + align_up(n * sizeof(double), 256) + 256);
  int e = cuda_check(cudaMemsetAsync(counts, 0, sizeof(unsigned long long), st), "cudaMemsetAsync(counts)");
  if (e) return e;
  enum_rownorm_kernel<<<static_cast<unsigned>(ceil_div(n, 128)), 128, 0, st>>>(V, static_cast<int>(n), r, rown,
                                                                               status);
  count_launch();
  int nbest = 0;
  for (int d = r; d >= 1; --d) {
    const int m = 2 * d - 1;
    const unsigned long long total = host_binom(static_cast<int>(n) * tb.BK, m);
    if (total == 0) continue;  // enumerate_check bounded every level's count
    const unsigned long long threads = (total + kEnumRanksPerThread - 1) / kEnumRanksPerThread;
    int blocks = static_cast<int>(std::min<unsigned long long>((threads + kEnumThreads - 1) / kEnumThreads, 4096));
    enum_kernel<<<blocks, kEnumThreads, 0, st>>>(V, static_cast<int>(n), r, d, total, tb, rown, bests + nbest,
                                                 counts, status);
    count_launch();
    nbest += blocks;
  }
  if ((e = cuda_check(cudaGetLastError(), "enum_kernel"))) return e;
  enum_final_kernel<<<1, 32, 0, st>>>(V, static_cast<int>(n), r, tb, rown, bests, nbest, counts, z_out, f_out,
                                      n_sets_out, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "enum_final_kernel");
}

}  // namespace lrq
