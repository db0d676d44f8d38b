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

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kEnumMaxN = 512;
constexpr int kEnumMaxD = 4;      // r <= 4
constexpr int kEnumMaxRows = 2 * kEnumMaxD - 1;
constexpr int kEnumMaxBranch = 12;
constexpr unsigned long long kEnumMaxCombos = 1ull << 16;
constexpr int kEnumThreads = 128;
constexpr int kEnumRanksPerThread = 64;
constexpr double kEnumDefaultBudget = 1e12;

struct EnumTables {
  int K, BK;
  double rho_c[kMaxTcK], rho_s[kMaxTcK];  // cos, sin of theta_m (rho_m = cos - i sin)
  double bcos[kMaxTcK], bsin[kMaxTcK];    // all K boundaries for margins
  double zr[kMaxTcK], zi[kMaxTcK];        // omega^k
};

struct EnumBest {
  double f;
  int level;
  int sign;
  unsigned long long rank;
  unsigned long long choice;
};

__host__ __device__ __forceinline__ unsigned long long binom(int nn, int k) {
  if (k < 0 || k > nn) return 0ull;
  unsigned long long b = 1;
  for (int t = 1; t <= k; ++t) b = b * static_cast<unsigned long long>(nn - k + t) / static_cast<unsigned long long>(t);
  return b;
}

// combinatorial number system: rank = sum_k C(idx[k], k + 1) -> sorted
// combination idx[0] < ... < idx[m-1] of [0, N) (colexicographic order)
__host__ __device__ void unrank(unsigned long long rank, int N, int m, int* idx) {
  int hi = N;
  for (int pos = m; pos >= 1; --pos) {
    int c = hi - 1;
    while (c >= pos - 1 && binom(c, pos) > rank) --c;
    idx[pos - 1] = c;
    rank -= binom(c, pos);
    hi = c;
  }
}

// successor in the same (colexicographic) order as unrank
__host__ __device__ bool next_comb(int N, int m, int* idx) {
  for (int pos = 0; pos < m; ++pos) {
    const int lim = (pos + 1 < m) ? idx[pos + 1] : N;
    if (idx[pos] + 1 < lim) {
      ++idx[pos];
      for (int q = 0; q < pos; ++q) idx[q] = q;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ double vre(const double2* V, int r, int i, int j) { return V[i * r + j].x; }
__device__ __forceinline__ double vim(const double2* V, int r, int i, int j) { return V[i * r + j].y; }

// Decision code and code set of coordinate value (x, y) for the superset rule.
// Returns the number of options written to opt (1, 2 or K).
__device__ int code_options(double x, double y, double rownorm, bool dbl, const EnumTables& tb, int* opt) {
  const int K = tb.K;
  if (rownorm == 0.0) {  // a zero row of V: its code does not change f; fixed at 0
    opt[0] = 0;
    return 1;
  }
  if (dbl || hypot(x, y) <= 1e-9 * fmax(rownorm, 1e-300)) {
    for (int k = 0; k < K; ++k) opt[k] = k;
    return K;
  }
  const int k = decide_fp64(x, y, K, tb.bcos, tb.bsin);
  // angular distance to the two boundaries of sector k: |p| / |w| = sin(dist)
  const double aw = hypot(x, y);
  const int mlo = (k == 0) ? K - 1 : k - 1;
  const double plo = fabs(y * tb.bcos[mlo] - x * tb.bsin[mlo]) / aw;
  const double phi = fabs(y * tb.bcos[k] - x * tb.bsin[k]) / aw;
  if (plo <= 1e-9) {
    opt[0] = mlo;   // sector below boundary mlo is mlo, above is mlo + 1 = k
    opt[1] = k;
    return 2;
  }
  if (phi <= 1e-9) {
    opt[0] = k;
    opt[1] = (k + 1) % K;
    return 2;
  }
  opt[0] = k;
  return 1;
}

// Evaluate every candidate of one (level, index set, sign); keep the best.
// If `want` >= 0 the choice `want` is decoded into z instead.
__device__ void eval_vertex(const double2* V, int n, int r, int d, const int* I, int m, const double* ct, int sign,
                            const EnumTables& tb, const double* rown, EnumBest& best, unsigned long long rank,
                            long long want, uint8_t* z_out, double* f_out, int32_t* status) {
  const int BK = tb.BK;
  double cr[kEnumMaxD], ci[kEnumMaxD];
  for (int j = 0; j < d; ++j) {
    cr[j] = sign * ct[j];
    ci[j] = sign * ct[d + j];
  }
  // groups of I: doubles
  int grp[kEnumMaxRows];
  for (int t = 0; t < m; ++t) grp[t] = I[t] / BK;
  double sr[2 * kMaxRank], si[2 * kMaxRank];
  for (int j = 0; j < r; ++j) sr[j] = si[j] = 0.0;
  int bidx[kEnumMaxBranch], bopt[kEnumMaxBranch][kMaxTcK], bcnt[kEnumMaxBranch], nb = 0;
  bool overflow = false;
  for (int i = 0; i < n; ++i) {
    double x = 0.0, y = 0.0;
    for (int j = 0; j < d; ++j) {
      x += vre(V, r, i, j) * cr[j] - vim(V, r, i, j) * ci[j];
      y += vre(V, r, i, j) * ci[j] + vim(V, r, i, j) * cr[j];
    }
    int cnt_in = 0;
    for (int t = 0; t < m; ++t) cnt_in += (grp[t] == i);
    int opt[kMaxK];
    const int no = code_options(x, y, rown[i], cnt_in >= 2, tb, opt);
    const int k0 = opt[0];
    if (no > 1) {
      if (nb < kEnumMaxBranch && no <= kMaxTcK) {
        bidx[nb] = i;
        bcnt[nb] = no;
        for (int q = 0; q < no; ++q) bopt[nb][q] = opt[q];
        ++nb;
      } else {
        overflow = true;
      }
    }
    if (z_out && no == 1) z_out[i] = static_cast<uint8_t>(k0);
    // base sum with the first option
    for (int j = 0; j < r; ++j) {
      const double vr = vre(V, r, i, j), vi = vim(V, r, i, j);
      sr[j] += vr * tb.zr[k0] + vi * tb.zi[k0];
      si[j] += vr * tb.zi[k0] - vi * tb.zr[k0];
    }
  }
  unsigned long long total = 1;
  for (int b = 0; b < nb; ++b) total *= static_cast<unsigned long long>(bcnt[b]);
  if (overflow || total > kEnumMaxCombos) {
    // a vertex where more coordinates touch boundaries than the branch budget
    // allows (a degenerate, highly structured V): the result could not be
    // certified exact, so the call reports LRQ_EUNSUPPORTED
    dev_fail(status, LRQ_EUNSUPPORTED);
    return;
  }
  for (unsigned long long ch = 0; ch < total; ++ch) {
    if (want >= 0 && ch != static_cast<unsigned long long>(want)) continue;
    double tr[2 * kMaxRank], ti[2 * kMaxRank];
    for (int j = 0; j < r; ++j) {
      tr[j] = sr[j];
      ti[j] = si[j];
    }
    unsigned long long rem = ch;
    for (int b = 0; b < nb; ++b) {
      const int q = static_cast<int>(rem % bcnt[b]);
      rem /= bcnt[b];
      const int i = bidx[b];
      const int k0 = bopt[b][0], k1 = bopt[b][q];
      if (z_out) z_out[i] = static_cast<uint8_t>(k1);
      if (q == 0) continue;
      const double dzr = tb.zr[k1] - tb.zr[k0], dzi = tb.zi[k1] - tb.zi[k0];
      for (int j = 0; j < r; ++j) {
        const double vr = vre(V, r, i, j), vi = vim(V, r, i, j);
        tr[j] += vr * dzr + vi * dzi;
        ti[j] += vr * dzi - vi * dzr;
      }
    }
    double f = 0.0;
    for (int j = 0; j < r; ++j) f += tr[j] * tr[j] + ti[j] * ti[j];
    if (want >= 0) {
      if (f_out) *f_out = f;
      return;
    }
    if (f > best.f) {
      best.f = f;
      best.level = d;
      best.sign = sign;
      best.rank = rank;
      best.choice = ch;
    }
  }
}

__device__ void build_rows(const double2* V, int r, int d, const int* I, int m, const EnumTables& tb, double* H) {
  const int nc = 2 * d;
  for (int t = 0; t < m; ++t) {
    const int i = I[t] / tb.BK, mm = I[t] % tb.BK;
    const double c = tb.rho_c[mm], s = tb.rho_s[mm];
    for (int j = 0; j < d; ++j) {
      const double vr = vre(V, r, i, j), vi = vim(V, r, i, j);
      // rho V = (c - i s)(vr + i vi) = (c vr + s vi) + i (c vi - s vr)
      H[t * nc + j] = c * vi - s * vr;       // Im(rho V_ij)
      H[t * nc + d + j] = c * vr + s * vi;   // Re(rho V_ij)
    }
  }
}

__host__ __device__ bool valid_set(const int* I, int m, int BK) {
  for (int t = 0; t + 2 < m; ++t)
    if (I[t] / BK == I[t + 2] / BK) return false;  // three rows of one group (sorted)
  return true;
}

__global__ void __launch_bounds__(kEnumThreads) enum_kernel(const double2* __restrict__ V, int n, int r, int d,
                                                            unsigned long long total, const __grid_constant__ EnumTables tb,
                                                            const double* __restrict__ rown, EnumBest* __restrict__ block_best,
                                                            unsigned long long* __restrict__ counts, int32_t* status) {
  __shared__ EnumBest sb[kEnumThreads];
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
      build_rows(V, r, d, I, m, tb, H);
      double ct[2 * kEnumMaxD];
      if (!null_vector_fp64<kEnumMaxRows>(H, m, ct)) continue;
      ++nfull;
      eval_vertex(V, n, r, d, I, m, ct, +1, tb, rown, best, rk, -1, nullptr, nullptr, status);
      eval_vertex(V, n, r, d, I, m, ct, -1, tb, rown, best, rk, -1, nullptr, nullptr, status);
    }
  }
  sb[threadIdx.x] = best;
  atomicAdd(counts, nfull);
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      EnumBest o = sb[threadIdx.x + h];
      EnumBest& me = sb[threadIdx.x];
      // deterministic: larger f, then smaller (level desc., rank, sign, choice)
      bool take = o.f > me.f || (o.f == me.f && o.f >= 0.0 &&
                                 (o.level > me.level || (o.level == me.level && (o.rank < me.rank ||
                                 (o.rank == me.rank && (o.sign > me.sign || (o.sign == me.sign && o.choice < me.choice)))))));
      if (take) me = o;
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
  rown[i] = sqrt(s);
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
    EnumBest o = block_best[b];
    bool take = o.f > best.f || (o.f == best.f && o.f >= 0.0 &&
                                 (o.level > best.level || (o.level == best.level && (o.rank < best.rank ||
                                 (o.rank == best.rank && (o.sign > best.sign || (o.sign == best.sign && o.choice < best.choice)))))));
    if (take) best = o;
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
  build_rows(V, r, d, I, m, tb, H);
  double ct[2 * kEnumMaxD];
  null_vector_fp64<kEnumMaxRows>(H, m, ct);
  EnumBest dummy = best;
  double f = 0.0;
  eval_vertex(V, n, r, d, I, m, ct, best.sign, tb, rown, dummy, best.rank, static_cast<long long>(best.choice), z_out,
              &f, status);
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
  EnumTables tb;
  std::memset(&tb, 0, sizeof(tb));
  tb.K = K;
  tb.BK = (K % 2 == 0) ? K / 2 : K;
  Alphabet a = make_alphabet(K);
  for (int mm = 0; mm < tb.BK; ++mm) {
    tb.rho_c[mm] = a.bcos64[mm];
    tb.rho_s[mm] = a.bsin64[mm];
  }
  for (int k = 0; k < K; ++k) {
    tb.bcos[k] = a.bcos64[k];
    tb.bsin[k] = a.bsin64[k];
    tb.zr[k] = a.zr64[k];
    tb.zi[k] = a.zi64[k];
  }
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
