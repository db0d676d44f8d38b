// k_nullsample.cu -- the null-vector direction sampler (Sec. 5, "The analyzed
// sampler matches the one used in practice"): the randomised form of
// Algorithm 2.  A candidate direction is the null vector of 2r - 1 rows of
// the augmented real matrix (Eq. 6), drawn uniformly without replacement; a
// draw whose rows are linearly dependent has no unique null direction and is
// rejected, and the slot draws again.
//
// Rows are h_(i,m) = [Im(rho_m V_i), Re(rho_m V_i)], rho_m = exp(-i theta_m),
// theta_m = pi (2m + 1) / K, m < B_K, numbered R = i B_K + m.  The draws are
// Philox4x32-10: row j of attempt a of slot s, try t, uses the counter
// (lo32 s, hi32 s, (a << 8) | (j << 4) | t, 0x4E56) and key (lo32 seed,
// hi32 seed); the row is the high 64 bits of (w0 << 32 | w1) * N, N = n B_K,
// and a row already drawn in the attempt is drawn again (next t).  The null
// vector (FP64 elimination with full pivoting) is made unit-norm with its
// largest-magnitude component positive (first on ties), then negated when
// bit 0 of word w2 of the attempt's first draw is set (both signs of a vertex
// are candidates, Algorithm 2); c = c~[:r] + i c~[r:].
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kNsThreads = 128;
constexpr int kNsMaxRows = 2 * kMaxRank - 1;
constexpr int kNsAttempts = 64;
constexpr uint32_t kNsTag = 0x4E56u;

struct NsTables {
  int K, BK;
  double c[kMaxK], s[kMaxK];  // cos, sin of theta_m
};

__global__ void __launch_bounds__(kNsThreads) null_sample_kernel(const float2* __restrict__ V, int64_t n, int r,
                                                                 const __grid_constant__ NsTables tb, uint64_t seed,
                                                                 int64_t S, float2* __restrict__ C,
                                                                 unsigned long long* draws, int32_t* status) {
  const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned long long mine = 0;
  if (s < S) {
    const int m = 2 * r - 1, nc = 2 * r;
    const uint64_t N = static_cast<uint64_t>(n) * static_cast<uint64_t>(tb.BK);
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const uint32_t c0 = static_cast<uint32_t>(s), c1 = static_cast<uint32_t>(static_cast<uint64_t>(s) >> 32);
    bool done = false;
    for (int a = 0; a < kNsAttempts && !done; ++a) {
      ++mine;
      uint64_t rows[kNsMaxRows];
      bool neg = false, drawn = true;
      for (int j = 0; j < m && drawn; ++j) {
        drawn = false;
        for (int t = 0; t < 16 && !drawn; ++t) {
          const PhiloxOut o = philox4x32_10(c0, c1, (static_cast<uint32_t>(a) << 8) | (j << 4) | t, kNsTag, k0, k1);
          if (j == 0 && t == 0) neg = o.w[2] & 1u;
          const uint64_t x = (static_cast<uint64_t>(o.w[0]) << 32) | o.w[1];
          const uint64_t R = __umul64hi(x, N);
          bool dup = false;
          for (int q = 0; q < j; ++q) dup |= rows[q] == R;
          if (!dup) {
            rows[j] = R;
            drawn = true;
          }
        }
      }
      if (!drawn) continue;
      double H[kNsMaxRows * (kNsMaxRows + 1)];
      for (int t = 0; t < m; ++t) {
        const int64_t i = static_cast<int64_t>(rows[t] / tb.BK);
        const int mm = static_cast<int>(rows[t] % tb.BK);
        const double cs = tb.c[mm], sn = tb.s[mm];
        for (int k = 0; k < r; ++k) {
          const float2 v = V[i * r + k];
          const double vr = v.x, vi = v.y;
          // rho V = (cs - i sn)(vr + i vi) = (cs vr + sn vi) + i (cs vi - sn vr)
          H[t * nc + k] = cs * vi - sn * vr;
          H[t * nc + r + k] = cs * vr + sn * vi;
        }
      }
      double ct[2 * kMaxRank];
      if (!null_vector_fp64<kNsMaxRows>(H, m, ct)) continue;
      int jmax = 0;
      for (int k = 1; k < nc; ++k)
        if (fabs(ct[k]) > fabs(ct[jmax])) jmax = k;
      const double sg = ((ct[jmax] < 0.0) != neg) ? -1.0 : 1.0;
      for (int k = 0; k < r; ++k)
        C[s * r + k] = make_float2(static_cast<float>(sg * ct[k]), static_cast<float>(sg * ct[r + k]));
      done = true;
    }
    if (!done) {
      for (int k = 0; k < r; ++k) C[s * r + k] = make_float2(0.f, 0.f);
      dev_fail(status, LRQ_EUNSUPPORTED);
    }
  }
#pragma unroll
  for (int q = 16; q > 0; q >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, q);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(draws, mine);
}

int launch_null_sample(const float2* V, int64_t n, int r, int K, uint64_t seed, int64_t S, float2* C,
                       int64_t* draws_out, int32_t* status, cudaStream_t st) {
  const Alphabet a = make_alphabet(K);
  NsTables tb;
  tb.K = K;
  tb.BK = a.BK;
  for (int m = 0; m < kMaxK; ++m) {
    tb.c[m] = m < a.BK ? a.bcos64[m] : 0.0;
    tb.s[m] = m < a.BK ? a.bsin64[m] : 0.0;
  }
  int e = cuda_check(cudaMemsetAsync(draws_out, 0, sizeof(int64_t), st), "cudaMemsetAsync(draws_out)");
  if (e) return e;
  null_sample_kernel<<<static_cast<unsigned>(ceil_div(S, kNsThreads)), kNsThreads, 0, st>>>(
      V, n, r, tb, seed, S, C, reinterpret_cast<unsigned long long*>(draws_out), status);
  count_launch();
  return cuda_check(cudaGetLastError(), "null_sample_kernel");
}

}  // namespace lrq
