// k_rescore.cu -- FP64-accurate re-scoring of selected candidates.
//
// For a selected direction c, recomputes w_i = V_i c, the decision rule of
// Sec. 3, Eq. 9 and f = ||V^H z||^2 (Sec. 4.2, Eq. 10) from the complex64 V
// and C taken exactly, so that the result equals the FP64 evaluation of the
// same candidate up to FP64 rounding.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the per-coordinate work
// avoids FP64 arithmetic while keeping FP64 accuracy:
//  * w is computed in FP32 together with a rigorous bound on its rounding
//    error; the FP32 decision is accepted only when both boundary lines of
//    the chosen sector are farther than that bound, which makes it equal to
//    the FP64 decision.  Otherwise w and the decision are recomputed in FP64
//    (rare: the angle must be within ~1e-6 of a boundary).
//  * conj(V_i) omega^k is accumulated in double-float form: exact products
//    (FMA residuals) and exact sums (two-sum) in FP32 registers; the per-thread
//    (hi, lo) pairs are combined in FP64 by a fixed tree.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kRsThreads = 256;

struct RescoreTables {
  int K;
  float bcos[kMaxK], bsin[kMaxK];     // all K boundary lines, theta_m = pi(2m+1)/K
  double bcos64[kMaxK], bsin64[kMaxK];
  float zrh[kMaxK], zrl[kMaxK], zih[kMaxK], zil[kMaxK];  // omega^k as double-float
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc (hi, lo) += a*bh + a*bl + c*dh + c*dl with exact leading products
__device__ __forceinline__ void acc_dot2(float& hi, float& lo, float a, float bh, float bl, float c, float dh,
                                         float dl) {
  float p1 = a * bh;
  float e1 = fmaf(a, bh, -p1);
  float p2 = c * dh;
  float e2 = fmaf(c, dh, -p2);
  float s, e3;
  two_sum(p1, p2, s, e3);
  float small = fmaf(a, bl, fmaf(c, dl, (e1 + e2) + e3));
  float h2, e4;
  two_sum(hi, s, h2, e4);
  hi = h2;
  lo += e4 + small;
}

// Work split: a block takes kRsCpb candidates and one chunk of coordinates;
// the chunk's rows of V are staged through shared memory 256 at a time
// (component-major, so that the 32 lanes of a warp read 32 consecutive
// entries) and every warp evaluates its kRsCpw candidates on them, one row
// per lane.  V is thus read from memory once per kRsCpb candidates instead of
// once per candidate.  RM is the largest rank the instance handles (4 or 8):
// it sizes the per-thread accumulators.
constexpr int kRsCpw = 2;                              // candidates per warp
constexpr int kRsCpb = kRsCpw * (kRsThreads / 32);     // candidates per block
constexpr int kRsTile = 256;                           // rows staged at a time
constexpr int kRsFlush = 256 * 32 / kRsTile;           // tiles between FP64 flushes (256 rows per lane)
static_assert(kRsCpw * 16 == 32 && 2 * kMaxRank <= 16, "one lane per (candidate, component) total");

template <int K, int RM>
__global__ void __launch_bounds__(kRsThreads) rescore_partial_kernel(
    const float2* __restrict__ V, int64_t n, int r, const float2* __restrict__ C, int64_t S,
    const int64_t* __restrict__ idx, int m, int nchunk, int64_t rows_per_chunk, const __grid_constant__ RescoreTables tab,
    double* __restrict__ part, uint8_t* __restrict__ z_out, int32_t* status) {
  __shared__ float2 vs[RM][kRsTile];
  __shared__ float2 cs[kRsCpb][RM];
  __shared__ float sbc[kMaxK], sbs[kMaxK], szrh[kMaxK], szrl[kMaxK], szih[kMaxK], szil[kMaxK];
  __shared__ double sbc64[kMaxK], sbs64[kMaxK];
  const int Kr = (K > 0) ? K : tab.K;
  for (int k = threadIdx.x; k < Kr; k += blockDim.x) {
    sbc[k] = tab.bcos[k];
    sbs[k] = tab.bsin[k];
    sbc64[k] = tab.bcos64[k];
    sbs64[k] = tab.bsin64[k];
    szrh[k] = tab.zrh[k];
    szrl[k] = tab.zrl[k];
    szih[k] = tab.zih[k];
    szil[k] = tab.zil[k];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = blockIdx.y;
  const int tb = blockIdx.x * kRsCpb;  // first candidate position of the block
  for (int e = threadIdx.x; e < kRsCpb * RM; e += blockDim.x) {
    const int c = e / RM, j = e % RM;
    const int t = tb + c;
    float2 v = make_float2(0.f, 0.f);
    if (t < m && j < r) {
      const int64_t s = idx[t];
      if (s >= 0 && s < S) v = C[s * r + j];
    }
    cs[c][j] = v;
  }
  __syncthreads();

  // this warp's candidates
  int tc[kRsCpw];
  bool act[kRsCpw], ok[kRsCpw];
#pragma unroll
  for (int q = 0; q < kRsCpw; ++q) {
    tc[q] = tb + warp * kRsCpw + q;
    act[q] = tc[q] < m;
    const int64_t s = act[q] ? idx[tc[q]] : 0;
    ok[q] = act[q] && s >= 0 && s < S;
    if (act[q] && !ok[q] && lane == 0 && chunk == 0) dev_fail(status, LRQ_EINVAL);
  }
  float cr[kRsCpw][RM], ci[kRsCpw][RM];
#pragma unroll
  for (int q = 0; q < kRsCpw; ++q)
#pragma unroll
    for (int j = 0; j < RM; ++j) {
      const float2 c = cs[warp * kRsCpw + q][j];
      cr[q][j] = c.x;
      ci[q][j] = c.y;
    }
  const float u = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of FP32
  const float gamma = static_cast<float>(2 * r + 4) * 2.0f * u;
  float hi[kRsCpw][2 * RM], lo[kRsCpw][2 * RM];
#pragma unroll
  for (int q = 0; q < kRsCpw; ++q)
#pragma unroll
    for (int j = 0; j < 2 * RM; ++j) hi[q][j] = lo[q][j] = 0.f;
  // Every kRsFlush tiles (at most 256 rows per lane, which bounds the error
  // of the FP32 low parts) the lanes' (hi, lo) pairs are added in FP64 over
  // the warp (xor tree) and the total of component j of candidate q is kept
  // by lane q * 16 + j.
  double tot = 0.0;
  auto flush = [&]() {
#pragma unroll
    for (int q = 0; q < kRsCpw; ++q) {
#pragma unroll
      for (int j = 0; j < 2 * RM; ++j) {
        if (j < 2 * r) {
          double v = static_cast<double>(hi[q][j]) + static_cast<double>(lo[q][j]);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane == q * 16 + j) tot += v;
          hi[q][j] = lo[q][j] = 0.f;
        }
      }
    }
  };
  int tiles = 0;

  const int64_t i0 = static_cast<int64_t>(chunk) * rows_per_chunk;
  const int64_t i1 = min(n, i0 + rows_per_chunk);
  for (int64_t ts = i0; ts < i1; ts += kRsTile) {
    if (tiles == kRsFlush) {
      flush();
      tiles = 0;
    }
    ++tiles;
    const int rows = static_cast<int>(min(static_cast<int64_t>(kRsTile), i1 - ts));
    __syncthreads();  // the previous tile has been read
    for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
      const int row = e / r, j = e - row * r;
      vs[j][row] = V[ts * r + e];
    }
    __syncthreads();
    for (int ro = lane; ro < rows; ro += 32) {
      const int64_t i = ts + ro;
      float vr[RM], vi[RM];
#pragma unroll
      for (int j = 0; j < RM; ++j) {
        const float2 v = (j < r) ? vs[j][ro] : make_float2(0.f, 0.f);
        vr[j] = v.x;
        vi[j] = v.y;
      }
#pragma unroll
      for (int q = 0; q < kRsCpw; ++q) {
        if (!act[q]) continue;
        float x = 0.f, y = 0.f, mag = 0.f;
#pragma unroll
        for (int j = 0; j < RM; ++j) {
          x = fmaf(vr[j], cr[q][j], x);
          x = fmaf(-vi[j], ci[q][j], x);
          y = fmaf(vr[j], ci[q][j], y);
          y = fmaf(vi[j], cr[q][j], y);
          mag = fmaf(fabsf(vr[j]) + fabsf(vi[j]), fabsf(cr[q][j]) + fabsf(ci[q][j]), mag);
        }
        int k;
        if constexpr (K > 0) {
          constexpr int BK = (K % 2 == 0) ? K / 2 : K;
          float bc[BK], bs[BK];
#pragma unroll
          for (int mm = 0; mm < BK; ++mm) {
            bc[mm] = sbc[mm];
            bs[mm] = sbs[mm];
          }
          k = decide_fp32<K>(x, y, bc, bs);
        } else {
          k = decide_fp32_generic(x, y, Kr);
        }
        // certify: w strictly inside sector k, away from both bounding lines
        // by more than the rounding bound (boundary k-1 below, k above)
        const float bound = gamma * mag + 4.0f * u * (fabsf(x) + fabsf(y));
        const int ma = (k == 0) ? Kr - 1 : k - 1;
        const float pa = fmaf(y, sbc[ma], -x * sbs[ma]);
        const float pb = fmaf(y, sbc[k], -x * sbs[k]);
        if (!(pa > bound && pb < -bound)) {
          double xd = 0.0, yd = 0.0;
#pragma unroll
          for (int j = 0; j < RM; ++j) {
            xd = fma(static_cast<double>(vr[j]), static_cast<double>(cr[q][j]), xd);
            xd = fma(-static_cast<double>(vi[j]), static_cast<double>(ci[q][j]), xd);
            yd = fma(static_cast<double>(vr[j]), static_cast<double>(ci[q][j]), yd);
            yd = fma(static_cast<double>(vi[j]), static_cast<double>(cr[q][j]), yd);
          }
          k = decide_fp64(xd, yd, Kr, sbc64, sbs64);
        }
        if (z_out && ok[q]) z_out[static_cast<int64_t>(tc[q]) * n + i] = static_cast<uint8_t>(k);
        const float zrh = szrh[k], zrl = szrl[k], zih = szih[k], zil = szil[k];
#pragma unroll
        for (int j = 0; j < RM; ++j) {
          if (j < r) {
            // Re(conj(V) z) = vr zr + vi zi ; Im(conj(V) z) = vr zi - vi zr
            acc_dot2(hi[q][2 * j], lo[q][2 * j], vr[j], zrh, zrl, vi[j], zih, zil);
            acc_dot2(hi[q][2 * j + 1], lo[q][2 * j + 1], vr[j], zih, zil, -vi[j], zrh, zrl);
          }
        }
      }
    }
  }
  flush();
  {
    const int q = lane >> 4, j = lane & 15;
    if (j < 2 * r && act[q]) part[(static_cast<int64_t>(tc[q]) * nchunk + chunk) * (2 * kMaxRank) + j] = tot;
  }
}

__global__ void rescore_final_kernel(const double* __restrict__ part, int m, int nchunk, int r,
                                     const int64_t* __restrict__ idx, int64_t S, double* __restrict__ f_out,
                                     int64_t* __restrict__ best_out, double* __restrict__ best_f_out) {
  __shared__ double bf[256];
  __shared__ int bt[256];
  double my_best = -1.0;
  int my_t = 0x7fffffff;
  // one warp per candidate: lanes sum fixed subsets of the chunks, then a
  // fixed shuffle tree adds the lanes (deterministic order)
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int t = threadIdx.x >> 5; t < m; t += nwarp) {
    double a[2 * kMaxRank];
#pragma unroll
    for (int j = 0; j < 2 * kMaxRank; ++j) a[j] = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
      const double* pc = part + (static_cast<int64_t>(t) * nchunk + c) * (2 * kMaxRank);
#pragma unroll
      for (int j = 0; j < 2 * kMaxRank; ++j)
        if (j < 2 * r) a[j] += pc[j];
    }
    double f = 0.0;
#pragma unroll
    for (int j = 0; j < 2 * kMaxRank; ++j) {
      if (j < 2 * r) {
        double v = a[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        f += v * v;  // meaningful in lane 0
      }
    }
    if (lane == 0) {
      const int64_t s = idx[t];
      if (s < 0 || s >= S) f = -1.0;
      f_out[t] = f;
      if (f > my_best || (f == my_best && t < my_t)) {
        my_best = f;
        my_t = t;
      }
    }
  }
  bf[threadIdx.x] = my_best;
  bt[threadIdx.x] = my_t;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      double a = bf[threadIdx.x + h];
      int at = bt[threadIdx.x + h];
      if (a > bf[threadIdx.x] || (a == bf[threadIdx.x] && at < bt[threadIdx.x])) {
        bf[threadIdx.x] = a;
        bt[threadIdx.x] = at;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int t = bt[0];
    if (best_out) *best_out = (t < m) ? idx[t] : -1;
    if (best_f_out) *best_f_out = bf[0];
  }
}

int rescore_blocks_x(int m) { return (m + kRsCpb - 1) / kRsCpb; }

int launch_rescore(const RescorePlan& p, const Alphabet& a, const float2* V, const float2* C, int64_t S,
                   const int64_t* idx, double* part, double* f_out, uint8_t* z_out, int64_t* best_out,
                   double* best_f_out, int32_t* status, cudaStream_t st) {
  RescoreTables tab;
  tab.K = a.K;
  for (int k = 0; k < kMaxK; ++k) {
    bool in = k < a.K;
    // all K boundary lines (not only the B_K distinct ones)
    double th = kPi * (2.0 * k + 1.0) / a.K;
    double c = in ? cos(th) : 0.0, s = in ? sin(th) : 0.0;
    if (fabs(c) < 1e-15) c = 0.0;
    if (fabs(s) < 1e-15) s = 0.0;
    tab.bcos64[k] = c;
    tab.bsin64[k] = s;
    tab.bcos[k] = static_cast<float>(c);
    tab.bsin[k] = static_cast<float>(s);
    double zr = in ? a.zr64[k] : 0.0, zi = in ? a.zi64[k] : 0.0;
    tab.zrh[k] = static_cast<float>(zr);
    tab.zrl[k] = static_cast<float>(zr - static_cast<double>(tab.zrh[k]));
    tab.zih[k] = static_cast<float>(zi);
    tab.zil[k] = static_cast<float>(zi - static_cast<double>(tab.zih[k]));
  }
  dim3 grid(static_cast<unsigned>(rescore_blocks_x(p.m)), static_cast<unsigned>(p.nchunk));
  const bool r4 = p.r <= 4;
  switch (a.K) {
#define LRQ_RS_CASE(KK)                                                                                          \
  case KK:                                                                                                       \
    if (r4)                                                                                                      \
      rescore_partial_kernel<KK, 4><<<grid, kRsThreads, 0, st>>>(V, p.n, p.r, C, S, idx, p.m, p.nchunk,          \
                                                                 p.rows_per_chunk, tab, part, z_out, status);    \
    else                                                                                                         \
      rescore_partial_kernel<KK, kMaxRank><<<grid, kRsThreads, 0, st>>>(V, p.n, p.r, C, S, idx, p.m, p.nchunk,   \
                                                                        p.rows_per_chunk, tab, part, z_out,      \
                                                                        status);                                 \
    break;
    LRQ_RS_CASE(2)
    LRQ_RS_CASE(3)
    LRQ_RS_CASE(4)
    LRQ_RS_CASE(5)
    LRQ_RS_CASE(6)
    LRQ_RS_CASE(7)
    LRQ_RS_CASE(8)
#undef LRQ_RS_CASE
    default:
      if (r4)
        rescore_partial_kernel<0, 4><<<grid, kRsThreads, 0, st>>>(V, p.n, p.r, C, S, idx, p.m, p.nchunk,
                                                                  p.rows_per_chunk, tab, part, z_out, status);
      else
        rescore_partial_kernel<0, kMaxRank><<<grid, kRsThreads, 0, st>>>(V, p.n, p.r, C, S, idx, p.m, p.nchunk,
                                                                         p.rows_per_chunk, tab, part, z_out, status);
  }
  count_launch();
  int e = cuda_check(cudaGetLastError(), "rescore_partial_kernel");
  if (e) return e;
  rescore_final_kernel<<<1, 256, 0, st>>>(part, p.m, p.nchunk, p.r, idx, S, f_out, best_out, best_f_out);
  count_launch();
  return cuda_check(cudaGetLastError(), "rescore_final_kernel");
}

}  // namespace lrq
