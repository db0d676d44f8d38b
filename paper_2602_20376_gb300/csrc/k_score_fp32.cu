// k_score_fp32.cu -- direction sampler, input checks, column sums, CUDA-core
// FP32 candidate scoring and the per-candidate finalisation shared by both
// scoring modes.
//
// Scoring follows Sec. 4.2, Eq. 10: for direction c, w_i = V_i c, the decision
// rule of Sec. 3, Eq. 9 picks k_i, and f(c) = ||V^H z(c)||^2.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

// Uniform directions on the complex unit sphere: sphere_component (lrq_device.cuh).
__global__ void sample_directions_kernel(uint64_t seed, int64_t S, int r, float2* __restrict__ C) {
  int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= S) return;
  // each component is drawn once and kept (r <= kMaxRank)
  double a[kMaxRank], b[kMaxRank];
  double nrm2 = 0.0;
#pragma unroll
  for (int j = 0; j < kMaxRank; ++j) {
    if (j < r) {
      sphere_component(seed, s, j, &a[j], &b[j]);
      nrm2 += a[j] * a[j] + b[j] * b[j];
    }
  }
  double inv = 1.0 / sqrt(nrm2);
#pragma unroll
  for (int j = 0; j < kMaxRank; ++j)
    if (j < r) C[s * r + j] = make_float2(static_cast<float>(a[j] * inv), static_cast<float>(b[j] * inv));
}

int launch_sample_directions(uint64_t seed, int64_t S, int r, float2* C, cudaStream_t st) {
  if (S <= 0) return LRQ_OK;
  int64_t blocks = ceil_div(S, 256);
  sample_directions_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(seed, S, r, C);
  count_launch();
  return cuda_check(cudaGetLastError(), "sample_directions_kernel");
}

// ---------------------------------------------------------------------------
// Non-finite input check (the ABI reports LRQ_EINVAL through dev_status).
// ---------------------------------------------------------------------------
__global__ void check_finite_kernel(const float* __restrict__ x, int64_t count, int32_t* status) {
  int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) dev_fail(status, LRQ_EINVAL);
}

int launch_check_finite(const float* x, int64_t count, int32_t* status, cudaStream_t st) {
  if (count <= 0) return LRQ_OK;
  int blocks = static_cast<int>(std::min<int64_t>(ceil_div(count, 256), 4 * 152));
  check_finite_kernel<<<blocks, 256, 0, st>>>(x, count, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "check_finite_kernel");
}

// ---------------------------------------------------------------------------
// T = sum_i conj(V_i) in FP64 (the class-0 base of the odd-K indicator form).
// Stage 1: each block sums a contiguous row range; stage 2 adds the blocks in
// order (deterministic).
// ---------------------------------------------------------------------------
__global__ void colsum_stage1(const float2* __restrict__ V, int64_t n, int r, double* __restrict__ Tpart) {
  __shared__ double red[256][2 * kMaxRank];
  int64_t rows_per_block = ceil_div(n, gridDim.x);
  int64_t i0 = static_cast<int64_t>(blockIdx.x) * rows_per_block;
  int64_t i1 = min(n, i0 + rows_per_block);
  double acc[2 * kMaxRank];
#pragma unroll
  for (int j = 0; j < 2 * kMaxRank; ++j) acc[j] = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
#pragma unroll
    for (int j = 0; j < kMaxRank; ++j)
      if (j < r) {
        float2 v = V[i * r + j];
        acc[2 * j] += v.x;
        acc[2 * j + 1] -= v.y;
      }
  }
#pragma unroll
  for (int j = 0; j < 2 * kMaxRank; ++j) red[threadIdx.x][j] = acc[j];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j < 2 * r; ++j) red[threadIdx.x][j] += red[threadIdx.x + h][j];
    __syncthreads();
  }
  if (threadIdx.x < 2 * r) Tpart[blockIdx.x * 2 * kMaxRank + threadIdx.x] = red[0][threadIdx.x];
}

__global__ void colsum_stage2(const double* __restrict__ Tpart, int nblocks, int r, double* __restrict__ T) {
  int j = threadIdx.x;
  if (j >= 2 * r) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) a += Tpart[b * 2 * kMaxRank + j];
  T[j] = a;
}

int launch_colsum(const float2* V, int64_t n, int r, double* Tpart, double* T, int nblocks, cudaStream_t st) {
  colsum_stage1<<<nblocks, 256, 0, st>>>(V, n, r, Tpart);
  count_launch();
  int e = cuda_check(cudaGetLastError(), "colsum_stage1");
  if (e) return e;
  colsum_stage2<<<1, 32, 0, st>>>(Tpart, nblocks, r, T);
  count_launch();
  return cuda_check(cudaGetLastError(), "colsum_stage2");
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core scoring.
// Block: 256 candidates (one per thread) x one coordinate chunk (blockIdx.y).
// Coordinates are staged through shared memory 256 rows at a time and read
// back as broadcasts.  Per coordinate: w = V_i c (FP32 FMA), decision from
// the boundary-line signs, V^H z += conj(V_i) omega^k.  The FP32 running sum
// covers one 256-row batch and is then added into FP64 (blocked partials, so
// the FP32 error is that of a 256-term sum).
// Output: partial[chunk][s][2r] doubles = (Re, Im) of sum_{i in chunk} conj(V_i) z_i.
// ---------------------------------------------------------------------------
struct Fp32Tables {
  float bcos[8], bsin[8];
  float zr[kMaxK], zi[kMaxK];
};

constexpr int kFp32Block = 256;
constexpr int kFp32Batch = 256;

template <int K, int R>
__global__ void __launch_bounds__(kFp32Block) score_fp32_kernel(const float2* __restrict__ V, int64_t n,
                                                                const float2* __restrict__ C, int64_t S,
                                                                int64_t S_pad, int64_t rows_per_chunk,
                                                                int Kdyn, const __grid_constant__ Fp32Tables tab,
                                                                double* __restrict__ partial) {
  __shared__ float2 vs[kFp32Batch * R];
  __shared__ float2 ztab[kMaxK];
  const int Kr = (K > 0) ? K : Kdyn;
  for (int k = threadIdx.x; k < Kr; k += blockDim.x) ztab[k] = make_float2(tab.zr[k], tab.zi[k]);

  const int64_t s = static_cast<int64_t>(blockIdx.x) * kFp32Block + threadIdx.x;
  const bool active = s < S;
  float cr[R], ci[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    float2 c = active ? C[s * R + j] : make_float2(0.f, 0.f);
    cr[j] = c.x;
    ci[j] = c.y;
  }
  float bc[8], bs[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    bc[m] = tab.bcos[m];
    bs[m] = tab.bsin[m];
  }
  double acc64[2 * R];
#pragma unroll
  for (int j = 0; j < 2 * R; ++j) acc64[j] = 0.0;

  const int64_t i_begin = static_cast<int64_t>(blockIdx.y) * rows_per_chunk;
  const int64_t i_end = min(n, i_begin + rows_per_chunk);
  for (int64_t b0 = i_begin; b0 < i_end; b0 += kFp32Batch) {
    const int rows = static_cast<int>(min(static_cast<int64_t>(kFp32Batch), i_end - b0));
    __syncthreads();
    for (int t = threadIdx.x; t < rows * R; t += blockDim.x) vs[t] = V[b0 * R + t];
    __syncthreads();
    float acc[2 * R];
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) acc[j] = 0.f;
    for (int i = 0; i < rows; ++i) {
      float vr[R], vi[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        float2 v = vs[i * R + j];
        vr[j] = v.x;
        vi[j] = v.y;
      }
      float x = 0.f, y = 0.f;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        x = fmaf(vr[j], cr[j], x);
        x = fmaf(-vi[j], ci[j], x);
        y = fmaf(vr[j], ci[j], y);
        y = fmaf(vi[j], cr[j], y);
      }
      int k;
      if constexpr (K > 0)
        k = decide_fp32<K>(x, y, bc, bs);
      else
        k = decide_fp32_generic(x, y, Kr);
      float2 z = ztab[k];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        // conj(V_ij) z = (vr zr + vi zi) + i (vr zi - vi zr)
        acc[2 * j] = fmaf(vr[j], z.x, fmaf(vi[j], z.y, acc[2 * j]));
        acc[2 * j + 1] = fmaf(vr[j], z.y, fmaf(-vi[j], z.x, acc[2 * j + 1]));
      }
    }
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) acc64[j] += static_cast<double>(acc[j]);
  }
  if (active) {
    double* out = partial + (static_cast<int64_t>(blockIdx.y) * S_pad + s) * (2 * R);
#pragma unroll
    for (int j = 0; j < 2 * R; ++j) out[j] = acc64[j];
  }
}

template <int K>
static int launch_fp32_r(const ScorePlan& p, const Fp32Tables& tab, const float2* V, const float2* C,
                         double* partial, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>(ceil_div(p.S, kFp32Block)), static_cast<unsigned>(p.nsplit));
  int64_t S_pad = p.c_tiles * 128;
  switch (p.r) {
#define LRQ_FP32_CASE(RR)                                                                            \
  case RR:                                                                                           \
    score_fp32_kernel<K, RR><<<grid, kFp32Block, 0, st>>>(V, p.n, C, p.S, S_pad,                     \
                                                          p.fp32_rows_per_chunk, p.K, tab, partial); \
    break;
    count_launch();
    LRQ_FP32_CASE(1)
    LRQ_FP32_CASE(2)
    LRQ_FP32_CASE(3)
    LRQ_FP32_CASE(4)
    LRQ_FP32_CASE(5)
    LRQ_FP32_CASE(6)
    LRQ_FP32_CASE(7)
    LRQ_FP32_CASE(8)
#undef LRQ_FP32_CASE
    default:
      return fail(LRQ_EUNSUPPORTED, "score_fp32: r out of range");
  }
  return cuda_check(cudaGetLastError(), "score_fp32_kernel");
}

int launch_score_fp32(const ScorePlan& p, const Alphabet& a, const float2* V, const float2* C,
                      double* partial, cudaStream_t st) {
  Fp32Tables tab;
  for (int m = 0; m < 8; ++m) {
    tab.bcos[m] = m < a.BK ? a.bcos[m] : 0.f;
    tab.bsin[m] = m < a.BK ? a.bsin[m] : 0.f;
  }
  for (int k = 0; k < kMaxK; ++k) {
    tab.zr[k] = k < a.K ? a.zr[k] : 0.f;
    tab.zi[k] = k < a.K ? a.zi[k] : 0.f;
  }
  switch (p.K) {
    case 2: return launch_fp32_r<2>(p, tab, V, C, partial, st);
    case 3: return launch_fp32_r<3>(p, tab, V, C, partial, st);
    case 4: return launch_fp32_r<4>(p, tab, V, C, partial, st);
    case 5: return launch_fp32_r<5>(p, tab, V, C, partial, st);
    case 6: return launch_fp32_r<6>(p, tab, V, C, partial, st);
    case 7: return launch_fp32_r<7>(p, tab, V, C, partial, st);
    case 8: return launch_fp32_r<8>(p, tab, V, C, partial, st);
    default: return launch_fp32_r<0>(p, tab, V, C, partial, st);
  }
}

// ---------------------------------------------------------------------------
// Finalisation: add the chunk partials in FP64 (in chunk order), add the base
// T for the odd-K indicator form, f = ||.||^2.  Writes the FP32 score and the
// selection key (score bits above the complemented index: larger key = larger
// f, ties to the smaller index).
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const double* __restrict__ partial, int nsplit, int64_t S, int64_t S_pad, int r,
                                const double* __restrict__ T, float* __restrict__ scores,
                                uint64_t* __restrict__ keys) {
  int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double v[2 * kMaxRank];
#pragma unroll
  for (int j = 0; j < 2 * kMaxRank; ++j) v[j] = (T && j < 2 * r) ? T[j] : 0.0;
  for (int c = 0; c < nsplit; ++c) {
    const double* src = partial + (static_cast<int64_t>(c) * S_pad + s) * (2 * r);
#pragma unroll
    for (int j = 0; j < 2 * kMaxRank; ++j)
      if (j < 2 * r) v[j] += src[j];
  }
  double f = 0.0;
#pragma unroll
  for (int j = 0; j < 2 * kMaxRank; ++j)
    if (j < 2 * r) f += v[j] * v[j];
  float ff = static_cast<float>(f);
  if (scores) scores[s] = ff;
  if (keys)
    keys[s] = (static_cast<uint64_t>(__float_as_uint(ff)) << 32) |
              static_cast<uint64_t>(0xFFFFFFFFu - static_cast<uint32_t>(s));
}

int launch_finalize(const ScorePlan& p, const Alphabet& a, const double* partial, const double* T,
                    float* scores, uint64_t* keys, cudaStream_t st) {
  (void)a;
  int64_t S_pad = p.c_tiles * 128;
  finalize_kernel<<<static_cast<unsigned>(ceil_div(p.S, 256)), 256, 0, st>>>(partial, p.npart, p.S, S_pad, p.r,
                                                                             T, scores, keys);
  count_launch();
  return cuda_check(cudaGetLastError(), "finalize_kernel");
}

}  // namespace lrq
