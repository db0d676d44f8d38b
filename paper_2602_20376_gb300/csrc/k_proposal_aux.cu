// k_proposal_aux.cu -- the learned proposal's data preparation: training
// targets in the canonical window, and feature standardisation.
//
// Targets.  Directions c and omega^k c (omega = exp(2 pi i / K)) give the
// same assignment up to a global phase and the same objective (Sec. 2.3, the
// K-fold equivalence of the rounding), so a direction is represented by the
// one of its K rotations whose first component has its argument in
// (-pi/K, pi/K]: c omega^-k with k = ceil(K arg(c_1) / (2 pi) - 1/2).  The
// selected directions (their indices come from the scoring's top-m
// selection) are gathered, rotated and written as 2r reals
// (Re c_1, Im c_1, Re c_2, ...).  FP64 inside; one thread per direction.
//
// Standardisation.  Each feature is centred on its mean over the training
// instances and divided by its sample standard deviation (ddof 1; at least
// 1e-6, and 1 for a single instance); FP64 sums, one block per feature.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

__global__ void proposal_targets_kernel(const float2* __restrict__ C, int64_t S, const int64_t* __restrict__ idx,
                                        int64_t m, int r, int K, float* __restrict__ out, int32_t* status) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int64_t s = idx[t];
  float* o = out + t * 2 * r;
  if (s < 0 || s >= S) {
    dev_fail(status, LRQ_EINVAL);
    for (int j = 0; j < 2 * r; ++j) o[j] = 0.f;
    return;
  }
  const float2* c = C + s * r;
  const double ang = atan2(static_cast<double>(c[0].y), static_cast<double>(c[0].x));
  const double k = ceil(ang * K / (2.0 * M_PI) - 0.5);  // arg - 2 pi k / K in (-pi/K, pi/K]
  double sn, cs;
  sincos(-2.0 * M_PI * k / K, &sn, &cs);
  for (int j = 0; j < r; ++j) {
    const double x = c[j].x, y = c[j].y;
    o[2 * j] = static_cast<float>(x * cs - y * sn);
    o[2 * j + 1] = static_cast<float>(x * sn + y * cs);
  }
}

__global__ void standardize_fit_kernel(const float* __restrict__ feat, int B, int F, float* __restrict__ mean,
                                       float* __restrict__ sd) {
  const int f = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += feat[static_cast<int64_t>(b) * F + f];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double mu = red[0] / B;
  __syncthreads();
  double q = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double d = feat[static_cast<int64_t>(b) * F + f] - mu;
    q += d * d;
  }
  red[threadIdx.x] = q;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mean[f] = static_cast<float>(mu);
    sd[f] = B > 1 ? static_cast<float>(fmax(sqrt(red[0] / (B - 1)), 1e-6)) : 1.f;
  }
}

__global__ void standardize_apply_kernel(const float* __restrict__ feat, int64_t total, int F,
                                         const float* __restrict__ mean, const float* __restrict__ sd,
                                         float* __restrict__ X) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int f = static_cast<int>(q % F);
  X[q] = (feat[q] - mean[f]) / sd[f];
}

int launch_proposal_targets(const float2* C, int64_t S, const int64_t* idx, int64_t m, int r, int K, float* out,
                            int32_t* status, cudaStream_t st) {
  proposal_targets_kernel<<<static_cast<unsigned>(ceil_div(m, 128)), 128, 0, st>>>(C, S, idx, m, r, K, out, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "proposal_targets_kernel");
}

int launch_standardize_fit(const float* feat, int B, int F, float* mean, float* sd, cudaStream_t st) {
  standardize_fit_kernel<<<F, 256, 0, st>>>(feat, B, F, mean, sd);
  count_launch();
  return cuda_check(cudaGetLastError(), "standardize_fit_kernel");
}

int launch_standardize(const float* feat, int B, int F, const float* mean, const float* sd, float* X,
                       cudaStream_t st) {
  const int64_t total = static_cast<int64_t>(B) * F;
  standardize_apply_kernel<<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(feat, total, F, mean, sd,
                                                                                        X);
  count_launch();
  return cuda_check(cudaGetLastError(), "standardize_apply_kernel");
}

}  // namespace lrq
