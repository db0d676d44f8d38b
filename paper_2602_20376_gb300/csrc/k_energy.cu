// k_energy.cu -- the spectral energy ratio rho_r (Sec. 5, "When does low-rank
// work?"): the share of Q's spectral energy that the top r eigenvalues leave
// out, rho_r = 1 - sum_{j<=r} lambda_j / sum_j lambda_j, over the positive
// spectrum.  For the PSD Q the paper assumes (Sec. 1) the denominator is
// trace(Q), so only the top r eigenvalues (from the truncation) and one
// reduction over Q are needed: sum_i Re Q_ii for a dense Q, the sum of all
// edge weights in both rows (self loops ignored) for a graph Laplacian.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kEnThreads = 256;

__device__ __forceinline__ void en_add(double v, double* out) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

// trace(D - A) = sum of the weighted degrees
__global__ void __launch_bounds__(kEnThreads) en_trace_csr(const int32_t* __restrict__ rowptr,
                                                           const int32_t* __restrict__ colidx,
                                                           const double* __restrict__ wts, int64_t n, int64_t nnz,
                                                           double* trace, int32_t* status) {
  double acc = 0.0;
  bool bad = false;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t0 == 0) bad |= rowptr[0] != 0 || static_cast<int64_t>(rowptr[n]) != nnz;
  for (int64_t i = t0; i < n; i += stride) {
    const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
    if (e0 < 0 || e0 > e1 || e1 > nnz) {
      bad = true;
      continue;
    }
    for (int64_t e = e0; e < e1; ++e) {
      const int32_t j = colidx[e];
      if (j < 0 || j >= n) {
        bad = true;
        continue;
      }
      const double w = wts ? wts[e] : 1.0;
      if (!isfinite(w)) bad = true;
      if (j != i) acc += w;
    }
  }
  if (bad) dev_fail(status, LRQ_EINVAL);
  en_add(acc, trace);
}

__global__ void __launch_bounds__(kEnThreads) en_trace_dense(const double2* __restrict__ Q, int64_t n, int64_t ld,
                                                             double* trace, int32_t* status) {
  double acc = 0.0;
  bool bad = false;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double d = Q[i * ld + i].x;
    if (!isfinite(d)) bad = true;
    acc += d;
  }
  if (bad) dev_fail(status, LRQ_EINVAL);
  en_add(acc, trace);
}

// rho_r from the trace and the top r eigenvalues (non-positive ones carry no
// energy); a zero trace (Q = 0) gives 0, a negative one (Q not PSD) EINVAL
__global__ void en_rho_kernel(const double* __restrict__ lambda, int r, const double* trace, double* rho,
                              int32_t* status) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int j = 0; j < r; ++j) {
    const double l = lambda[j];
    if (!isfinite(l)) dev_fail(status, LRQ_EINVAL);
    s += l > 0.0 ? l : 0.0;
  }
  const double t = *trace;
  if (t < 0.0 || !isfinite(t)) {
    dev_fail(status, LRQ_EINVAL);
    *rho = 0.0;
    return;
  }
  *rho = t > 0.0 ? 1.0 - s / t : 0.0;
}

int launch_spectral_energy(const lrq_matrix* Q, const double* lambda, int r, double* trace_out, double* rho_out,
                           int32_t* status, cudaStream_t st) {
  int e = cuda_check(cudaMemsetAsync(trace_out, 0, sizeof(double), st), "cudaMemsetAsync(trace_out)");
  if (e) return e;
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(Q->n, kEnThreads), 152 * 8)));
  if (Q->kind == LRQ_MATRIX_DENSE_C128) {
    en_trace_dense<<<blocks, kEnThreads, 0, st>>>(static_cast<const double2*>(Q->values), Q->n, Q->ld, trace_out,
                                                  status);
  } else {
    en_trace_csr<<<blocks, kEnThreads, 0, st>>>(Q->rowptr, Q->colidx, Q->weights, Q->n, Q->nnz, trace_out, status);
  }
  en_rho_kernel<<<1, 32, 0, st>>>(lambda, r, trace_out, rho_out, status);
  count_launch(2);
  return cuda_check(cudaGetLastError(), "spectral energy kernels");
}

}  // namespace lrq
