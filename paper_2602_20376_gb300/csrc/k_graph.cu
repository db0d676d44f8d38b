// k_graph.cu -- exact Max-K-Cut count on a CSR graph (Sec. 1: K = 3 with a
// Laplacian objective is Max-3-Cut).  cut(z) = #{ {i,j} in E : k_i != k_j },
// each undirected edge counted once, from its lower endpoint, in int64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

__global__ void cut_count_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                 int64_t n, const uint8_t* __restrict__ z, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long red[256];
  unsigned long long cnt = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint8_t zi = z[i];
    const int32_t e1 = rowptr[i + 1];
    for (int32_t e = rowptr[i]; e < e1; ++e) {
      const int32_t j = colidx[e];
      cnt += (j > i && z[j] != zi) ? 1ull : 0ull;
    }
  }
  red[threadIdx.x] = cnt;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

int launch_cut_count(const int32_t* rowptr, const int32_t* colidx, int64_t n, const uint8_t* z, int64_t* cut_out,
                     cudaStream_t st) {
  int e = cuda_check(cudaMemsetAsync(cut_out, 0, sizeof(int64_t), st), "cudaMemsetAsync(cut_out)");
  if (e) return e;
  if (n <= 0) return LRQ_OK;
  int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 8 * 152));
  cut_count_kernel<<<blocks, 256, 0, st>>>(rowptr, colidx, n, z, reinterpret_cast<unsigned long long*>(cut_out));
  count_launch();
  return cuda_check(cudaGetLastError(), "cut_count_kernel");
}

}  // namespace lrq
