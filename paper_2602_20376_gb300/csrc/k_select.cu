// k_select.cu -- top-m selection of scored candidates ("returns only the best
// candidate found", Sec. 5; best-of-S, Sec. 4.2), generalised to the m best
// for the FP64 re-scoring step.
//
// Keys are 64-bit: the FP32 score bits (scores are >= 0, so their bit
// patterns order like the values) above 0xFFFFFFFF - index, so the key order
// is "larger score first, then smaller index".  Each pass sorts segments of
// kSeg keys in shared memory with a bitonic network (descending) and keeps
// the first m of every segment; passes repeat until one segment remains.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kSeg = 2048;
constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads) topm_pass_kernel(const uint64_t* __restrict__ in, int64_t count,
                                                                int m, uint64_t* __restrict__ out,
                                                                int64_t* __restrict__ top_idx,
                                                                float* __restrict__ top_f) {
  __shared__ uint64_t sk[kSeg];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSeg;
  for (int t = threadIdx.x; t < kSeg; t += blockDim.x) sk[t] = (base + t < count) ? in[base + t] : 0ull;
  __syncthreads();
  // bitonic sort, descending
  for (int size = 2; size <= kSeg; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < kSeg / 2; t += blockDim.x) {
        int lo = 2 * t - (t & (stride - 1));
        int hi = lo + stride;
        bool desc = ((lo & size) == 0);
        uint64_t a = sk[lo], b = sk[hi];
        bool swap = desc ? (a < b) : (a > b);
        if (swap) {
          sk[lo] = b;
          sk[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  if (top_idx) {  // final pass: decode
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      uint64_t k = sk[t];
      top_idx[t] = static_cast<int64_t>(0xFFFFFFFFu - static_cast<uint32_t>(k & 0xFFFFFFFFull));
      top_f[t] = __uint_as_float(static_cast<uint32_t>(k >> 32));
    }
  } else {
    for (int t = threadIdx.x; t < m; t += blockDim.x) out[static_cast<int64_t>(blockIdx.x) * m + t] = sk[t];
  }
}

size_t topm_scratch_keys(int64_t count, int m) {
  // two ping-pong buffers, each large enough for the first pass output
  int64_t segs = ceil_div(count, kSeg);
  return static_cast<size_t>(2 * segs * m);
}

int launch_topm(const uint64_t* keys_in, int64_t count, int m, uint64_t* scratch, int64_t* top_idx, float* top_f,
                cudaStream_t st) {
  if (m < 1 || m > kSeg / 4) return fail(LRQ_EUNSUPPORTED, "top_m out of range");
  int64_t segs0 = ceil_div(count, kSeg);
  uint64_t* buf[2] = {scratch, scratch + segs0 * m};
  const uint64_t* src = keys_in;
  int64_t cnt = count;
  int which = 0;
  for (;;) {
    int64_t segs = ceil_div(cnt, kSeg);
    if (segs <= 1) {
      topm_pass_kernel<<<1, kSelThreads, 0, st>>>(src, cnt, m, nullptr, top_idx, top_f);
      count_launch();
      return cuda_check(cudaGetLastError(), "topm_pass_kernel(final)");
    }
    topm_pass_kernel<<<static_cast<unsigned>(segs), kSelThreads, 0, st>>>(src, cnt, m, buf[which], nullptr,
                                                                          nullptr);
    count_launch();
    int e = cuda_check(cudaGetLastError(), "topm_pass_kernel");
    if (e) return e;
    src = buf[which];
    cnt = segs * m;
    which ^= 1;
  }
}

}  // namespace lrq
