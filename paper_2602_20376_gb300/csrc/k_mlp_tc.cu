// k_mlp_tc.cu -- the learned proposal's GEMMs in BF16 mode on the tensor
// cores (tcgen05): C = act(op(A) op(B) + bias), optionally zeroed where
// mask <= 0, with op(A) M x K and op(B) K x N, either stored transposed.
// The operands are rounded to bfloat16 (nearest even) as they are staged and
// the products accumulate in FP32 in tensor memory.
//
// One CTA of four warps per 128 x 64 output tile.  Per chunk of 64 along K
// the warps stage op(A) (128 rows x 64) and op(B) transposed (64 rows x 64)
// into shared memory in the no-swizzle K-major core-matrix order (8 rows x
// 16 bytes per core matrix; per MMA of K = 16, the rows' K 0..7 for all rows,
// then K 8..15), make the stores visible to the tensor core, and one elected
// thread issues four tcgen05.mma kind::f16 (BF16 x BF16 -> FP32, M 128, N 64,
// K 16) and commits them to an mbarrier that every thread waits for before
// the buffers are refilled.  Epilogue: each warp reads its 32 tensor-memory
// lanes (rows) x 64 columns and adds the bias, applies ReLU and the mask.
// The wait is bounded (~1 s); if it runs out (never observed) the kernel
// records the fault, writes NaN into its tile, waits (bounded) for its MMAs,
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lrq_device.cuh"
#include "lrq_internal.h"
#include "ptx_sm100.cuh"

namespace lrq {

constexpr int kMgM = 128, kMgN = 64, kMgK = 64, kMgThreads = 128;
constexpr long long kMgWait = 2000000000LL;
constexpr int kMgPadSmem = 8 * 1024;  // 24.6 KB static + 8 KB: 7 CTAs per SM at most

__device__ int32_t g_mlp_tc_fault = 0;

__global__ void __launch_bounds__(kMgThreads) mlp_gemm_tc_kernel(int M, int N, int K, const float* __restrict__ A,
                                                                 int lda, int ta, const float* __restrict__ Bm,
                                                                 int ldb, int tb, const float* __restrict__ bias,
                                                                 int relu, const float* __restrict__ mask,
                                                                 float* __restrict__ C, int ldc) {
  // 16 KB + 8 KB of operands (the launch adds unused dynamic shared memory
  // so that at most 7 CTAs share an SM and their 64-column tensor-memory
  // allocations always fit the 512)
  __shared__ __align__(1024) uint16_t sa[kMgM * kMgK];
  __shared__ __align__(1024) uint16_t sb[kMgN * kMgK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.y * kMgM, col0 = blockIdx.x * kMgN;
  if (tid == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(&tmem_slot, kMgN);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t sa_u = ptx::smem_u32(sa), sb_u = ptx::smem_u32(sb);
  constexpr uint32_t idesc = ptx::idesc_bf16_f32(kMgM, kMgN);
  volatile int never = 0;
  bool ok = true;
  uint32_t phase = 0;
  const int nchunk = (K + kMgK - 1) / kMgK;
  for (int ch = 0; ch < nchunk && ok; ++ch) {
    const int k0 = ch * kMgK;
    // op(A)(i, k) -> element ((q * 2 + h) * 128 + i) * 8 + e, k = 16 q + 8 h + e
    for (int t = tid; t < kMgM * kMgK; t += kMgThreads) {
      const int i = ta ? t % kMgM : t / kMgK;
      const int k = ta ? t / kMgM : t % kMgK;
      const int gi = row0 + i, gk = k0 + k;
      float v = 0.f;
      if (gi < M && gk < K) v = ta ? A[static_cast<int64_t>(gk) * lda + gi] : A[static_cast<int64_t>(gi) * lda + gk];
      sa[(((k >> 4) * 2 + ((k >> 3) & 1)) * kMgM + i) * 8 + (k & 7)] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    // op(B)(k, j) as row j of B's transpose -> ((q * 2 + h) * 64 + j) * 8 + e
    for (int t = tid; t < kMgN * kMgK; t += kMgThreads) {
      const int j = tb ? t / kMgK : t % kMgN;
      const int k = tb ? t % kMgK : t / kMgN;
      const int gj = col0 + j, gk = k0 + k;
      float v = 0.f;
      if (gj < N && gk < K) v = tb ? Bm[static_cast<int64_t>(gj) * ldb + gk] : Bm[static_cast<int64_t>(gk) * ldb + gj];
      sb[(((k >> 4) * 2 + ((k >> 3) & 1)) * kMgN + j) * 8 + (k & 7)] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    ptx::fence_proxy_async_smem();  // the staged operands, visible to the tensor core
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      ptx::tc_fence_after();
#pragma unroll
      for (int q = 0; q < kMgK / 16; ++q) {
        const uint64_t ad = ptx::smem_desc(sa_u + q * 2 * kMgM * 16, kMgM * 16, 128);
        const uint64_t bd = ptx::smem_desc(sb_u + q * 2 * kMgN * 16, kMgN * 16, 128);
        ptx::mma_f16_ss_elect(tmem, ad, bd, idesc, (ch > 0 || q > 0) ? 1u : 0u);
      }
      ptx::mma_commit_elect(&bar);
    }
    // the chunk's MMAs (and their reads of the buffers) are complete
    const bool done = ptx::mbar_wait(&bar, phase, &never, kMgWait);
    ok = __syncthreads_and(done) != 0;
    phase ^= 1u;
    ptx::tc_fence_after();
  }
  const int gi = row0 + warp * 32 + lane;
  if (ok) {
#pragma unroll
    for (int c0 = 0; c0 < kMgN; c0 += 16) {
      uint32_t v[16];
      ptx::tmem_ld_x16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      ptx::tmem_wait_ld();
      if (gi < M) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int gj = col0 + c0 + c;
          if (gj >= N) continue;
          float x = __uint_as_float(v[c]) + (bias ? bias[gj] : 0.f);
          if (relu) x = fmaxf(x, 0.f);
          if (mask && !(mask[static_cast<int64_t>(gi) * ldc + gj] > 0.f)) x = 0.f;
          C[static_cast<int64_t>(gi) * ldc + gj] = x;
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(&g_mlp_tc_fault, 1);
    if (gi < M)
      for (int gj = col0; gj < col0 + kMgN && gj < N; ++gj) C[static_cast<int64_t>(gi) * ldc + gj] = __int_as_float(0x7fc00000);
    // the MMAs still in flight complete before the tensor memory and the
    // shared buffers are released
    ptx::mbar_wait(&bar, phase ^ 1u, &never, kMgWait);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kMgN);
  }
}

void launch_mlp_gemm_tc(cudaStream_t st, int M, int N, int K, const float* A, int lda, int ta, const float* Bm,
                        int ldb, int tb, const float* bias, int relu, const float* mask, float* C, int ldc) {
  dim3 grid(static_cast<unsigned>(ceil_div(N, kMgN)), static_cast<unsigned>(ceil_div(M, kMgM)));
  mlp_gemm_tc_kernel<<<grid, kMgThreads, kMgPadSmem, st>>>(M, N, K, A, lda, ta, Bm, ldb, tb, bias, relu, mask, C,
                                                           ldc);
  count_launch();
}

}  // namespace lrq
