// k_greedy.cu -- greedy local search for Max-K-Cut on a CSR graph, the
// refinement step of the hybrid solver (App. "Hybrid Warm-Start": rank-1
// sweep first, then greedy hill-climbing from its partition).
//
// A vertex i with label z_i and neighbour counts n_i(c) = #{j in N(i), j != i :
// z_j = c} gains g_i = n_i(z_i) - min_{c != z_i} n_i(c) by moving to the label
// of that minimum (ties to the smallest label).  Steepest ascent moves the
// vertex of largest gain.  On the GPU a round moves, at once, every gaining
// vertex that no gaining neighbour outranks, under the strict order (larger
// gain, then smaller index): the moved set is independent, so the gains add
// exactly, and it always contains the steepest move, so every round raises
// the cut and the search ends at a state no single move improves.
//
// A round is two kernels over the adjacency (gains, then moves), 8 lanes per
// row.  Rounds are issued in batches of kGrBatch; each round's move count
// lands in a device ring, the next round returns at once when it is zero, and
// the host reads the ring once per batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kGrThreads = 256;
constexpr int kGrBatch = 8;
constexpr int kGrMaxK = 8;

__device__ __forceinline__ bool gr_row(const int32_t* __restrict__ rowptr, int64_t i, int64_t nnz, int64_t* e0,
                                       int64_t* e1) {
  const int64_t a = rowptr[i], b = rowptr[i + 1];
  *e0 = a;
  *e1 = b;
  return a >= 0 && a <= b && b <= nnz;
}

// gain and target label of every vertex (0 gain when no move helps)
__global__ void __launch_bounds__(kGrThreads) gr_gain_kernel(const int32_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ colidx, int64_t n,
                                                             int64_t nnz, int K, const uint8_t* __restrict__ z,
                                                             int32_t* __restrict__ gain, uint8_t* __restrict__ best,
                                                             const unsigned long long* prev, int32_t* status) {
  if (prev && *prev == 0ull) return;
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t rb = warp * 4; rb < n; rb += nwarps * 4) {  // warp-uniform trip count
    const int64_t i = rb + (lane >> 3);
    int cnt[kGrMaxK];
#pragma unroll
    for (int c = 0; c < kGrMaxK; ++c) cnt[c] = 0;
    int zi = 0;
    bool ok = false;
    if (i < n) {
      zi = z[i];
      int64_t e0, e1;
      ok = gr_row(rowptr, i, nnz, &e0, &e1);
      if (!ok || zi >= K) {
        if (sub == 0) dev_fail(status, LRQ_EINVAL);
        ok = false;
      } else {
        for (int64_t e = e0 + sub; e < e1; e += 8) {
          const int32_t j = colidx[e];
          if (j < 0 || j >= n) {
            dev_fail(status, LRQ_EINVAL);
            continue;
          }
          if (j == i) continue;
          const int zj = z[j];
#pragma unroll
          for (int c = 0; c < kGrMaxK; ++c) cnt[c] += (zj == c) ? 1 : 0;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kGrMaxK; ++c) {
#pragma unroll
      for (int m = 4; m > 0; m >>= 1) cnt[c] += __shfl_xor_sync(0xffffffffu, cnt[c], m);
    }
    if (sub == 0 && i < n) {
      int same = 0, bc = -1, bv = 0;
#pragma unroll
      for (int c = 0; c < kGrMaxK; ++c) {
        if (c >= K) break;
        if (c == zi) {
          same = cnt[c];
        } else if (bc < 0 || cnt[c] < bv) {
          bc = c;
          bv = cnt[c];
        }
      }
      const int g = (ok && bc >= 0) ? same - bv : 0;
      gain[i] = g > 0 ? g : 0;
      best[i] = static_cast<uint8_t>(g > 0 ? bc : zi);
    }
  }
}

// move every gaining vertex that no gaining neighbour outranks
__global__ void __launch_bounds__(kGrThreads) gr_move_kernel(const int32_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ colidx, int64_t n,
                                                             int64_t nnz, const int32_t* __restrict__ gain,
                                                             const uint8_t* __restrict__ best, uint8_t* __restrict__ z,
                                                             const unsigned long long* prev,
                                                             unsigned long long* moved) {
  if (prev && *prev == 0ull) return;
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  unsigned long long mine = 0;
  for (int64_t rb = warp * 4; rb < n; rb += nwarps * 4) {
    const int64_t i = rb + (lane >> 3);
    const int gi = i < n ? gain[i] : 0;
    bool blocked = gi <= 0;
    if (!blocked) {
      int64_t e0, e1;
      if (gr_row(rowptr, i, nnz, &e0, &e1)) {
        for (int64_t e = e0 + sub; e < e1 && !blocked; e += 8) {
          const int32_t j = colidx[e];
          if (j < 0 || j >= n || j == i) continue;
          const int gj = gain[j];
          blocked = gj > gi || (gj == gi && j < i);
        }
      } else {
        blocked = true;
      }
    }
    // a row's 8 lanes agree on the verdict
    const unsigned any = __ballot_sync(0xffffffffu, blocked);
    const bool row_blocked = (any >> (lane & ~7)) & 0xFFu;
    if (sub == 0 && i < n && gi > 0 && !row_blocked) {
      z[i] = best[i];
      ++mine;
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, m);
  if (lane == 0 && mine) atomicAdd(moved, mine);
}

size_t greedy_workspace_bytes(int64_t n) {
  return align_up(sizeof(int32_t) * static_cast<size_t>(n), 256) + align_up(static_cast<size_t>(n), 256) +
         align_up(sizeof(unsigned long long) * 2 * kGrBatch, 256);
}

int launch_greedy(const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz, int K, uint8_t* z,
                  int64_t max_rounds, int64_t* cut_out, int64_t* rounds_out, int64_t* moves_out,
                  int32_t* converged_out, void* ws, int32_t* status, cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  int32_t* gain = reinterpret_cast<int32_t*>(base);
  base += align_up(sizeof(int32_t) * static_cast<size_t>(n), 256);
  uint8_t* best = reinterpret_cast<uint8_t*>(base);
  base += align_up(static_cast<size_t>(n), 256);
  unsigned long long* ring = reinterpret_cast<unsigned long long*>(base);

  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 32), 152 * 16)));
  int64_t launched = 0, rounds = 0, moves = 0;
  bool converged = false;
  int e = LRQ_OK;
  for (int64_t b = 0; launched < max_rounds && !converged; ++b) {
    unsigned long long* slot = ring + (b & 1) * kGrBatch;
    if ((e = cuda_check(cudaMemsetAsync(slot, 0, sizeof(unsigned long long) * kGrBatch, st), "memset ring")))
      return e;
    const int nr = static_cast<int>(std::min<int64_t>(kGrBatch, max_rounds - launched));
    for (int t = 0; t < nr; ++t) {
      const unsigned long long* prev =
          (b == 0 && t == 0) ? nullptr : (t == 0 ? ring + ((b - 1) & 1) * kGrBatch + (kGrBatch - 1) : slot + t - 1);
      gr_gain_kernel<<<blocks, kGrThreads, 0, st>>>(rowptr, colidx, n, nnz, K, z, gain, best, prev, status);
      gr_move_kernel<<<blocks, kGrThreads, 0, st>>>(rowptr, colidx, n, nnz, gain, best, z, prev, slot + t);
      count_launch(2);
    }
    if ((e = cuda_check(cudaGetLastError(), "greedy kernels"))) return e;
    unsigned long long hm[kGrBatch];
    int32_t hs = 0;
    if ((e = cuda_check(cudaMemcpyAsync(hm, slot, sizeof(hm), cudaMemcpyDeviceToHost, st), "copy moves"))) return e;
    if ((e = cuda_check(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy status")))
      return e;
    if ((e = cuda_check(cudaStreamSynchronize(st), "greedy sync"))) return e;
    if (hs != 0) return fail(hs, "lrq_greedy_cut: the device reported an invalid graph or label");
    for (int t = 0; t < nr; ++t) {
      if (hm[t] == 0) {
        converged = true;
        break;
      }
      ++rounds;
      moves += static_cast<int64_t>(hm[t]);
    }
    launched += nr;
  }
  if (max_rounds == 0) {  // no round ran: validate labels and graph before the cut reads them
    gr_gain_kernel<<<blocks, kGrThreads, 0, st>>>(rowptr, colidx, n, nnz, K, z, gain, best, nullptr, status);
    count_launch();
    int32_t hs = 0;
    if ((e = cuda_check(cudaGetLastError(), "greedy gain kernel"))) return e;
    if ((e = cuda_check(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy status")))
      return e;
    if ((e = cuda_check(cudaStreamSynchronize(st), "greedy sync"))) return e;
    if (hs != 0) return fail(hs, "lrq_greedy_cut: the device reported an invalid graph or label");
  }
  if (rounds_out) *rounds_out = rounds;
  if (moves_out) *moves_out = moves;
  if (converged_out) *converged_out = converged ? 1 : 0;
  if (cut_out) return launch_cut_count(rowptr, colidx, n, z, cut_out, st);
  return LRQ_OK;
}

}  // namespace lrq
