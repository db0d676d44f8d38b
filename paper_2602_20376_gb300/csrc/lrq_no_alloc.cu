// lrq_no_alloc.cu -- lrq_rescore_no_alloc: the FP64 re-scoring of
// lrq_rescore for callers that cannot allocate device memory.
//
// Who needs it: callers that must not call the CUDA allocator at all -- a
// plugin whose host framework owns every device allocation and hands it no
// allocator, a latency-critical request path where cudaMalloc / cudaFree
// (which may synchronise the whole device) are not acceptable, or a service
// that reserves a fixed memory budget at start-up and forbids allocation
// afterwards.  lrq_rescore needs a caller-provided workspace; this variant
// instead uses a fixed scratch array that lives in the library itself.
//
// The scratch is the file-scope array below (kNoAllocScratchBytes = 4 MiB).
// Every GPU that loads the library holds one copy of it until the process
// exits.  Host code cannot use the array's name as a device address, so the
// address is looked up with cudaGetSymbolAddress in the calling thread's
// current CUDA context the first time a call runs in that context, and
// cached per context: the address belongs to a context (a caller running in
// its own driver-API context, or one that reset the device and so got a new
// primary context, gets that context's address, never a stale one).  The
// first call in each context does this set-up; make it before any stream
// capture.  All calls in a context share the one array and it keeps the last
// call's contents: calls whose kernels overlap on the GPU (for instance on
// two streams) race on it and must be serialised by the caller.  Nothing in
// the array has to start at zero: every entry the kernels read is written
// earlier in the same call.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>
#include <vector>

#include "lrq_internal.h"

namespace lrq {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;

static __device__ __align__(256) unsigned char g_rescore_scratch[kNoAllocScratchBytes];

// The calling thread's current context and its process-unique id (driver
// entry points reached through the runtime, so the library links no
// libcuda).  False when no context is current.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

static bool current_context_id(unsigned long long* id) {
  static std::once_flag once;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

static int scratch_address(void** out) {
  static std::mutex mu;
  static std::vector<std::pair<unsigned long long, void*>> cache;  // context id -> address
  unsigned long long id = 0;
  void* p = nullptr;
  if (!current_context_id(&id)) {
    // no context current yet: the runtime's lookup makes the device's
    // primary context current; then it has an id
    cudaError_t e = cudaGetSymbolAddress(&p, g_rescore_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(LRQ_ECUDA, std::string("lrq_rescore_no_alloc: cudaGetSymbolAddress failed: ") +
                                 cudaGetErrorString(e));
    if (!current_context_id(&id)) return fail(LRQ_ECUDA, "lrq_rescore_no_alloc: no current CUDA context");
  }
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& kv : cache)
    if (kv.first == id) {
      *out = kv.second;
      return LRQ_OK;
    }
  if (p == nullptr) {
    cudaError_t e = cudaGetSymbolAddress(&p, g_rescore_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(LRQ_ECUDA, std::string("lrq_rescore_no_alloc: cudaGetSymbolAddress failed: ") +
                                 cudaGetErrorString(e));
  }
  cache.emplace_back(id, p);
  *out = p;
  return LRQ_OK;
}

}  // namespace lrq

using namespace lrq;

extern "C" int lrq_rescore_no_alloc(const void* V, int64_t n, int r, int K, const void* C, int64_t S,
                                    const int64_t* idx, int m, double* f_out, uint8_t* z_out, int64_t* best_out,
                                    double* best_f_out, int32_t* dev_status, void* stream) {
  if (n < 1) return fail(LRQ_EINVAL, "n must be >= 1");
  if (r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "r must be in [1, 8]");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (m < 1 || m > kMaxRescoreM) return fail(LRQ_EINVAL, "m must be in [1, 4096]");
  if (S < 1) return fail(LRQ_EINVAL, "S must be >= 1");
  if (!V || !C || !idx || !f_out || !best_out || !best_f_out || !dev_status)
    return fail(LRQ_EINVAL, "NULL pointer argument");
  RescorePlan p;
  plan_rescore(n, r, m, &p);
  if (p.total > kNoAllocScratchBytes)
    return fail(LRQ_EUNSUPPORTED, "lrq_rescore_no_alloc: this (n, r, m) needs " + std::to_string(p.total) +
                                      " bytes of scratch, more than the fixed 4 MiB (4194304 bytes); use "
                                      "lrq_rescore with a workspace");
  void* scratch = nullptr;
  int e = scratch_address(&scratch);
  if (e) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Alphabet a = make_alphabet(K);
  if ((e = launch_check_finite(reinterpret_cast<const float*>(V), 2 * n * r, dev_status, st))) return e;
  return launch_rescore(p, a, static_cast<const float2*>(V), static_cast<const float2*>(C), S, idx,
                        reinterpret_cast<double*>(static_cast<uint8_t*>(scratch) + p.off_part), f_out, z_out,
                        best_out, best_f_out, dev_status, st);
}
