// k_score_tc.cu -- tensor-core (tcgen05 + TMEM + TMA) candidate scoring.
//
// The scoring of Sec. 4.2, Eq. 10 is cast as two contractions per
// (128-candidate tile, coordinate tile):
//
// GEMM1 (boundary projections, F16).  The augmented real matrix of Eq. 6 has
// one row per (coordinate i, boundary m): [Im(rho_m V_i), Re(rho_m V_i)] with
// rho_m = exp(-i theta_m), theta_m = pi(2m+1)/K, m < B_K (Definition 2.1).
// Against c~ = [Re c; Im c] a row gives p_m = Im(rho_m V_i c), whose sign says
// on which side of decision boundary m the value w_i = V_i c lies.  So
//   D1[s, (m, i)] = sum_k C~[s, k] * Vaug[(m, i), k]     (M = 128, K = 2r -> 16)
// and the decision rule (Sec. 3, Eq. 9) becomes a sign test per row.  Signs
// do not change under positive scales, so every coordinate row and every
// direction is scaled by a power of two (largest component into [1, 2)) and
// GEMM1 runs in F16 with an F16 accumulator: full range safety, F16's
// precision, and the projections come back two per register.
//
// Sector rounding in the epilogue.  With N_m the sign mask of p_m:
//   odd K  : class k in 1..K-1 iff p_{k-1} > 0 and p_k < 0  -> indicator 1/0
//   even K : z = sum_m beta_m sign(p_m), beta_m = (w^{m+1} - w^m)/2   -> +-1
// (w = exp(2 pi i/K)).  Indicators are exact in FP8 (E4M3 0x38 = 1.0, 0xB8 =
// -1.0, times a per-coordinate power of two, see GEMM2); the signs of four
// coordinates are gathered into one word by one byte permute (sign
// replication) of two packed F16 registers and turned into indicators with
// one 3-input logic op -- no trigonometry, no branches.
//
// GEMM2 (per-class sums, FP8 x FP8 -> FP32).  V^H z = T + sum_k (w^k - 1) P_k
// (odd K, T the column sum of conj(V)) or sum_m beta_m S_m (even K), where
// P_k / S_m are sums of conj(V_i) selected or signed by the indicators:
//   D2[s, :] += sum_{(g, i)} Ind[s, (g, i)] * B2[(g, i), :]
// with B2 rows the real form of beta_g conj(V_i), scaled by a power of two s
// and split as hi + lo, two E4M3 numbers whose sum carries about 8
// significant bits (like BF16).  hi and lo are separate output columns
// (N = 2 x 8, or 2 x 16 for r > 4); the epilogue adds them and divides by s.
// An FP8 MMA reduces 32 entries where a BF16 one reduces 16, so GEMM2 takes
// half the MMA instructions.  D2 accumulates in TMEM (FP32) over an
// accumulation period of at most 2048 coordinates, then is folded into FP32
// two-sum registers (error-free) and written as FP64 partials per coordinate
// chunk.
//
// Pipeline (one CTA per SM, persistent over (chunk, candidate tile) items,
// every role a warp or warpgroup of its own, all hand-offs through
// mbarriers):
//   TMA warp      fills a ring of NS stages (one packed coordinate tile each:
//                 GEMM1 rows | GEMM2 rows | indicator magnitudes, one box)
//                 and two direction buffers (one per item);
//   GEMM1 warp    for every tile g: waits for the tile's stage and for D1
//                 buffer g % ND (a ring of ND buffers in tensor memory),
//                 arrives on the buffer's barrier (telling the rounding warps
//                 that the stage has landed) and issues the projections; the
//                 buffer's barrier completes on that arrival and the MMA.  It
//                 runs ahead of the rounding as far as the ring allows, and
//                 polls its two barriers together (every mbarrier wait costs
//                 ~100 cycles even when its phase has completed);
//   GEMM2 warps   two streams (one thread issues a small FP8 MMA only every
//                 ~32 cycles): stream v = g % 2 issues tile g from
//                 A2[g % NWG] into its accumulator D2[v][p % NB2], p the
//                 stream's accumulation period (at most 2048 coordinates of
//                 one item); warpgroup w signals stream v's tiles on its own
//                 barrier [w][v], so that every barrier of the pipeline is
//                 waited for by one party, phase after phase (a parity wait
//                 that runs a phase ahead of its barrier passes on the wrong
//                 phase);
//   rounding      NWG = ND warpgroups, one thread per candidate row;
//                 warpgroup w = g % NWG takes tile g and owns D1 buffer w
//                 and A2 buffer w: one wait, then D1 chunk by chunk (16 or
//                 32 coordinates), the next chunk's tensor-memory load in
//                 flight while the current one is rounded with its indicator
//                 magnitudes (read from the tile's stage); the buffer is
//                 released once its last chunk is in registers, and the
//                 indicator words go into the warpgroup's own A2 buffer
//                 (three warpgroups hide the latency of their waits);
//   fold          a warpgroup that owns the two-sum partials: per item it
//                 reads period i of stream 0, then period i of stream 1, for
//                 i = 0, 1, ..., releases each accumulator, and writes the
//                 item's FP64 partials at its end.
// The rounding warpgroups, which do all the per-evaluation work, never wait
// for an MMA they have just asked for: D1 of their next tile was issued while
// they rounded the previous ones, and their A2 buffer was released by a GEMM2
// issued a tile earlier.  Every wait is an mbarrier try_wait loop (try_wait
// blocks in hardware until the phase completes or a time limit passes) and
// is bounded; on expiry the kernel records LRQ_ETIMEOUT, every role leaves
// its loop, in-flight
// copies and MMAs are drained, TMEM is freed and the CTA returns.  The
// protocol is model-checked on the CPU (tests/protocol_model.py).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "lrq_device.cuh"
#include "lrq_internal.h"
#include "ptx_sm100.cuh"

namespace lrq {

constexpr int kTcM = 128;
constexpr int kTcMaxStages = 24;
constexpr int kTcPeriodCoords = 2048;  // coordinates per FP32 accumulation period
constexpr long long kWaitLimit = 2000000000LL;
constexpr int kTcMaxNwg = 3;  // rounding warpgroups at most (one per D1 buffer)

// Tile shape per alphabet and rank class (KCH = 1 for r <= 4, 2 above).  R is
// the number of coordinates per tile.  Tensor memory (512 columns of 128
// lanes) holds
//   D1 : ND buffers of N1 = BKG * R columns     GEMM1 projections (F16, one per column)
//   D2 : 2 x NB2 buffers of N2 = 2 * NOUT cols  GEMM2 accumulators, hi | lo, NB2 per stream
// and shared memory the GEMM2 indicator operand A2 (128 rows x KD2 FP8 bytes
// per rounding warpgroup).  The cost of a tile is nearly fixed (its
// hand-offs), so R is the largest that lets three D1 buffers and the
// accumulators fit.
template <int K, int KCH>
struct TcShape {
  static constexpr int BK = (K % 2 == 0) ? K / 2 : K;
  // boundary lines projected by GEMM1: all B_K, except K = 3 where the three
  // lines' directions sum to zero, so p_1 = -(p_0 + p_2) is formed on the
  // CUDA cores
  static constexpr int BKG = (K == 3) ? 2 : BK;
  static constexpr int G = (K % 2 == 0) ? K / 2 : K - 1;
  static constexpr int R = K == 2 ? 128 : (K == 3 || K == 4) ? (KCH == 1 ? 80 : 64) : K == 7 ? 16 : 32;
  static constexpr int ROWS = R;  // coordinates per tile (packing granularity)
  static constexpr int N1 = BKG * R;   // GEMM1 N
  static constexpr int KD2 = G * R;    // GEMM2 reduction length per tile
  static constexpr int A2WORDS = KD2 / 4;  // indicator words (4 FP8 each) per candidate row
  static constexpr int NOUT = KCH == 1 ? 8 : 16;  // real outputs per candidate (>= 2r)
  static constexpr int N2 = 2 * NOUT;             // GEMM2 N: hi and lo halves
  // D1 buffers (one per rounding warpgroup) and accumulators per stream:
  // the deepest that fit, D1 first
  static constexpr int cols(int nd, int nb2) { return nd * N1 + 2 * nb2 * N2; }
  static constexpr int ND = cols(3, 1) <= 512 ? 3 : 2;
  // rounding warpgroups: warpgroup w owns D1 buffer w, so that every
  // barrier of the pipeline is waited for by one party, phase after phase
  // (a parity wait that runs a phase ahead of its barrier passes on the
  // wrong phase)
  static constexpr int NWG = ND;
  static constexpr int NB2 = cols(ND, 2) <= 512 ? 2 : 1;
  static constexpr int D1_OFF = 0;
  static constexpr int D2_OFF = ND * N1;
  static constexpr int TMEM_COLS = D2_OFF + 2 * NB2 * N2;
  static_assert(TMEM_COLS <= 512, "TMEM budget");
  static_assert(N1 % 16 == 0 && N1 <= 256, "GEMM1 N");
  static_assert(KD2 % 32 == 0, "GEMM2 K (FP8 MMAs reduce 32 entries)");
  static_assert(R % 16 == 0 && R <= 128, "rows are processed 16 at a time; magnitudes fit one 256-byte row");
  // coordinates per tensor-memory load: 32 (x16 packed loads) when they
  // divide the tile and the lines of 32 coordinates fit the rounding
  // thread's registers, else 16
  static constexpr int RC = (R % 32 == 0 && BKG * 16 <= 64) ? 32 : 16;
  // a warpgroup's tiles per accumulation period
  static constexpr int FLUSH = kTcPeriodCoords / R;
  // warps: NWG rounding warpgroups, the fold warpgroup, TMA, GEMM1, two GEMM2
  static constexpr int WARP_FOLD0 = 4 * NWG, WARP_TMA = WARP_FOLD0 + 4, WARP_G1 = WARP_TMA + 1,
                       WARP_G2 = WARP_G1 + 1;
  static constexpr int THREADS = 32 * (WARP_G2 + 2);
  // boundary line whose projections fill GEMM1 row block b
  static constexpr __host__ __device__ int line(int b) { return (K == 3 && b == 1) ? 2 : b; }
};

template <int K, int KCH>
struct TcLayout {
  using Sh = TcShape<K, KCH>;
  static constexpr int N2R = Sh::N2;                      // B2 rows (16 B each) per 16-entry K-chunk
  static constexpr int B2ROWS = Sh::KD2 / 16 * N2R;       // 16-byte rows of B2 per tile
  static constexpr int B1_BYTES = Sh::N1 * 16 * KCH;
  static constexpr int B2_BYTES = B2ROWS * 16;
  static constexpr int MAG_BYTES = 256;                   // R indicator-magnitude bytes, padded
  static_assert(B1_BYTES % 256 == 0 && B2_BYTES % 256 == 0, "tiles are whole 256-byte TMA rows");
  // one packed tile = GEMM1 rows | GEMM2 rows | magnitudes, contiguous: one TMA box
  static constexpr int B1_OFF_IN_STAGE = 0;
  static constexpr int B2_OFF_IN_STAGE = B1_BYTES;
  static constexpr int MAG_OFF_IN_STAGE = B1_BYTES + B2_BYTES;
  static constexpr int TILE_BYTES = B1_BYTES + B2_BYTES + MAG_BYTES;
  static_assert(TILE_BYTES / 256 <= 256, "TMA box height");
  static constexpr int STAGE_BYTES = TILE_BYTES;          // a multiple of 256: TMA destinations stay aligned
  static constexpr uint32_t STAGE_TX = TILE_BYTES;
  static constexpr int A1_BYTES = kTcM * 16 * KCH;
  // GEMM2's A operand per rounding warpgroup: 128 rows x KD2 E4M3 bytes,
  // K-major core matrices (chunk of 16 along K, then the 128 rows, 16 bytes each)
  static constexpr int A2S_BYTES = kTcM * Sh::KD2;
  static constexpr int ZERO_BYTES = 4096;
  static constexpr int NBARS = 2 * kTcMaxStages + 2 + 2 + 2 * 3 + 3 * kTcMaxNwg + 4 + 4 + 3;
  static constexpr int FIXED = 2 * A1_BYTES + Sh::NWG * A2S_BYTES + ZERO_BYTES + NBARS * 8 + 64 + 1024;
  // at least 120 KB of shared memory, so that two CTAs never share an SM
  // (each holds all 512 TMEM columns); the stage ring takes what is left of
  // 200 KB
  static constexpr int NS_FIT = (200 * 1024 - FIXED) / STAGE_BYTES;
  static constexpr int NS = NS_FIT < kTcMaxStages ? NS_FIT : kTcMaxStages;
  static_assert(NS >= 4, "pipeline depth");
  static constexpr int DIRS_OFF = NS * STAGE_BYTES;
  static constexpr int A2S_OFF = (DIRS_OFF + 2 * A1_BYTES + 1023) / 1024 * 1024;
  // the zero region lies above every operand: the descriptors' K-direction
  // byte offsets (LBO) to it are positive
  static constexpr int ZERO_OFF = A2S_OFF + Sh::NWG * A2S_BYTES;
  static constexpr int BAR_OFF = ZERO_OFF + ZERO_BYTES;
  static constexpr int USED = BAR_OFF + NBARS * 8 + 64;
  static constexpr int TOTAL = USED < 120 * 1024 ? 120 * 1024 : USED;
  static_assert(Sh::N1 * 16 <= ZERO_BYTES && kTcM * 16 <= ZERO_BYTES, "zero pad");
  static_assert(TOTAL <= 227 * 1024, "shared memory");
};

struct TcParams {
  int64_t n_tiles;
  int64_t c_tiles;
  int64_t tiles_per_chunk;
  int64_t num_items;
  int64_t S_pad;
  int r;
};

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Every lane of the warp polls and the warp agrees on the outcome.  A
// try_wait blocks in hardware for a while before it reports an incomplete
// phase (measured: faster here than a try_wait with a suspend-time hint).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const bool ok = ptx::mbar_wait(bar, parity, abort, kWaitLimit);
  return __all_sync(0xffffffffu, ok);
}

// Position in a ring of N slots: slot index and the parity of the current
// lap (the phase parity a wait for this slot's current use expects).
template <int N>
struct Ring {
  uint32_t idx = 0, ph = 0;
  __device__ __forceinline__ void next() {
    if (++idx == N) {
      idx = 0;
      ph ^= 1u;
    }
  }
  template <int D>
  __device__ __forceinline__ void step() {  // D slots on
    idx += D;
#pragma unroll
    for (int i = 0; i < (D + N - 1) / N; ++i) {
      if (idx >= N) {
        idx -= N;
        ph ^= 1u;
      }
    }
  }
  __device__ __forceinline__ void set(int64_t g) {  // the slot of use g
    idx = static_cast<uint32_t>(g % N);
    ph = static_cast<uint32_t>((g / N) & 1);
  }
};

// Two barriers: both polled at once first, so that the latencies of two
// complete phases overlap; `use2` false skips the second.
__device__ __forceinline__ bool warp_wait2(uint64_t* bar1, uint32_t par1, uint64_t* bar2, uint32_t par2, bool use2,
                                           volatile int* abort) {
  uint32_t both;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 q, [%3], %4;\n\t"
      "and.pred p, p, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(both)
      : "r"(ptx::smem_u32(bar1)), "r"(par1), "r"(ptx::smem_u32(use2 ? bar2 : bar1)), "r"(use2 ? par2 : par1)
      : "memory");
  if (__all_sync(0xffffffffu, both != 0)) return true;
  return warp_wait(bar1, par1, abort) && (!use2 || warp_wait(bar2, par2, abort));
}

// The tiles of an item (whose first tile is the CTA's tile g_base) that fall
// to member w of a round robin of M: j = j0, j0 + M, ... < ntile.
template <int M>
__device__ __forceinline__ int own_first(int64_t g_base, int w) {
  return static_cast<int>((w - static_cast<int>(g_base % M) + M) % M);
}

// The CTA's items are blockIdx.x, blockIdx.x + gridDim.x, ...; item it covers
// coordinate chunk it / c_tiles (tiles t0 .. t0 + ntile - 1) against candidate
// tile it % c_tiles.
struct TcItem {
  int64_t chunk, ct, t0;
  int ntile;
};

__device__ __forceinline__ TcItem tc_item(const TcParams& prm, int64_t it) {
  TcItem c;
  c.chunk = it / prm.c_tiles;
  c.ct = it - c.chunk * prm.c_tiles;
  c.t0 = c.chunk * prm.tiles_per_chunk;
  c.ntile = static_cast<int>(min(prm.n_tiles, c.t0 + prm.tiles_per_chunk) - c.t0);
  return c;
}

template <int K, int KCH>
__global__ void __maxnreg__(96)
    score_tc_kernel(const __grid_constant__ CUtensorMap tm_vt, const __grid_constant__ CUtensorMap tm_ct,
                    TcParams prm, const float* __restrict__ scale, double* __restrict__ partial,
                    int32_t* status) {
  using Sh = TcShape<K, KCH>;
  using L = TcLayout<K, KCH>;
  constexpr int R = Sh::R;
  constexpr int BK = Sh::BK;
  constexpr int BKG = Sh::BKG;
  constexpr int G = Sh::G;
  constexpr int ND = Sh::ND;
  constexpr int NS = L::NS;
  constexpr int NOUT = Sh::NOUT;
  constexpr int F = Sh::FLUSH;
  constexpr int CW = R / 4;  // indicator words per class per tile
  constexpr int RC = Sh::RC;
  constexpr int NWG = Sh::NWG;

  extern __shared__ __align__(1024) uint8_t smem[];
  // the warp index read through a shuffle from lane 0: the compiler then
  // knows it is the same on every lane, so each role's branch is warp-uniform
  // and the per-tile bookkeeping (ring positions, tile and item counters,
  // barrier and operand addresses) runs on the uniform datapath instead of
  // taking 32 lanes of the ALU pipe that the rounding needs
  const int warp = __shfl_sync(0xffffffffu, static_cast<int>(threadIdx.x >> 5), 0);
  const int lane = threadIdx.x & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* sfull = bars;                     // [NS]  stage landed (TMA)
  uint64_t* sempty = sfull + kTcMaxStages;    // [NS]  both GEMMs of the stage's tile done
  uint64_t* dfull = sempty + kTcMaxStages;    // [2]   direction buffer landed
  uint64_t* dempty = dfull + 2;               // [2]   every GEMM1 of the buffer's item done
  uint64_t* d1full = dempty + 2;              // [3]   D1 buffer holds its tile, stage landed (MMA + arrival)
  uint64_t* d1empty = d1full + 3;             // [3]   every rounding warp has loaded it (4 arrivals)
  // A2 buffer written (4 arrivals), one barrier per (warpgroup, GEMM2
  // stream): each is waited for by one stream, phase after phase
  uint64_t* a2full = d1empty + 3;             // [NWG][2]
  uint64_t* a2empty = a2full + 2 * kTcMaxNwg; // [NWG] GEMM2 that read it done
  uint64_t* d2full = a2empty + kTcMaxNwg;     // [2][2] accumulation period of stream v complete
  uint64_t* d2empty = d2full + 4;             // [2][2] folded (4 arrivals)
  uint64_t* drain = d2empty + 4;              // [3]   teardown of the GEMM2 / GEMM1 warps
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR_OFF + L::NBARS * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      ptx::mbar_init(&sfull[i], 1);
      ptx::mbar_init(&sempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&dfull[i], 1);
      ptx::mbar_init(&dempty[i], 1);
    }
    for (int i = 0; i < NWG; ++i) {
      ptx::mbar_init(&a2full[2 * i], 4);
      ptx::mbar_init(&a2full[2 * i + 1], 4);
      ptx::mbar_init(&a2empty[i], 1);
    }
    for (int i = 0; i < 4; ++i) {
      ptx::mbar_init(&d2full[i], 1);
      ptx::mbar_init(&d2empty[i], 4);
    }
    for (int i = 0; i < 3; ++i) ptx::mbar_init(&drain[i], 1);
    for (int i = 0; i < 3; ++i) {
      ptx::mbar_init(&d1full[i], 2);
      ptx::mbar_init(&d1empty[i], 4);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem + L::ZERO_OFF);
    for (int i = threadIdx.x; i < L::ZERO_BYTES / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  ptx::fence_proxy_async_smem();
  if (warp == Sh::WARP_TMA && lane == 0) {
    ptx::tma_prefetch_desc(&tm_vt);
    ptx::tma_prefetch_desc(&tm_ct);
  }
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t smem_base = ptx::smem_u32(smem);
  const int64_t grid = gridDim.x;
  const int64_t first_item = blockIdx.x;

  if (warp == Sh::WARP_TMA) {
    // ------------------------------------------------------------ TMA warp
    Ring<NS> st;
    int64_t loads = 0, dloads = 0;
    bool ok = true;
    for (int64_t it = first_item, k = 0; it < prm.num_items && ok; it += grid, ++k) {
      const TcItem c = tc_item(prm, it);
      const uint32_t b = static_cast<uint32_t>(k & 1);
      if (k >= 2) ok = warp_wait(&dempty[b], static_cast<uint32_t>(((k - 2) >> 1) & 1), abort_flag);
      if (!ok) break;
      if (lane == 0) {
        ptx::mbar_arrive_expect_tx(&dfull[b], L::A1_BYTES);
        ptx::tma_load_2d(smem + L::DIRS_OFF + b * L::A1_BYTES, &tm_ct, 0,
                         static_cast<int>(c.ct * (L::A1_BYTES / 256)), &dfull[b]);
      }
      ++dloads;
      for (int j = 0; j < c.ntile; ++j) {
        if (loads >= NS) ok = warp_wait(&sempty[st.idx], st.ph ^ 1u, abort_flag);
        if (!ok) break;
        if (lane == 0) {
          ptx::mbar_arrive_expect_tx(&sfull[st.idx], L::STAGE_TX);
          ptx::tma_load_2d(smem + st.idx * L::STAGE_BYTES, &tm_vt, 0,
                           static_cast<int>((c.t0 + j) * (L::TILE_BYTES / 256)), &sfull[st.idx]);
        }
        ++loads;
        st.next();
      }
    }
    if (!ok) *abort_flag = 1;
    // drain: the copies still in flight land before shared memory is released
    volatile int never = 0;
    for (int64_t t = loads > NS ? loads - NS : 0; t < loads; ++t)
      ptx::mbar_wait_sleep(&sfull[t % NS], static_cast<uint32_t>((t / NS) & 1), &never, kWaitLimit);
    for (int64_t t = dloads > 2 ? dloads - 2 : 0; t < dloads; ++t)
      ptx::mbar_wait_sleep(&dfull[t & 1], static_cast<uint32_t>((t >> 1) & 1), &never, kWaitLimit);
  } else if (warp == Sh::WARP_G1) {
    // ---------------------------------------------------------- GEMM1 warp
    constexpr uint32_t idesc1 = ptx::idesc_f16_f16(kTcM, Sh::N1);
    Ring<NS> st;
    Ring<ND> d1;
    int64_t g = 0;
    bool ok = true;
    for (int64_t it = first_item, k = 0; it < prm.num_items && ok; it += grid, ++k) {
      const TcItem c = tc_item(prm, it);
      const uint32_t b = static_cast<uint32_t>(k & 1);
      ok = warp_wait(&dfull[b], static_cast<uint32_t>((k >> 1) & 1), abort_flag);
      if (!ok) break;
      const uint32_t a1 = smem_base + L::DIRS_OFF + b * L::A1_BYTES;
      const uint32_t lbo_a1 = KCH == 2 ? kTcM * 16u : (smem_base + L::ZERO_OFF - a1);
      const uint64_t adesc = ptx::smem_desc(a1, lbo_a1, 128);
      for (int j = 0; j < c.ntile; ++j, ++g) {
        // the tile's stage has landed and its D1 buffer is free (both
        // barriers polled together: their latencies overlap)
        ok = warp_wait2(&sfull[st.idx], st.ph, &d1empty[d1.idx], d1.ph ^ 1u, g >= ND, abort_flag);
        if (!ok) break;
        // one arrival of the buffer's barrier (the MMA's commit is the
        // other): the rounding warps read the magnitudes from the stage
        if (lane == 0) ptx::mbar_arrive(&d1full[d1.idx]);
        ptx::tc_fence_after();
        const uint32_t b1 = smem_base + st.idx * L::STAGE_BYTES + L::B1_OFF_IN_STAGE;
        const uint32_t lbo_b1 = KCH == 2 ? Sh::N1 * 16u : (smem_base + L::ZERO_OFF - b1);
        ptx::mma_f16_ss_commit(tmem + Sh::D1_OFF + d1.idx * Sh::N1, adesc, ptx::smem_desc(b1, lbo_b1, 128), idesc1,
                               &d1full[d1.idx]);
        st.next();
        d1.next();
      }
      if (!ok) break;
      ptx::mma_commit_elect(&dempty[b]);
    }
    if (!ok) *abort_flag = 1;
    volatile int never = 0;
    ptx::mma_commit_elect(&drain[2]);
    warp_wait(&drain[2], 0u, &never);
  } else if (warp == Sh::WARP_G2 || warp == Sh::WARP_G2 + 1) {
    // ---------------------------------------------------------- GEMM2 warps
    const int v = warp - Sh::WARP_G2;  // stream: the tiles g with g % 2 == v
    constexpr int NB2 = Sh::NB2;
    constexpr uint32_t idesc2 = ptx::idesc_e4m3_f32(kTcM, Sh::N2);
    constexpr uint32_t lbo_b2 = L::N2R * 16;
    const uint32_t d2 = tmem + Sh::D2_OFF + v * NB2 * Sh::N2;
    Ring<NS> st;
    // tile g's warpgroup is g % NWG and its A2-full barrier [g % NWG][v]
    // completes once per lcm(NWG, 2) tiles: a ring of that length gives both
    constexpr int LCM = NWG % 2 == 0 ? NWG : 2 * NWG;
    Ring<LCM> a2;
    int64_t g_base = 0, p = 0;  // the CTA's first tile of the item; this stream's periods
    bool ok = true;
    for (int64_t it = first_item; it < prm.num_items && ok; it += grid) {
      const TcItem c = tc_item(prm, it);
      int j = own_first<2>(g_base, v);
      st.set(g_base + j);
      a2.set(g_base + j);
      int pos = 0;
      for (; j < c.ntile; j += 2, st.template step<2>(), a2.template step<2>()) {
        const bool first = pos == 0;
        const bool last = (pos == F - 1) || (j + 2 >= c.ntile);
        const uint32_t pb = static_cast<uint32_t>(p % NB2);
        if (first && p >= NB2)
          ok = warp_wait(&d2empty[v * 2 + pb], static_cast<uint32_t>(((p / NB2) - 1) & 1), abort_flag);
        const uint32_t w = a2.idx % NWG;
        if (ok) ok = warp_wait(&a2full[2 * w + v], a2.ph, abort_flag);
        if (!ok) break;
        ptx::tc_fence_after();
        const uint32_t b2 = smem_base + st.idx * L::STAGE_BYTES + L::B2_OFF_IN_STAGE;
        // A2 of warpgroup w in shared memory: K chunks of 16 bytes, 128 rows each
        const uint32_t a2s = smem_base + L::A2S_OFF + w * L::A2S_BYTES;
        if constexpr (Sh::KD2 / 32 == 5) {
          uint64_t da[5], db[5];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            da[q] = ptx::smem_desc(a2s + q * 2 * kTcM * 16, kTcM * 16, 128);
            db[q] = ptx::smem_desc(b2 + q * 2 * lbo_b2, lbo_b2, 128);
          }
          ptx::mma_e4m3_ss_x5_commit(d2 + pb * Sh::N2, da, db, idesc2, first ? 0u : 1u, &a2empty[w], &sempty[st.idx],
                                     &d2full[v * 2 + pb], last ? 1u : 0u);
        } else {
#pragma unroll
          for (int q = 0; q < Sh::KD2 / 32; ++q)
            ptx::mma_e4m3_ss_elect(d2 + pb * Sh::N2, ptx::smem_desc(a2s + q * 2 * kTcM * 16, kTcM * 16, 128),
                                   ptx::smem_desc(b2 + q * 2 * lbo_b2, lbo_b2, 128), idesc2,
                                   (q > 0 || !first) ? 1u : 0u);
          ptx::mma_commit_elect(&a2empty[w]);
          ptx::mma_commit_elect(&sempty[st.idx]);
          if (last) ptx::mma_commit_elect(&d2full[v * 2 + pb]);
        }
        if (last) {
          ++p;
          pos = 0;
        } else {
          ++pos;
        }
      }
      g_base += c.ntile;
    }
    if (!ok) *abort_flag = 1;
    volatile int never = 0;
    ptx::mma_commit_elect(&drain[v]);
    warp_wait(&drain[v], 0u, &never);
  } else if (warp >= Sh::WARP_FOLD0) {
    // --------------------------------------------------------- fold warpgroup
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    const float inv_s = scale[1];
    const int r2 = 2 * prm.r;
    float hi[NOUT], lo[NOUT];
#pragma unroll
    for (int jj = 0; jj < NOUT; ++jj) hi[jj] = lo[jj] = 0.f;
    constexpr int NB2 = Sh::NB2;
    int64_t g_base = 0;
    int64_t pw[2] = {0, 0};  // periods folded per stream
    bool ok = true;
    for (int64_t it = first_item; it < prm.num_items && ok; it += grid) {
      const TcItem c = tc_item(prm, it);
      // the item's periods per stream: its tiles, F at a time
      int nper[2];
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int own = (c.ntile - own_first<2>(g_base, w) + 1) / 2;
        nper[w] = (own + F - 1) / F;
      }
      const int imax = nper[0] > nper[1] ? nper[0] : nper[1];
      for (int i = 0; i < imax && ok; ++i) {
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          if (i >= nper[w] || !ok) continue;
          const uint32_t pb = static_cast<uint32_t>(pw[w] % NB2);
          ok = warp_wait(&d2full[2 * w + pb], static_cast<uint32_t>((pw[w] / NB2) & 1), abort_flag);
          if (!ok) break;
          ptx::tc_fence_after();
          uint32_t dh[NOUT], dl[NOUT];
          const uint32_t ta = tmem + lane_base + Sh::D2_OFF + (w * NB2 + pb) * Sh::N2;
          if constexpr (NOUT == 8) {
            uint32_t v[16];
            ptx::tmem_ld_x16(ta, v);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              dh[jj] = v[jj];
              dl[jj] = v[8 + jj];
            }
          } else {
            ptx::tmem_ld_x16(ta, dh);
            ptx::tmem_ld_x16(ta + 16, dl);
            ptx::tmem_wait_ld();
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&d2empty[2 * w + pb]);
          ++pw[w];
#pragma unroll
          for (int jj = 0; jj < NOUT; ++jj) {
            float s, er;
            two_sum_f(hi[jj], __uint_as_float(dh[jj]), s, er);
            hi[jj] = s;
            lo[jj] += er;
            two_sum_f(hi[jj], __uint_as_float(dl[jj]), s, er);
            hi[jj] = s;
            lo[jj] += er;
          }
        }
      }
      if (!ok) break;
      // the item's chunk partial sums
      double* out = partial + (c.chunk * prm.S_pad + c.ct * kTcM + row) * r2;
#pragma unroll
      for (int jj = 0; jj < NOUT; ++jj) {
        if (jj < r2) out[jj] = (static_cast<double>(hi[jj]) + static_cast<double>(lo[jj])) * static_cast<double>(inv_s);
        hi[jj] = lo[jj] = 0.f;
      }
      g_base += c.ntile;
    }
    if (!ok) *abort_flag = 1;
  } else if (warp < 4 * NWG) {
    // ----------------------------------------------------- rounding warpgroups
    const int wg = warp >> 2;
    const int q = warp & 3;
    const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
    // this warpgroup's A2 in shared memory; thread row q * 32 + lane
    uint8_t* const a2s_row = smem + L::A2S_OFF + wg * L::A2S_BYTES + (q * 32 + lane) * 16;
    constexpr int NCH = R / RC;
    Ring<ND> d1;
    Ring<NS> st;
    uint32_t a2ph = 0;  // parity of this warpgroup's A2 buffer uses
    int64_t g_base = 0;
    bool ok = true;
    for (int64_t it = first_item; it < prm.num_items && ok; it += grid) {
      const TcItem c = tc_item(prm, it);
      int j = own_first<NWG>(g_base, wg);
      d1.set(g_base + j);
      st.set(g_base + j);
      for (; j < c.ntile; j += NWG, d1.template step<NWG>(), st.template step<NWG>()) {
        const int64_t g = g_base + j;
        // D1 of tile g; its completion also says that the tile's stage has
        // landed (the GEMM1 warp saw the stage's barrier before arriving)
        ok = warp_wait(&d1full[d1.idx], d1.ph, abort_flag);
        if (!ok) break;
        ptx::tc_fence_after();
        const uint32_t* const magp =
            reinterpret_cast<const uint32_t*>(smem + st.idx * L::STAGE_BYTES + L::MAG_OFF_IN_STAGE);
        const uint32_t d1_tmem = tmem + lane_base + Sh::D1_OFF + d1.idx * Sh::N1;
        uint32_t wv[G * CW];
        // D1 holds F16 projections, one per column; a packed load gives two
        // coordinates per register, so one byte permute gathers the signs of
        // four coordinates
        // chunk ch + 1 is loaded while chunk ch is rounded (two register sets)
        uint32_t pl2[2][BKG][RC / 2];
        auto load_chunk = [&](int ch, uint32_t (&dst)[BKG][RC / 2]) {
#pragma unroll
          for (int b = 0; b < BKG; ++b) {
            const uint32_t ta = d1_tmem + b * R + ch * RC;
            if constexpr (RC == 32)
              ptx::tmem_ld_x16_pack16(ta, *reinterpret_cast<uint32_t(*)[16]>(dst[b]));
            else
              ptx::tmem_ld_x8_pack16(ta, *reinterpret_cast<uint32_t(*)[8]>(dst[b]));
          }
        };
        // after tcgen05.wait::ld: the registers a load wrote are tied to the
        // wait, so no use of them is scheduled above it
        auto loaded = [&](uint32_t (&dst)[BKG][RC / 2]) {
          ptx::tmem_wait_ld();
#pragma unroll
          for (int b = 0; b < BKG; ++b)
#pragma unroll
            for (int i = 0; i < RC / 2; ++i) asm volatile("" : "+r"(dst[b][i]));
        };
        auto release_d1 = [&]() {
          // every projection of the tile is in registers: release D1
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&d1empty[d1.idx]);
        };
        load_chunk(0, pl2[0]);
        loaded(pl2[0]);
        if (NCH == 1) release_d1();
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          uint32_t (&pl)[BKG][RC / 2] = pl2[ch & 1];
          if (ch + 1 < NCH) load_chunk(ch + 1, pl2[(ch + 1) & 1]);
          uint32_t mag[RC / 4];
#pragma unroll
          for (int v4 = 0; v4 < RC / 16; ++v4) {
            const uint4 m4 = reinterpret_cast<const uint4*>(magp + ch * (RC / 4))[v4];
            mag[4 * v4] = m4.x;
            mag[4 * v4 + 1] = m4.y;
            mag[4 * v4 + 2] = m4.z;
            mag[4 * v4 + 3] = m4.w;
          }
#pragma unroll
          for (int pq = 0; pq < RC / 4; ++pq) {
            uint32_t nm[BK];
            if constexpr (K == 3) {
              // p_1 = -(p_0 + p_2): the three boundary directions sum to zero, so
              // p_1 < 0 exactly where p_0 + p_2 > 0
              const uint32_t sum_neg = ptx::prmt(ptx::hadd2(pl[0][2 * pq], pl[1][2 * pq]),
                                                 ptx::hadd2(pl[0][2 * pq + 1], pl[1][2 * pq + 1]), 0xFDB9u);
              nm[0] = ptx::prmt(pl[0][2 * pq], pl[0][2 * pq + 1], 0xFDB9u);
              nm[1] = ~sum_neg;
              nm[2] = ptx::prmt(pl[1][2 * pq], pl[1][2 * pq + 1], 0xFDB9u);
            } else {
#pragma unroll
              for (int m = 0; m < BK; ++m) nm[m] = ptx::prmt(pl[m][2 * pq], pl[m][2 * pq + 1], 0xFDB9u);
            }
            const int wi = ch * (RC / 4) + pq;
#pragma unroll
            for (int gc = 0; gc < G; ++gc) {
              if constexpr (K % 2 == 1)
                wv[gc * CW + wi] = ~nm[gc] & nm[gc + 1] & mag[pq];  // p_{k-1} > 0 and p_k < 0
              else
                wv[gc * CW + wi] = (nm[gc] & 0x80808080u) | mag[pq];  // sign(p_m) as +-1
            }
          }
          if (ch + 1 < NCH) {
            loaded(pl2[(ch + 1) & 1]);
            if (ch + 1 == NCH - 1) release_d1();
          }
        }
        // the GEMM2 that read this warpgroup's A2 buffer last (its previous tile) is done
        if (g >= NWG) ok = warp_wait(&a2empty[wg], a2ph ^ 1u, abort_flag);
        if (!ok) break;
        ptx::tc_fence_after();
        // words w .. w + 3 of a class (16 coordinates) are one 16-byte chunk of
        // the row; chunk c of all 128 rows lies at c * 128 * 16
#pragma unroll
        for (int cc = 0; cc < Sh::A2WORDS / 4; ++cc)
          *reinterpret_cast<uint4*>(a2s_row + cc * kTcM * 16) =
              make_uint4(wv[4 * cc], wv[4 * cc + 1], wv[4 * cc + 2], wv[4 * cc + 3]);
        // the stores, visible to the tensor core's operand reads
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&a2full[2 * wg + (g & 1)]);
        a2ph ^= 1u;
      }
      g_base += c.ntile;
    }
    if (!ok) *abort_flag = 1;
  }
  // ------------------------------------------------------------ teardown
  if (threadIdx.x == 0) {
    __threadfence_block();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) dev_fail(status, LRQ_ETIMEOUT);
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// Operand packing (run once per call): tiles in the exact shared-memory order
// the MMA descriptors expect, so each stage is one TMA box.
// ---------------------------------------------------------------------------
struct PackTables {
  float bcos[8], bsin[8];    // boundary directions theta_m, m < B_K
  float beta_r[8], beta_i[8];  // per-indicator coefficients
};

// augmented rows: tile t, chunk ch, row (b*ROWS + i) for boundary line
// line(b), 8 slots
template <int K, int KCH>
__global__ void pack_vaug_kernel(const float2* __restrict__ V, int64_t n, int r, int64_t n_tiles, PackTables tb,
                                 uint8_t* __restrict__ tiles) {
  using Sh = TcShape<K, KCH>;
  using L = TcLayout<K, KCH>;
  const int64_t total = n_tiles * Sh::N1;
  int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int64_t t = q / Sh::N1;
  const int rowin = static_cast<int>(q % Sh::N1);
  const int m = Sh::line(rowin / Sh::ROWS), i = rowin % Sh::ROWS;
  const int64_t ig = t * Sh::ROWS + i;
  float slot[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) slot[k] = 0.f;
  if (ig < n) {
    // a row's signs do not change under a positive scale: a power of two
    // brings its largest component into [1, 2), so every product and the F16
    // accumulator stay far inside the F16 range and keep its precision
    float mx = 0.f;
    for (int jj = 0; jj < r; ++jj) {
      const float2 v = V[ig * r + jj];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    const int sh = (mx > 0.f && isfinite(mx)) ? -ilogbf(mx) : 0;
    const float bc = tb.bcos[m], bs = tb.bsin[m];
    for (int jj = 0; jj < r; ++jj) {
      const float2 v = V[ig * r + jj];
      // rho_m V = (bc - i bs)(vr + i vi)
      slot[jj] = ldexpf(fmaf(bc, v.y, -bs * v.x), sh);     // Im(rho_m V_ij)
      slot[r + jj] = ldexpf(fmaf(bc, v.x, bs * v.y), sh);  // Re(rho_m V_ij)
    }
  }
#pragma unroll
  for (int ch = 0; ch < KCH; ++ch) {
    __align__(16) __half h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = __float2half_rn(slot[ch * 8 + k]);
    *reinterpret_cast<uint4*>(tiles + t * L::TILE_BYTES + (ch * Sh::N1 + rowin) * 16) = *reinterpret_cast<uint4*>(h);
  }
}

// Scales of the GEMM2 operands.  B2 entries are components of
// beta conj(V_i) with |beta| <= 2, so |B2| < 3 m_i, m_i = max |V_i component|.
// Coordinate i is scaled by 2^e_i, e_i = 5 - ilogb(m_i), which moves m_i into
// [32, 64) and its entries below 192 (E4M3 reaches 448): every coordinate
// keeps the full hi + lo precision however small its row.
// Its indicator carries the inverse, 2^(g - e_i), so each product is the
// entry times 2^g, one global power of two (g = 5 - ilogb(max_i m_i)) that the
// epilogue removes.  2^(g - e_i) must be an E4M3 number (down to 2^-9), so
// e_i <= g + 9: rows more than 2^9 below the largest lose relative precision
// (their share of the sums is as small).  scale = {2^g, 2^-g, max m_i bits}.
__global__ void b2_amax_kernel(const float2* __restrict__ V, int64_t count, float* __restrict__ scale) {
  float m = 0.f;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < count;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float2 v = V[q];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative floats order like their bit patterns
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(reinterpret_cast<unsigned*>(scale + 2), __float_as_uint(m));
}

__device__ __forceinline__ int b2_global_exp(const float* scale) {
  const float a = scale[2];
  return 5 - ((a > 0.f && isfinite(a)) ? ilogbf(a) : 5);
}

__global__ void b2_scale_kernel(float* scale) {
  if (threadIdx.x != 0) return;
  const int g = b2_global_exp(scale);
  scale[0] = ldexpf(1.f, g);
  scale[1] = ldexpf(1.f, -g);
}

// e_i of coordinate ig (see above); g for a zero row
__device__ __forceinline__ int b2_coord_exp(const float2* __restrict__ V, int64_t ig, int r, int g) {
  float m = 0.f;
  for (int jj = 0; jj < r; ++jj) {
    const float2 v = V[ig * r + jj];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  const int e = (m > 0.f && isfinite(m)) ? 5 - ilogbf(m) : g;
  return e < g ? g : (e > g + 9 ? g + 9 : e);
}

// GEMM2 B rows (FP8 E4M3): tile t, K-chunk kc (16 reduction entries), row nr:
// output column nr (hi part) for nr < NOUT, output column nr - NOUT (lo part,
// the rounding remainder of hi) above
// e_i from the coordinate's indicator magnitude byte 2^(g - e_i) (written by
// pack_indicator_scale_kernel, below): d = g - e_i in [-9, 0]
__device__ __forceinline__ int b2_exp_from_code(uint32_t code, int g) {
  const int d = code >= 8u ? static_cast<int>(code >> 3) - 7 : (code == 4u ? -7 : (code == 2u ? -8 : -9));
  return g - d;
}

template <int K, int KCH>
__global__ void pack_b2_kernel(const float2* __restrict__ V, int64_t n, int r, int64_t n_tiles, PackTables tb,
                               const float* __restrict__ scale, const uint8_t* __restrict__ iwb,
                               uint8_t* __restrict__ tiles) {
  using Sh = TcShape<K, KCH>;
  using L = TcLayout<K, KCH>;
  const int64_t total = n_tiles * L::B2ROWS;
  int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int64_t t = q / L::B2ROWS;
  const int within = static_cast<int>(q % L::B2ROWS);
  const int kc = within / L::N2R, nr = within % L::N2R;
  const bool lo = nr >= Sh::NOUT;
  const int nc = lo ? nr - Sh::NOUT : nr;
  const int g = b2_global_exp(scale);
  __align__(16) uint8_t h[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int kk = kc * 16 + k;
    const int gc = kk / Sh::ROWS, i = kk % Sh::ROWS;
    const int64_t ig = t * Sh::ROWS + i;
    const int jj = nc >> 1;
    float val = 0.f;
    if (ig < n && jj < r) {
      float2 v = V[ig * r + jj];
      const float br = tb.beta_r[gc], bi = tb.beta_i[gc];
      // beta conj(V) = (br vr + bi vi) + i (bi vr - br vi)
      val = ldexpf((nc & 1) ? fmaf(bi, v.x, -br * v.y) : fmaf(br, v.x, bi * v.y), b2_exp_from_code(iwb[ig], g));
    }
    const __nv_fp8_e4m3 hi(val);
    h[k] = lo ? __nv_fp8_e4m3(val - static_cast<float>(hi)).__x : hi.__x;
  }
  *reinterpret_cast<uint4*>(tiles + t * L::TILE_BYTES + L::B2_OFF_IN_STAGE + within * 16) =
      *reinterpret_cast<uint4*>(h);
}

// Indicator magnitudes 2^(g - e_i) as E4M3 bytes, four coordinates per word
// (lowest coordinate in the lowest byte), R / 4 words per tile; 0 past n.
// Written twice: into `iw` (read back by the GEMM2 row packing) and into the
// magnitude row of each packed tile (read by the scoring kernel's rounding
// threads from the tile's stage).
template <int K, int KCH>
__global__ void pack_indicator_scale_kernel(const float2* __restrict__ V, int64_t n, int r, int64_t words,
                                            const float* __restrict__ scale, uint32_t* __restrict__ iw,
                                            uint8_t* __restrict__ tiles) {
  using Sh = TcShape<K, KCH>;
  using L = TcLayout<K, KCH>;
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= words) return;
  const int g = b2_global_exp(scale);
  uint32_t w = 0;
  for (int c = 0; c < 4; ++c) {
    const int64_t ig = q * 4 + c;
    if (ig >= n) continue;
    const int d = g - b2_coord_exp(V, ig, r, g);  // in [-9, 0]
    // E4M3 2^d: normal ((d + 7) << 3) down to 2^-6, subnormal 0x4 >> (-7 - d) below
    const uint32_t code = d >= -6 ? static_cast<uint32_t>(d + 7) << 3 : (0x4u >> (-7 - d));
    w |= code << (8 * c);
  }
  iw[q] = w;
  const int64_t t = q / (Sh::ROWS / 4);
  const int wi = static_cast<int>(q % (Sh::ROWS / 4));
  *reinterpret_cast<uint32_t*>(tiles + t * L::TILE_BYTES + L::MAG_OFF_IN_STAGE + 4 * wi) = w;
}

// directions: candidate tile ct, chunk ch, row s: slots [Re c, Im c, 0...]
template <int KCH>
__global__ void pack_dirs_kernel(const float2* __restrict__ C, int64_t S, int r, int64_t c_tiles,
                                 __half* __restrict__ ctp) {
  const int64_t total = c_tiles * kTcM;
  int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int64_t ct = q / kTcM;
  const int row = static_cast<int>(q % kTcM);
  float slot[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) slot[k] = 0.f;
  if (q < S) {
    // a positive power-of-two scale (the largest component into [1, 2))
    // changes no decision and keeps the F16 products in range
    float mx = 0.f;
    for (int jj = 0; jj < r; ++jj) {
      const float2 c = C[q * r + jj];
      mx = fmaxf(mx, fmaxf(fabsf(c.x), fabsf(c.y)));
    }
    const int sh = (mx > 0.f && isfinite(mx)) ? -ilogbf(mx) : 0;
    for (int jj = 0; jj < r; ++jj) {
      const float2 c = C[q * r + jj];
      slot[jj] = ldexpf(c.x, sh);
      slot[r + jj] = ldexpf(c.y, sh);
    }
  }
#pragma unroll
  for (int ch = 0; ch < KCH; ++ch) {
    __align__(16) __half h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = __float2half_rn(slot[ch * 8 + k]);
    *reinterpret_cast<uint4*>(ctp + ((ct * KCH + ch) * kTcM + row) * 8) = *reinterpret_cast<uint4*>(h);
  }
}

static PackTables make_pack_tables(const Alphabet& a) {
  PackTables tb;
  for (int m = 0; m < 8; ++m) {
    tb.bcos[m] = m < a.BK ? a.bcos[m] : 0.f;
    tb.bsin[m] = m < a.BK ? a.bsin[m] : 0.f;
    tb.beta_r[m] = m < a.G ? static_cast<float>(a.beta_r[m]) : 0.f;
    tb.beta_i[m] = m < a.G ? static_cast<float>(a.beta_i[m]) : 0.f;
  }
  return tb;
}

// The instance's operands (depend on V only): augmented rows, the GEMM2
// scale, the per-coordinate indicator magnitudes and the class rows.
template <int K, int KCH>
static int pack_v_impl(const ScorePlan& p, const Alphabet& a, const float2* V, void* tiles, float* scale,
                       uint32_t* iw, cudaStream_t st) {
  using Sh = TcShape<K, KCH>;
  using L = TcLayout<K, KCH>;
  PackTables tb = make_pack_tables(a);
  int64_t nv = p.n_tiles * Sh::N1;
  pack_vaug_kernel<K, KCH><<<static_cast<unsigned>(ceil_div(nv, 256)), 256, 0, st>>>(
      V, p.n, p.r, p.n_tiles, tb, static_cast<uint8_t*>(tiles));
  count_launch();
  int e = cuda_check(cudaMemsetAsync(scale + 2, 0, sizeof(float), st), "cudaMemsetAsync(scale)");
  if (e) return e;
  const int64_t nvr = p.n * p.r;
  b2_amax_kernel<<<static_cast<unsigned>(std::min<int64_t>(ceil_div(nvr, 256), 152 * 8)), 256, 0, st>>>(V, nvr,
                                                                                                           scale);
  b2_scale_kernel<<<1, 32, 0, st>>>(scale);
  count_launch(2);
  // the per-coordinate exponents first: the GEMM2 rows read them back
  const int64_t words = p.n_tiles * (Sh::ROWS / 4);
  pack_indicator_scale_kernel<K, KCH><<<static_cast<unsigned>(ceil_div(words, 256)), 256, 0, st>>>(
      V, p.n, p.r, words, scale, iw, static_cast<uint8_t*>(tiles));
  int64_t nb = p.n_tiles * L::B2ROWS;
  pack_b2_kernel<K, KCH><<<static_cast<unsigned>(ceil_div(nb, 256)), 256, 0, st>>>(
      V, p.n, p.r, p.n_tiles, tb, scale, reinterpret_cast<const uint8_t*>(iw), static_cast<uint8_t*>(tiles));
  count_launch(2);
  return cuda_check(cudaGetLastError(), "tc operand packing");
}

// The directions (depend on C only).
template <int KCH>
static int pack_dirs_impl(const ScorePlan& p, const float2* C, void* ct, cudaStream_t st) {
  int64_t nc = p.c_tiles * kTcM;
  pack_dirs_kernel<KCH><<<static_cast<unsigned>(ceil_div(nc, 256)), 256, 0, st>>>(C, p.S, p.r, p.c_tiles,
                                                                                  static_cast<__half*>(ct));
  count_launch();
  return cuda_check(cudaGetLastError(), "pack_dirs_kernel");
}

// ---------------------------------------------------------------------------
// Tensor maps: every packed operand is viewed as a 2-D bf16 array of 16-byte
// rows ([rows][8]); a box of `box_rows` rows lands in shared memory exactly in
// the no-swizzle core-matrix order.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Every packed operand tile is a contiguous byte range whose size is a
// multiple of 256 bytes, so the buffer is viewed as rows of 128 bf16 (256 B)
// and one box of (tile bytes / 256) rows copies a whole tile.  Wide rows keep
// the TMA requests at full 32-byte-sector efficiency.
static int make_rows_map(CUtensorMap* map, const void* base, size_t total_bytes, int tile_bytes) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) return fail(LRQ_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if (total_bytes % 256 != 0 || tile_bytes % 256 != 0 || tile_bytes / 256 > 256)
    return fail(LRQ_EUNSUPPORTED, "packed operand tile is not a whole number of 256-byte rows");
  cuuint64_t dims[2] = {128, static_cast<cuuint64_t>(total_bytes / 256)};
  cuuint64_t strides[1] = {256};
  cuuint32_t box[2] = {128, static_cast<cuuint32_t>(tile_bytes / 256)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(LRQ_ECUDA, "cuTensorMapEncodeTiled failed");
  return LRQ_OK;
}

template <int K, int KCH>
static int score_impl(const ScorePlan& p, const void* tiles, const void* ct, const float* scale, double* partial,
                      int32_t* status, cudaStream_t st) {
  using L = TcLayout<K, KCH>;
  CUtensorMap m_vt, m_ct;
  int e;
  if ((e = make_rows_map(&m_vt, tiles, static_cast<size_t>(p.n_tiles) * L::TILE_BYTES, L::TILE_BYTES))) return e;
  if ((e = make_rows_map(&m_ct, ct, static_cast<size_t>(p.c_tiles) * L::A1_BYTES, L::A1_BYTES))) return e;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, []() {
    attr_err = cudaFuncSetAttribute(score_tc_kernel<K, KCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
  });
  if ((e = cuda_check(attr_err, "cudaFuncSetAttribute(score_tc_kernel)"))) return e;
  TcParams prm;
  prm.n_tiles = p.n_tiles;
  prm.c_tiles = p.c_tiles;
  prm.tiles_per_chunk = p.tiles_per_chunk;
  prm.num_items = p.c_tiles * p.nsplit;
  prm.S_pad = p.c_tiles * kTcM;
  prm.r = p.r;
  int grid = static_cast<int>(std::min<int64_t>(prm.num_items, num_sms_current()));
  score_tc_kernel<K, KCH><<<grid, TcShape<K, KCH>::THREADS, L::TOTAL, st>>>(m_vt, m_ct, prm, scale, partial, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "score_tc_kernel");
}

#define LRQ_TC_SHAPE_SWITCH(EXPR)                                  \
  do {                                                             \
    switch (K) {                                                   \
      case 2: return two ? EXPR(2, 2) : EXPR(2, 1);                \
      case 3: return two ? EXPR(3, 2) : EXPR(3, 1);                \
      case 4: return two ? EXPR(4, 2) : EXPR(4, 1);                \
      case 5: return two ? EXPR(5, 2) : EXPR(5, 1);                \
      case 6: return two ? EXPR(6, 2) : EXPR(6, 1);                \
      case 7: return two ? EXPR(7, 2) : EXPR(7, 1);                \
      case 8: return two ? EXPR(8, 2) : EXPR(8, 1);                \
      default: return 0;                                           \
    }                                                              \
  } while (0)

int tc_rows_per_tile(int K, int r) {
  const bool two = r > 4;
#define LRQ_ROWS(k, c) TcShape<k, c>::ROWS
  LRQ_TC_SHAPE_SWITCH(LRQ_ROWS);
#undef LRQ_ROWS
}

int tc_workers_per_cta(int K, int r) {
  (void)K;
  (void)r;
  return 1;  // one pipeline per CTA
}

size_t tc_bytes_tiles(int K, int r, int64_t n_tiles) {
  const bool two = r > 4;
#define LRQ_TILE(k, c) static_cast<size_t>(n_tiles) * TcLayout<k, c>::TILE_BYTES
  LRQ_TC_SHAPE_SWITCH(LRQ_TILE);
#undef LRQ_TILE
}

size_t tc_bytes_indicator_scale(int K, int r, int64_t n_tiles) {
  return static_cast<size_t>(n_tiles) * static_cast<size_t>(tc_rows_per_tile(K, r));  // one byte per coordinate
}

size_t tc_bytes_dirs(int r, int64_t c_tiles) {
  int kch = r <= 4 ? 1 : 2;
  return static_cast<size_t>(c_tiles) * kch * kTcM * 16;
}

#define LRQ_TC_DISPATCH(FN, ...)                                        \
  do {                                                                  \
    const bool two = p.r > 4;                                           \
    switch (p.K) {                                                      \
      case 2: return two ? FN<2, 2>(__VA_ARGS__) : FN<2, 1>(__VA_ARGS__); \
      case 3: return two ? FN<3, 2>(__VA_ARGS__) : FN<3, 1>(__VA_ARGS__); \
      case 4: return two ? FN<4, 2>(__VA_ARGS__) : FN<4, 1>(__VA_ARGS__); \
      case 5: return two ? FN<5, 2>(__VA_ARGS__) : FN<5, 1>(__VA_ARGS__); \
      case 6: return two ? FN<6, 2>(__VA_ARGS__) : FN<6, 1>(__VA_ARGS__); \
      case 7: return two ? FN<7, 2>(__VA_ARGS__) : FN<7, 1>(__VA_ARGS__); \
      case 8: return two ? FN<8, 2>(__VA_ARGS__) : FN<8, 1>(__VA_ARGS__); \
      default: return fail(LRQ_EUNSUPPORTED, "tensor-core path supports 2 <= K <= 8"); \
    }                                                                   \
  } while (0)

int launch_tc_pack_v(const ScorePlan& p, const Alphabet& a, const float2* V, void* tiles, void* scale, void* iw,
                     cudaStream_t st) {
  LRQ_TC_DISPATCH(pack_v_impl, p, a, V, tiles, static_cast<float*>(scale), static_cast<uint32_t*>(iw), st);
}

int launch_tc_pack_dirs(const ScorePlan& p, const float2* C, void* ct, cudaStream_t st) {
  return p.r > 4 ? pack_dirs_impl<2>(p, C, ct, st) : pack_dirs_impl<1>(p, C, ct, st);
}

int launch_score_tc(const ScorePlan& p, const Alphabet& a, const void* tiles, const void* ct, const void* scale,
                    const void* iw, double* partial, int32_t* status, cudaStream_t st) {
  (void)a;
  (void)iw;  // the magnitudes travel inside the packed tiles
  LRQ_TC_DISPATCH(score_impl, p, tiles, ct, static_cast<const float*>(scale), partial, status, st);
}

}  // namespace lrq
