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
// half the MMA instructions (N is the problem's 2r outputs, so the MMAs are
// small and the kernel is bounded by each worker's per-tile chain of waits,
// issues and rounding, not by arithmetic).  D2 accumulates in TMEM (FP32) for
// at most `flush` tiles, then is folded into FP32 two-sum registers
// (error-free) and written as FP64 partials per coordinate chunk.
//
// Pipeline (one CTA per SM, persistent over (chunk, candidate tile) items):
// NW independent workers per CTA, each a warpgroup (one thread per candidate
// of the 128-candidate tile) with its own stage ring and TMEM slice (D1
// projections, A2 indicator words, D2 accumulator).  Per tile, after the
// warpgroup has turned D1 into indicator words in A2 and met at a barrier,
// its warp 0 issues GEMM1 of the next tile and its warp 2 GEMM2 of this one,
// each from the whole converged warp through one elected lane (measured:
// about a third of the cost of issuing from a lone active lane).  Separate
// commits (D1 ready; A2 free) let the two run side by side; the rounding
// threads wait for "A2 free" only just before they overwrite A2.  One lane of
// warp 1 keeps the stage ring full: a stage is free once both GEMMs of its
// tile are known complete; each packed tile -- GEMM1 rows and GEMM2 rows -- is
// one TMA box.  The workers of a CTA interleave on the tensor core.  Every
// wait is bounded; on expiry the kernel records LRQ_ETIMEOUT, drains its
// in-flight copies and MMAs, frees TMEM and returns.
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
constexpr int kTcStages = 8;
constexpr int kTcFlush = 64;
constexpr long long kWaitLimit = 2000000000LL;

// Tile shape per alphabet and rank class (KCH = 1 for r <= 4, 2 above).  A
// CTA runs NW independent workers; each worker is one warpgroup (128
// threads, one per candidate of the tile) and owns a TMEM slice of WCOLS
// columns:
//   D1 : N1 = BKG * R columns    GEMM1 projections of one tile
//   A2 : KD2 / 4 columns         GEMM2 indicator operand (4 FP8 per column)
//   D2 : N2 = 2 * NOUT columns   GEMM2 accumulator, hi | lo
// NW * WCOLS <= 512.  R is the number of coordinates per tile.
template <int K, int KCH>
struct TcShape {
  static constexpr int BK = (K % 2 == 0) ? K / 2 : K;
  // boundary lines projected by GEMM1: all B_K, except K = 3 where the three
  // lines' directions sum to zero, so p_1 = -(p_0 + p_2) is formed on the
  // CUDA cores
  static constexpr int BKG = (K == 3) ? 2 : BK;
  static constexpr int G = (K % 2 == 0) ? K / 2 : K - 1;
  static constexpr int R = K == 2 ? 64 : K == 7 ? 16 : 32;
  static constexpr int ROWS = R;  // coordinates per tile (packing granularity)
  static constexpr int N1 = BKG * R;   // GEMM1 N
  static constexpr int KD2 = G * R;    // GEMM2 reduction length per tile
  static constexpr int A2COLS = KD2 / 4;
  static constexpr int NOUT = KCH == 1 ? 8 : 16;  // real outputs per candidate (>= 2r)
  static constexpr int N2 = 2 * NOUT;             // GEMM2 N: hi and lo halves
  static constexpr int WCOLS = N1 + A2COLS + N2;
  static constexpr int NW = (512 / WCOLS) < 5 ? (512 / WCOLS) : 5;
  static constexpr int D1_OFF = 0, A2_OFF = N1, D2_OFF = N1 + A2COLS;
  static_assert(NW >= 1 && NW * WCOLS <= 512, "TMEM budget");
  static_assert(N1 % 16 == 0 && N1 <= 256, "GEMM1 N");
  static_assert(KD2 % 32 == 0, "GEMM2 K (FP8 MMAs reduce 32 entries)");
  static_assert(R % 16 == 0, "rows are processed 16 at a time");
  static_assert(A2COLS % 8 == 0, "indicator words are stored 8 columns at a time");
  static constexpr int THREADS = 128 * NW;
  // boundary line whose projections fill GEMM1 row block b
  static constexpr __host__ __device__ int line(int b) { return (K == 3 && b == 1) ? 2 : b; }
};

constexpr int align1k(int x) { return (x + 1023) / 1024 * 1024; }

template <int K, int KCH>
struct TcLayout {
  using Sh = TcShape<K, KCH>;
  static constexpr int N2R = Sh::N2;                      // B2 rows (16 B each) per 16-entry K-chunk
  static constexpr int B2ROWS = Sh::KD2 / 16 * N2R;       // 16-byte rows of B2 per tile
  static constexpr int B1_BYTES = Sh::N1 * 16 * KCH;
  static constexpr int B2_BYTES = B2ROWS * 16;
  static_assert(B1_BYTES % 256 == 0 && B2_BYTES % 256 == 0, "tiles are whole 256-byte TMA rows");
  // one packed tile = GEMM1 rows | GEMM2 rows, contiguous: one TMA box
  static constexpr int TILE_BYTES = B1_BYTES + B2_BYTES;
  static_assert(TILE_BYTES / 256 <= 256, "TMA box height");
  static constexpr int B1_OFF_IN_STAGE = 0;
  static constexpr int B2_OFF_IN_STAGE = B1_BYTES;
  static constexpr int STAGE_BYTES = align1k(TILE_BYTES);
  static constexpr uint32_t STAGE_TX = TILE_BYTES;
  static constexpr int A1_BYTES = kTcM * 16 * KCH;
  static constexpr int ACC_BYTES = kTcM * 16 * 8;         // two-sum partials, 128 x 16 x (hi, lo)
  static constexpr int ZERO_BYTES = 4096;
  static constexpr int WFIXED = align1k(2 * A1_BYTES) + ACC_BYTES;
  static constexpr int NST_FIT = (200 * 1024 - ZERO_BYTES - 4096 - Sh::NW * WFIXED) / (Sh::NW * STAGE_BYTES);
  static constexpr int NST = NST_FIT < kTcStages ? NST_FIT : kTcStages;  // stages per worker
  static_assert(NST >= 3, "pipeline depth");
  static constexpr int WSMEM = NST * STAGE_BYTES + WFIXED;  // per worker: stages | A1 x 2 | ACC
  static constexpr int W_A1 = NST * STAGE_BYTES;
  static constexpr int W_ACC = W_A1 + align1k(2 * A1_BYTES);
  static constexpr int ZERO_OFF = Sh::NW * WSMEM;
  static constexpr int BAR_OFF = ZERO_OFF + ZERO_BYTES;
  // per worker: full per stage, A1 full x 2, D1-full, D2-ready, drain of the
  // GEMM1 warp, A2-free, drain of the GEMM2 warp
  static constexpr int WBARS = NST + 7;
  static constexpr int USED = BAR_OFF + Sh::NW * WBARS * 8 + 16;
  // at least 120 KB so that two CTAs never share an SM (each holds all 512
  // TMEM columns)
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
  int flush;
};

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Every lane of the warp polls the barrier and the warp agrees on the outcome
// (measured: cheaper than one lane polling while the rest of its warp waits).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const bool ok = ptx::mbar_wait(bar, parity, abort, kWaitLimit);
  return __all_sync(0xffffffffu, ok);
}

// The worker's sequence of tiles: items gw, gw + workers, ... and the tiles of
// each item in order.
struct TcCursor {
  int64_t item;
  int j, ntile;
  int64_t ic;     // items passed
  int64_t chunk;  // coordinate chunk of the item
  int64_t ct;     // candidate tile of the item
  int64_t t0;     // first coordinate tile of the chunk
};

// The item's chunk, candidate tile and tile range, computed once per item
// (64-bit divisions are kept off the per-tile path).
__device__ __forceinline__ TcCursor tc_start(const TcParams& prm, int64_t item, int64_t ic) {
  TcCursor c;
  c.item = item;
  c.j = 0;
  c.ic = ic;
  c.chunk = item / prm.c_tiles;
  c.ct = item - c.chunk * prm.c_tiles;
  c.t0 = c.chunk * prm.tiles_per_chunk;
  c.ntile = item < prm.num_items ? static_cast<int>(min(prm.n_tiles, c.t0 + prm.tiles_per_chunk) - c.t0) : 0;
  return c;
}

__device__ __forceinline__ void tc_advance(const TcParams& prm, int64_t workers, TcCursor& c) {
  if (++c.j == c.ntile) c = tc_start(prm, c.item + workers, c.ic + 1);
}

template <int K, int KCH>
__global__ void __launch_bounds__(TcShape<K, KCH>::THREADS, 1)
    score_tc_kernel(const __grid_constant__ CUtensorMap tm_vt, const __grid_constant__ CUtensorMap tm_ct,
                    TcParams prm, const float* __restrict__ scale, const uint32_t* __restrict__ iw,
                    double* __restrict__ partial, int32_t* status) {
  using Sh = TcShape<K, KCH>;
  using L = TcLayout<K, KCH>;
  constexpr int R = Sh::R;
  constexpr int BK = Sh::BK;
  constexpr int BKG = Sh::BKG;
  constexpr int G = Sh::G;
  constexpr int NW = Sh::NW;
  constexpr int NST = L::NST;
  constexpr int NOUT = Sh::NOUT;
  constexpr int CW = R / 4;  // indicator words per class per tile

  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR_OFF + NW * L::WBARS * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (threadIdx.x == 0) {
    for (int i = 0; i < NW * L::WBARS; ++i) ptx::mbar_init(reinterpret_cast<uint64_t*>(smem + L::BAR_OFF) + i, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem + L::ZERO_OFF);
    for (int i = threadIdx.x; i < L::ZERO_BYTES / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int w = 0; w < NW; ++w) {
      uint4* acc = reinterpret_cast<uint4*>(smem + w * L::WSMEM + L::W_ACC);
      for (int i = threadIdx.x; i < L::ACC_BYTES / 16; i += blockDim.x) acc[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  ptx::fence_proxy_async_smem();
  if (warp == 0 && lane == 0) {
    ptx::tma_prefetch_desc(&tm_vt);
    ptx::tma_prefetch_desc(&tm_ct);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t smem_base = ptx::smem_u32(smem);
  const float inv_s = scale[1];

  const int F = prm.flush;
  const int64_t workers = static_cast<int64_t>(gridDim.x) * NW;
  const int w = warp >> 2;                                        // worker
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * NW + w;  // global worker id
  uint8_t* wsm = smem + w * L::WSMEM;
  const uint32_t wsm_s = smem_base + w * L::WSMEM;
  uint64_t* wb = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF) + w * L::WBARS;
  uint64_t* full_b = wb;
  uint64_t* a1_full = wb + NST;  // [2]
  uint64_t* d1_full = a1_full + 2;
  uint64_t* d2_ready = a1_full + 3;
  uint64_t* drain_bar = a1_full + 4;
  uint64_t* a2_free = a1_full + 5;
  uint64_t* drain2 = a1_full + 6;

  // Thread `row` owns candidate `row` of every tile.  Per tile g:
  //   wait D1(g) -> round its R coordinates into indicator words -> wait until
  //   GEMM2(g-1) has released A2 -> store them into A2 -> one warpgroup
  //   rendezvous -> warp 0 issues GEMM1(g+1) behind d1_full while warp 2
  //   issues GEMM2(g) behind a2_free (and d2_ready at the end of a period);
  //   both issue from the converged warp through one elected lane, and every
  //   wait is polled by whole warps -> every `flush` tiles fold D2 into the
  //   two-sum partials.  After the rendezvous the loader (one lane of warp 1)
  //   refills the stages freed by tile g-1.
  const int qtr = warp & 3;         // TMEM lane quarter
  const int row = qtr * 32 + lane;  // candidate row within the tile
  const bool loader = (qtr == 1 && lane == 0);  // issues the worker's TMA copies
  const uint32_t lane_base = static_cast<uint32_t>(qtr * 32) << 16;
  const uint32_t tw = tmem + w * Sh::WCOLS;  // this worker's TMEM slice
  constexpr uint32_t idesc1 = ptx::idesc_f16_f16(kTcM, Sh::N1);
  constexpr uint32_t idesc2 = ptx::idesc_e4m3_f32(kTcM, Sh::N2);
  constexpr uint32_t lbo_b2 = L::N2R * 16;
  float2* acc = reinterpret_cast<float2*>(wsm + L::W_ACC) + row * 16;  // (hi, lo) per component

  TcCursor cc = tc_start(prm, gw, 0);           // consumer: the tile being rounded
  TcCursor lc = cc;                             // loader: the next tile to load
  int64_t lg = 0, cg = 0;                       // tiles loaded / stages waited for
  int64_t la = 0, ca = 0;                       // direction tiles loaded / waited for

  // loader helpers: copies into the stage ring and the direction buffers
  auto load_tile = [&]() {
    const uint32_t s = static_cast<uint32_t>(lg % NST);
    uint8_t* st = wsm + s * L::STAGE_BYTES;
    const int64_t t = lc.t0 + lc.j;
    ptx::mbar_arrive_expect_tx(&full_b[s], L::STAGE_TX);
    ptx::tma_load_2d(st, &tm_vt, 0, static_cast<int>(t * (L::TILE_BYTES / 256)), &full_b[s]);
    ++lg;
    tc_advance(prm, workers, lc);
  };
  auto load_dirs = [&]() {  // directions of the worker's la-th item, if it exists
    const int64_t it = gw + la * workers;
    if (it >= prm.num_items) return;
    const uint32_t b = static_cast<uint32_t>(la & 1);
    ptx::mbar_arrive_expect_tx(&a1_full[b], L::A1_BYTES);
    ptx::tma_load_2d(wsm + L::W_A1 + b * L::A1_BYTES, &tm_ct, 0,
                     static_cast<int>((it % prm.c_tiles) * (L::A1_BYTES / 256)), &a1_full[b]);  // once per item
    ++la;
  };
  auto wait_stage = [&]() -> bool {  // the stage of tile cg (warp 0)
    const bool ok = warp_wait(&full_b[cg % NST], static_cast<uint32_t>((cg / NST) & 1), abort_flag);
    ++cg;
    return ok;
  };
  auto wait_dirs = [&]() -> bool {  // the direction buffer of item ca (warp 0)
    const bool ok = warp_wait(&a1_full[ca & 1], static_cast<uint32_t>((ca >> 1) & 1), abort_flag);
    ++ca;
    return ok;
  };
  auto gemm1 = [&](uint32_t stage, uint32_t ab) {
    constexpr bool two_chunks = (KCH == 2);
    const uint32_t a1 = wsm_s + L::W_A1 + ab * L::A1_BYTES;
    const uint32_t lbo_a1 = two_chunks ? kTcM * 16u : (smem_base + L::ZERO_OFF - a1);
    const uint32_t b1 = wsm_s + stage * L::STAGE_BYTES + L::B1_OFF_IN_STAGE;
    const uint32_t lbo_b1 = two_chunks ? Sh::N1 * 16u : (smem_base + L::ZERO_OFF - b1);
    ptx::mma_f16_ss_elect(tw + Sh::D1_OFF, ptx::smem_desc(a1, lbo_a1, 128), ptx::smem_desc(b1, lbo_b1, 128), idesc1,
                          0u);
    ptx::mma_commit_elect(d1_full);
  };

  uint32_t g = 0, pe = 0;
  int pos = 0;       // tile position within the accumulation period
  bool bad = false;  // this thread saw a wait give up (carried to the next barrier)
  if (cc.item < prm.num_items && loader) {
    // prologue: directions of the first two items, the first NST tiles
    load_dirs();
    load_dirs();
    while (lg < NST && lc.item < prm.num_items) load_tile();
  }
  if (cc.item < prm.num_items && qtr == 0) {
    // GEMM1(0) once its operands have landed
    const bool ok = wait_dirs() && wait_stage();
    if (ok) {
      ptx::tc_fence_after();
      gemm1(0u, 0u);
    } else if (lane == 0) {
      *abort_flag = 1;
    }
  }
  while (cc.item < prm.num_items) {
    const bool first = pos == 0;
    const bool item_end = (cc.j == cc.ntile - 1);
    const bool last = (pos == F - 1) || item_end;
    const bool has_next = !item_end || cc.item + workers < prm.num_items;
    // indicator magnitudes 2^(g - e_i) of the tile's coordinates (E4M3 bytes),
    // read while D1 is on its way
    uint32_t mag[CW];
    {
      const uint4* iwt = reinterpret_cast<const uint4*>(iw + (cc.t0 + cc.j) * CW);
#pragma unroll
      for (int c = 0; c < CW / 4; ++c) {
        const uint4 v4 = __ldg(iwt + c);
        mag[4 * c] = v4.x;
        mag[4 * c + 1] = v4.y;
        mag[4 * c + 2] = v4.z;
        mag[4 * c + 3] = v4.w;
      }
    }
    bad = bad || !warp_wait(d1_full, g & 1u, abort_flag);
    // ---- round the projections of tile g into indicator words in A2
    if (!bad) {
      ptx::tc_fence_after();
      uint32_t wv[G * CW];
      // D1 holds F16 projections, one per column; a packed load gives two
      // coordinates per register, so one byte permute gathers the signs of
      // four coordinates
      constexpr int RC = R < 32 ? R : 32;  // coordinates per load
#pragma unroll
      for (int ch = 0; ch < R / RC; ++ch) {
        uint32_t pl[BKG][RC / 2];
#pragma unroll
        for (int b = 0; b < BKG; ++b) {
          const uint32_t ta = tw + lane_base + Sh::D1_OFF + b * R + ch * RC;
          if constexpr (RC == 32)
            ptx::tmem_ld_x16_pack16(ta, *reinterpret_cast<uint32_t(*)[16]>(pl[b]));
          else
            ptx::tmem_ld_x8_pack16(ta, *reinterpret_cast<uint32_t(*)[8]>(pl[b]));
        }
        ptx::tmem_wait_ld();
#pragma unroll
        for (int p = 0; p < RC / 4; ++p) {
          uint32_t nm[BK];
          if constexpr (K == 3) {
            // p_1 = -(p_0 + p_2): the three boundary directions sum to zero, so
            // p_1 < 0 exactly where p_0 + p_2 > 0
            const uint32_t sum_neg = ptx::prmt(ptx::hadd2(pl[0][2 * p], pl[1][2 * p]),
                                               ptx::hadd2(pl[0][2 * p + 1], pl[1][2 * p + 1]), 0xFDB9u);
            nm[0] = ptx::prmt(pl[0][2 * p], pl[0][2 * p + 1], 0xFDB9u);
            nm[1] = ~sum_neg;
            nm[2] = ptx::prmt(pl[1][2 * p], pl[1][2 * p + 1], 0xFDB9u);
          } else {
#pragma unroll
            for (int m = 0; m < BK; ++m) nm[m] = ptx::prmt(pl[m][2 * p], pl[m][2 * p + 1], 0xFDB9u);
          }
          const int wi = ch * (RC / 4) + p;
#pragma unroll
          for (int gc = 0; gc < G; ++gc) {
            if constexpr (K % 2 == 1)
              wv[gc * CW + wi] = ~nm[gc] & nm[gc + 1] & mag[wi];  // p_{k-1} > 0 and p_k < 0
            else
              wv[gc * CW + wi] = (nm[gc] & 0x80808080u) | mag[wi];  // sign(p_m) as +-1
          }
        }
      }
      // GEMM2(g-1) has released A2
      if (g > 0) bad = !warp_wait(a2_free, (g - 1) & 1u, abort_flag);
      if (!bad) {
        ptx::tc_fence_after();
#pragma unroll
        for (int c = 0; c < Sh::A2COLS / 8; ++c)
          ptx::tmem_st_x8(tw + lane_base + Sh::A2_OFF + c * 8, *reinterpret_cast<const uint32_t(*)[8]>(&wv[c * 8]));
        ptx::tmem_wait_st();
      }
    }
    ptx::tc_fence_before();
    // D1 read and A2 written by the whole warpgroup; all leave together on failure
    if (ptx::named_barrier_or(1 + w, 128, bad)) break;
    // ---- the loader: GEMM1(g) is done (D1(g) was seen) and so is GEMM2(g-1)
    // (every warp saw a2_free before storing A2): the stages up to tile g-1
    // are free, and at the end of an item its direction buffer
    if (loader) {
      while (lg <= static_cast<int64_t>(g) - 1 + NST && lc.item < prm.num_items) load_tile();
      if (item_end) load_dirs();
    }
    // ---- warp 0: GEMM1(g+1) into D1
    if (qtr == 0) {
      ptx::tc_fence_after();
      bool ok = true;
      if (has_next) {
        ok = item_end ? wait_dirs() : true;
        ok = ok && wait_stage();
        if (ok) gemm1((g + 1) % NST, static_cast<uint32_t>((cc.ic + (item_end ? 1 : 0)) & 1));
      }
      if (!ok && lane == 0) *abort_flag = 1;
    }
    // ---- warp 2: GEMM2(g) from A2 and the tile's stage into D2
    if (qtr == 2) {
      ptx::tc_fence_after();
      const uint32_t b2 = wsm_s + (g % NST) * L::STAGE_BYTES + L::B2_OFF_IN_STAGE;
#pragma unroll
      for (int q = 0; q < Sh::KD2 / 32; ++q)
        ptx::mma_e4m3_ts_elect(tw + Sh::D2_OFF, tw + Sh::A2_OFF + q * 8,
                               ptx::smem_desc(b2 + q * 2 * lbo_b2, lbo_b2, 128), idesc2, (q > 0 || !first) ? 1u : 0u);
      if (last) ptx::mma_commit_elect(d2_ready);
      ptx::mma_commit_elect(a2_free);
    }
    // ---- fold the period's accumulator into the two-sum partials
    if (last) {
      bad = !warp_wait(d2_ready, pe & 1u, abort_flag);
      if (!bad) {
        ptx::tc_fence_after();
        uint32_t dh[16], dl[16];
        if constexpr (NOUT == 8) {
          ptx::tmem_ld_x16(tw + lane_base + Sh::D2_OFF, dh);
          ptx::tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) dl[jj] = dh[8 + jj];
        } else {
          ptx::tmem_ld_x16(tw + lane_base + Sh::D2_OFF, dh);
          ptx::tmem_ld_x16(tw + lane_base + Sh::D2_OFF + 16, dl);
          ptx::tmem_wait_ld();
        }
        ptx::tc_fence_before();
        const int r2 = 2 * prm.r;
        double* out = partial + (cc.chunk * prm.S_pad + cc.ct * kTcM + row) * r2;
#pragma unroll
        for (int jj = 0; jj < NOUT; ++jj) {
          if (jj < r2) {
            float2 hl = acc[jj];
            float s, er;
            two_sum_f(hl.x, __uint_as_float(dh[jj]), s, er);
            hl.x = s;
            hl.y += er;
            two_sum_f(hl.x, __uint_as_float(dl[jj]), s, er);
            hl.x = s;
            hl.y += er;
            if (item_end) {
              out[jj] = (static_cast<double>(hl.x) + static_cast<double>(hl.y)) * static_cast<double>(inv_s);
              hl = make_float2(0.f, 0.f);
            }
            acc[jj] = hl;
          }
        }
      }
      ++pe;
    }
    // ---- advance
    pos = last ? 0 : pos + 1;
    ++g;
    tc_advance(prm, workers, cc);
  }
  if (bad || *abort_flag) {
    *abort_flag = 1;
    dev_fail(status, LRQ_ETIMEOUT);
  }
  // drain: the MMAs of warps 0 and 2 and the loader's copies complete before
  // TMEM and shared memory are released (a stage or direction buffer is
  // refilled only after its previous copy was consumed, so only the last NST
  // tile copies and the last two direction copies can be outstanding)
  if (qtr == 0 || qtr == 2) {
    volatile int never = 0;
    uint64_t* db = qtr == 0 ? drain_bar : drain2;
    ptx::mma_commit_elect(db);
    warp_wait(db, 0u, &never);
  }
  if (loader) {
    volatile int never = 0;
    for (int64_t t = lg > NST ? lg - NST : 0; t < lg; ++t)
      ptx::mbar_wait(&full_b[t % NST], static_cast<uint32_t>((t / NST) & 1), &never, kWaitLimit);
    for (int64_t t = la > 2 ? la - 2 : 0; t < la; ++t)
      ptx::mbar_wait(&a1_full[t & 1], static_cast<uint32_t>((t >> 1) & 1), &never, kWaitLimit);
  }
  // ------------------------------------------------------------ teardown
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
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
__global__ void pack_indicator_scale_kernel(const float2* __restrict__ V, int64_t n, int r, int64_t words,
                                            const float* __restrict__ scale, uint32_t* __restrict__ iw) {
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

template <int K, int KCH>
static int pack_impl(const ScorePlan& p, const Alphabet& a, const float2* V, const float2* C, void* tiles,
                     void* ct, float* scale, uint32_t* iw, cudaStream_t st) {
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
  pack_indicator_scale_kernel<<<static_cast<unsigned>(ceil_div(words, 256)), 256, 0, st>>>(V, p.n, p.r, words, scale,
                                                                                          iw);
  int64_t nb = p.n_tiles * L::B2ROWS;
  pack_b2_kernel<K, KCH><<<static_cast<unsigned>(ceil_div(nb, 256)), 256, 0, st>>>(
      V, p.n, p.r, p.n_tiles, tb, scale, reinterpret_cast<const uint8_t*>(iw), static_cast<uint8_t*>(tiles));
  count_launch(2);
  int64_t nc = p.c_tiles * kTcM;
  pack_dirs_kernel<KCH><<<static_cast<unsigned>(ceil_div(nc, 256)), 256, 0, st>>>(C, p.S, p.r, p.c_tiles,
                                                                                  static_cast<__half*>(ct));
  count_launch();
  return cuda_check(cudaGetLastError(), "tc pack kernels");
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
static int score_impl(const ScorePlan& p, const void* tiles, const void* ct, const float* scale,
                      const uint32_t* iw, double* partial, int32_t* status, cudaStream_t st) {
  using Sh = TcShape<K, KCH>;
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
  prm.flush = kTcFlush;
  int grid = static_cast<int>(std::min<int64_t>(ceil_div(prm.num_items, Sh::NW), num_sms_current()));
  score_tc_kernel<K, KCH><<<grid, Sh::THREADS, L::TOTAL, st>>>(m_vt, m_ct, prm, scale, iw, partial, status);
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

int tc_rows_per_tile(int K) {
  const bool two = false;
#define LRQ_ROWS(k, c) TcShape<k, c>::ROWS
  LRQ_TC_SHAPE_SWITCH(LRQ_ROWS);
#undef LRQ_ROWS
}

int tc_workers_per_cta(int K, int r) {
  const bool two = r > 4;
#define LRQ_NW(k, c) TcShape<k, c>::NW
  LRQ_TC_SHAPE_SWITCH(LRQ_NW);
#undef LRQ_NW
}

size_t tc_bytes_tiles(int K, int r, int64_t n_tiles) {
  const bool two = r > 4;
#define LRQ_TILE(k, c) static_cast<size_t>(n_tiles) * TcLayout<k, c>::TILE_BYTES
  LRQ_TC_SHAPE_SWITCH(LRQ_TILE);
#undef LRQ_TILE
}

size_t tc_bytes_indicator_scale(int K, int64_t n_tiles) {
  return static_cast<size_t>(n_tiles) * static_cast<size_t>(tc_rows_per_tile(K));  // one byte per coordinate
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

int launch_tc_pack(const ScorePlan& p, const Alphabet& a, const float2* V, const float2* C, void* tiles, void* ct,
                   void* scale, void* iw, cudaStream_t st) {
  LRQ_TC_DISPATCH(pack_impl, p, a, V, C, tiles, ct, static_cast<float*>(scale), static_cast<uint32_t*>(iw), st);
}

int launch_score_tc(const ScorePlan& p, const Alphabet& a, const void* tiles, const void* ct, const void* scale,
                    const void* iw, double* partial, int32_t* status, cudaStream_t st) {
  (void)a;
  LRQ_TC_DISPATCH(score_impl, p, tiles, ct, static_cast<const float*>(scale), static_cast<const uint32_t*>(iw),
                  partial, status, st);
}

}  // namespace lrq
