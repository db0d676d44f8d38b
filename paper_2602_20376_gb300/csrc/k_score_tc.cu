// k_score_tc.cu -- tensor-core (tcgen05 + TMEM + TMA) candidate scoring.
//
// The scoring of Sec. 4.2, Eq. 10 is cast as two contractions per
// (128-candidate tile, coordinate tile):
//
// GEMM1 (boundary projections).  The augmented real matrix of Eq. 6 has one
// row per (coordinate i, boundary m): [Im(rho_m V_i), Re(rho_m V_i)] with
// rho_m = exp(-i theta_m), theta_m = pi(2m+1)/K, m < B_K (Definition 2.1).
// Against c~ = [Re c; Im c] a row gives p_m = Im(rho_m V_i c), whose sign says
// on which side of decision boundary m the value w_i = V_i c lies.  So
//   D1[s, (m, i)] = sum_k C~[s, k] * Vaug[(m, i), k]     (M = 128, K = 2r -> 16)
// and the decision rule (Sec. 3, Eq. 9) becomes a sign test per row.
//
// Sector rounding in the epilogue.  With N_m the sign mask of p_m:
//   odd K  : class k in 1..K-1 iff p_{k-1} > 0 and p_k < 0  -> indicator 1/0
//   even K : z = sum_m beta_m sign(p_m), beta_m = (w^{m+1} - w^m)/2   -> +-1
// (w = exp(2 pi i/K)).  Indicators are exact in BF16; pairs of rows are
// turned into packed BF16 words with byte permutes (sign replication) and
// one 3-input logic op -- no trigonometry, no branches.
//
// GEMM2 (per-class sums).  V^H z = T + sum_k (w^k - 1) P_k (odd K, T the
// column sum of conj(V)) or sum_m beta_m S_m (even K), where P_k / S_m are
// sums of conj(V_i) selected or signed by the indicators:
//   D2[s, :] += sum_{(g, i)} Ind[s, (g, i)] * B2[(g, i), :]   (N = 16 >= 2r)
// with B2 rows the real form of beta_g conj(V_i).  D2 accumulates in TMEM
// (FP32) for at most `flush` tiles, then is folded into FP32 two-sum
// registers (error-free) and written as FP64 partials per coordinate chunk.
//
// Pipeline (one CTA per SM, persistent over (chunk, candidate tile) items):
// NW independent workers per CTA, each a warpgroup (one thread per
// candidate of the 128-candidate tile) with its own TMA producer thread
// (warps 0..NW-1), stage ring and TMEM slice (D1 projections, A2 indicator
// words, D2 accumulator).  Per tile the worker reads D1 from TMEM, rounds it
// into indicator words written back to TMEM (tcgen05.st) as GEMM2's A
// operand, and one fixed thread of the worker issues GEMM2 of this tile and
// GEMM1 of the next; the workers of a CTA interleave on the tensor core.
// Every wait is bounded; on expiry the kernel records LRQ_ETIMEOUT, drains
// its in-flight copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
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

// Tile shape per alphabet.  A CTA runs NW independent workers; each worker is
// one warpgroup (128 threads, one per candidate of the tile) plus a producer
// thread, and owns a TMEM slice of WCOLS columns:
//   D1 : N1 = BK * R columns    GEMM1 projections of one tile
//   A2 : KD2 / 2 columns         GEMM2 indicator operand (bf16 pairs)
//   D2 : 16 columns              GEMM2 accumulator
// NW * WCOLS <= 512.  R is the number of coordinates per tile.
template <int K>
struct TcShape {
  static constexpr int BK = (K % 2 == 0) ? K / 2 : K;
  // boundary lines projected by GEMM1: all B_K, except K = 3 where the three
  // lines' directions sum to zero, so p_1 = -(p_0 + p_2) is formed on the
  // CUDA cores
  static constexpr int BKG = (K == 3) ? 2 : BK;
  static constexpr int G = (K % 2 == 0) ? K / 2 : K - 1;
  static constexpr int NW = K == 2 ? 4 : K == 3 ? 4 : K == 4 ? 4 : K == 5 ? 2 : K == 6 ? 3 : K == 7 ? 2 : 2;
  static constexpr int R = K == 2 ? 64 : K == 7 ? 16 : 32;
  static constexpr int ROWS = R;  // coordinates per tile (packing granularity)
  static constexpr int N1 = BKG * R;   // GEMM1 N
  static constexpr int KD2 = G * R;    // GEMM2 reduction length per tile
  static constexpr int A2COLS = KD2 / 2;
  static constexpr int WCOLS = N1 + A2COLS + 16;
  static constexpr int D1_OFF = 0, A2_OFF = N1, D2_OFF = N1 + A2COLS;
  static_assert(NW * WCOLS <= 512, "TMEM budget");
  static_assert(N1 % 16 == 0 && N1 <= 256, "GEMM1 N");
  static_assert(KD2 % 16 == 0, "GEMM2 K");
  static_assert(R % 16 == 0, "rows are processed 16 at a time");
  static constexpr int THREADS = 128 + 128 * NW;
  // boundary line whose projections fill GEMM1 row block b
  static constexpr __host__ __device__ int line(int b) { return (K == 3 && b == 1) ? 2 : b; }
};

constexpr int align1k(int x) { return (x + 1023) / 1024 * 1024; }

template <int K, int KCH>
struct TcLayout {
  using Sh = TcShape<K>;
  static constexpr int N2R = (KCH == 1) ? 8 : 16;         // B2 rows stored per K-chunk
  static constexpr int B2ROWS = Sh::KD2 / 8 * N2R;        // 16-byte rows of B2 per tile
  static constexpr int B1_BYTES = Sh::N1 * 16 * KCH;
  static constexpr int B2_BYTES = B2ROWS * 16;
  static_assert(B1_BYTES % 256 == 0 && B2_BYTES % 256 == 0, "tiles are whole 256-byte TMA rows");
  static constexpr int B1_OFF_IN_STAGE = 0;
  static constexpr int B2_OFF_IN_STAGE = align1k(B1_BYTES);
  static constexpr int STAGE_BYTES = align1k(B2_OFF_IN_STAGE + B2_BYTES);
  static constexpr uint32_t STAGE_TX = B1_BYTES + B2_BYTES;
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
  // per worker: full / empty per stage, A1 full / empty pairs, D1-full, D2-ready, 4 drains
  static constexpr int WBARS = 2 * NST + 4 + 2 + 4;
  static constexpr int USED = BAR_OFF + Sh::NW * WBARS * 8 + 16;
  // at least 120 KB so that two CTAs never share an SM (each holds all 512
  // TMEM columns)
  static constexpr int TOTAL = USED < 120 * 1024 ? 120 * 1024 : USED;
  static_assert(Sh::N1 * 16 <= ZERO_BYTES && kTcM * 16 <= ZERO_BYTES && Sh::KD2 * 16 <= ZERO_BYTES, "zero pad");
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

// One lane of the warp polls the barrier (keeps shared-memory traffic low);
// the outcome is broadcast to the warp, which is converged afterwards.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int lane) {
  int ok = 1;
  if (lane == 0) ok = ptx::mbar_wait(bar, parity, abort, kWaitLimit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// GEMM1 of one tile of a worker: wait for the stage's operands (unless the
// caller already did), then D1 = A1[ab] x Vaug(stage)^T and commit to d1_full.  wsm_s is the shared
// address of the worker's region.
template <class L>
__device__ __forceinline__ bool tc_issue_gemm1(uint32_t tw, uint32_t wsm_s, uint32_t smem_base, uint64_t* full_b,
                                               uint64_t* d1_full, uint32_t stage, uint32_t sphase, uint32_t ab,
                                               volatile int* abort, bool wait_stage = true) {
  using Sh = typename L::Sh;
  constexpr bool two_chunks = (L::N2R == 16);
  if (wait_stage && !ptx::mbar_wait(&full_b[stage], sphase, abort, kWaitLimit)) return false;
  ptx::tc_fence_after();
  const uint32_t a1 = wsm_s + L::W_A1 + ab * L::A1_BYTES;
  const uint32_t lbo_a1 = two_chunks ? kTcM * 16u : (smem_base + L::ZERO_OFF - a1);
  const uint32_t b1 = wsm_s + stage * L::STAGE_BYTES + L::B1_OFF_IN_STAGE;
  const uint32_t lbo_b1 = two_chunks ? Sh::N1 * 16u : (smem_base + L::ZERO_OFF - b1);
  ptx::mma_bf16_ss(tw + Sh::D1_OFF, ptx::smem_desc(a1, lbo_a1, 128), ptx::smem_desc(b1, lbo_b1, 128),
                   ptx::idesc_bf16_f32(kTcM, Sh::N1), 0u);
  ptx::mma_commit(d1_full);
  return true;
}

template <int K, int KCH>
__global__ void __launch_bounds__(TcShape<K>::THREADS, 1)
    score_tc_kernel(const __grid_constant__ CUtensorMap tm_vt, const __grid_constant__ CUtensorMap tm_b2,
                    const __grid_constant__ CUtensorMap tm_ct, TcParams prm, double* __restrict__ partial,
                    int32_t* status) {
  using Sh = TcShape<K>;
  using L = TcLayout<K, KCH>;
  constexpr int R = Sh::R;
  constexpr int BK = Sh::BK;
  constexpr int G = Sh::G;
  constexpr int NW = Sh::NW;
  constexpr int NST = L::NST;

  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR_OFF + NW * L::WBARS * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (threadIdx.x == 0) {
    for (int w = 0; w < NW; ++w) {
      uint64_t* wb = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF) + w * L::WBARS;
      for (int s = 0; s < NST; ++s) {
        ptx::mbar_init(&wb[s], 1);        // stage landed (TMA)
        ptx::mbar_init(&wb[NST + s], 1);  // stage consumed (GEMM2 commit)
      }
      for (int i = 2 * NST; i < L::WBARS; ++i) ptx::mbar_init(&wb[i], 1);
    }
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
    ptx::tma_prefetch_desc(&tm_b2);
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

  const int64_t c_tiles = prm.c_tiles;
  const int64_t tpc = prm.tiles_per_chunk;
  const int F = prm.flush;
  const int64_t workers = static_cast<int64_t>(gridDim.x) * NW;

  // worker index within the CTA: producers are warps 0..NW-1, warpgroups follow
  const int w = (warp < 4) ? warp : (warp - 4) >> 2;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * NW + w;  // global worker id
  uint8_t* wsm = smem + w * L::WSMEM;
  const uint32_t wsm_s = smem_base + w * L::WSMEM;
  uint64_t* wb = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF) + w * L::WBARS;
  uint64_t* full_b = wb;
  uint64_t* empty_b = wb + NST;
  uint64_t* a1_full = wb + 2 * NST;
  uint64_t* a1_empty = a1_full + 2;
  uint64_t* d1_full = a1_full + 4;
  uint64_t* d2_ready = a1_full + 5;
  uint64_t* drain_bar = a1_full + 6;  // [4]

  if (warp < NW) {
    // ------------------------------------------------------------ producer of worker w
    uint32_t issued = 0, a1_issued = 0;
    if (lane == 0) {
      uint32_t stage = 0, sphase = 0;
      bool ok = true;
      for (int64_t item = gw; item < prm.num_items && ok; item += workers) {
        const int64_t chunk = item / c_tiles, ct = item % c_tiles;
        const int64_t t0 = chunk * tpc;
        const int ntile = static_cast<int>(min(prm.n_tiles, t0 + tpc) - t0);
        const uint32_t ab = a1_issued & 1u;
        if (!ptx::mbar_wait(&a1_empty[ab], ((a1_issued >> 1) & 1u) ^ 1u, abort_flag, kWaitLimit)) {
          ok = false;
          break;
        }
        ptx::mbar_arrive_expect_tx(&a1_full[ab], L::A1_BYTES);
        ptx::tma_load_2d(wsm + L::W_A1 + ab * L::A1_BYTES, &tm_ct, 0, static_cast<int>(ct * (L::A1_BYTES / 256)),
                         &a1_full[ab]);
        ++a1_issued;
        for (int j = 0; j < ntile; ++j) {
          if (!ptx::mbar_wait(&empty_b[stage], sphase ^ 1u, abort_flag, kWaitLimit)) {
            ok = false;
            break;
          }
          uint8_t* st = wsm + stage * L::STAGE_BYTES;
          const int64_t t = t0 + j;
          ptx::mbar_arrive_expect_tx(&full_b[stage], L::STAGE_TX);
          ptx::tma_load_2d(st + L::B1_OFF_IN_STAGE, &tm_vt, 0, static_cast<int>(t * (L::B1_BYTES / 256)),
                           &full_b[stage]);
          ptx::tma_load_2d(st + L::B2_OFF_IN_STAGE, &tm_b2, 0, static_cast<int>(t * (L::B2_BYTES / 256)),
                           &full_b[stage]);
          ++issued;
          if (++stage == NST) {
            stage = 0;
            sphase ^= 1u;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        dev_fail(status, LRQ_ETIMEOUT);
      }
      // drain: every issued copy must have landed before the CTA exits
      volatile int never = 0;
      for (uint32_t s = 0; s < NST && s < issued; ++s) {
        uint32_t cnt = issued / NST + (s < issued % NST ? 1u : 0u);
        ptx::mbar_wait(&full_b[s], (cnt - 1) & 1u, &never, kWaitLimit);
      }
      for (uint32_t b = 0; b < 2 && b < a1_issued; ++b) {
        uint32_t cnt = a1_issued / 2 + (b < a1_issued % 2 ? 1u : 0u);
        ptx::mbar_wait(&a1_full[b], (cnt - 1) & 1u, &never, kWaitLimit);
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ worker warpgroup w
    // Thread `row` owns candidate `row` of every tile.  Per tile g:
    //   wait D1(g) -> round its R coordinates into indicator words -> store
    //   them into A2 -> one warpgroup rendezvous -> the issuing thread issues
    //   GEMM2(g) and then GEMM1(g+1), both committed behind one d1_full
    //   arrival, so seeing D1(g+1) also certifies that GEMM2(g) has released
    //   A2 (tcgen05.commit tracks every earlier MMA of the committing thread)
    //   -> every `flush` tiles fold D2 into the two-sum partials.
    // One fixed thread issues every MMA of the worker (needed for the
    // ordering argument); it also waits for the TMA stage of tile g+2 while
    // the tensor core runs, so that GEMM1(g+1) never waits on a copy.
    const int qtr = warp & 3;         // TMEM lane quarter
    const int row = qtr * 32 + lane;  // candidate row within the tile
    const bool issuer = (qtr == 0 && lane == 0);
    const uint32_t lane_base = static_cast<uint32_t>(qtr * 32) << 16;
    const uint32_t tw = tmem + w * Sh::WCOLS;  // this worker's TMEM slice
    constexpr uint32_t idesc2 = ptx::idesc_bf16_f32(kTcM, 16);
    constexpr uint32_t lbo_b2 = L::N2R * 16;
    constexpr int BKG = Sh::BKG;
    float2* acc = reinterpret_cast<float2*>(wsm + L::W_ACC) + row * 16;  // (hi, lo) per component

    // the worker's tile sequence: items gw, gw + workers, ...; tiles in order
    int64_t item = gw;
    int ntile = 0, j = 0, next_ntile = 0;  // tiles of the current / next item (0: none)
    int64_t chunk = 0, ct = 0;
    auto tiles_of = [&](int64_t it) -> int {
      if (it >= prm.num_items) return 0;
      const int64_t t0 = (it / c_tiles) * tpc;
      return static_cast<int>(min(prm.n_tiles, t0 + tpc) - t0);
    };
    auto stage_next = [](uint32_t& s, uint32_t& ph) {
      if (++s == NST) {
        s = 0;
        ph ^= 1u;
      }
    };
    uint32_t g = 0, pe = 0, stage = 0, sphase = 0, a1c = 0;
    int pos = 0;       // tile position within the accumulation period
    bool bad = false;  // this thread saw a wait give up (carried to the next barrier)
    if (item < prm.num_items) {
      chunk = item / c_tiles;
      ct = item % c_tiles;
      ntile = tiles_of(item);
      next_ntile = tiles_of(item + workers);
      // prologue: GEMM1 of the first tile, then the stage of the second
      // (a failure reaches every thread through the abort flag)
      if (issuer) {
        bool ok = ptx::mbar_wait(&a1_full[0], 0u, abort_flag, kWaitLimit) &&
                  tc_issue_gemm1<L>(tw, wsm_s, smem_base, full_b, d1_full, 0u, 0u, 0u, abort_flag);
        if (ok && ntile == 1) ptx::mma_commit(&a1_empty[0]);
        if (ok && (ntile > 1 || next_ntile > 0)) {
          uint32_t s1 = 0, p1 = 0;
          stage_next(s1, p1);
          ok = ptx::mbar_wait(&full_b[s1], p1, abort_flag, kWaitLimit);
        }
        if (!ok) *abort_flag = 1;
      }
    }
    while (item < prm.num_items) {
      const bool first = pos == 0;
      const bool last = (pos == F - 1) || (j == ntile - 1);
      const bool item_end = (j == ntile - 1);
      const bool has_next = !item_end || next_ntile > 0;
      // ---- round the projections of tile g into indicator words in A2
      bad = bad || !warp_wait(d1_full, g & 1u, abort_flag, lane);
      if (!bad) {
        ptx::tc_fence_after();
        uint32_t wv[G][R / 2];
#pragma unroll
        for (int h = 0; h < R / 16; ++h) {
          uint32_t pl[BKG][16];
#pragma unroll
          for (int b = 0; b < BKG; ++b) ptx::tmem_ld_x16(tw + lane_base + Sh::D1_OFF + b * R + h * 16, pl[b]);
          ptx::tmem_wait_ld();
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            uint32_t nm[BK];
            if constexpr (K == 3) {
              // p_1 = -(p_0 + p_2): the three boundary directions sum to zero
              const float q0 = -(__uint_as_float(pl[0][2 * p]) + __uint_as_float(pl[1][2 * p]));
              const float q1 = -(__uint_as_float(pl[0][2 * p + 1]) + __uint_as_float(pl[1][2 * p + 1]));
              nm[0] = ptx::prmt(pl[0][2 * p], pl[0][2 * p + 1], 0xFFBBu);
              nm[1] = ptx::prmt(__float_as_uint(q0), __float_as_uint(q1), 0xFFBBu);
              nm[2] = ptx::prmt(pl[1][2 * p], pl[1][2 * p + 1], 0xFFBBu);
            } else {
#pragma unroll
              for (int m = 0; m < BK; ++m) nm[m] = ptx::prmt(pl[m][2 * p], pl[m][2 * p + 1], 0xFFBBu);
            }
#pragma unroll
            for (int gc = 0; gc < G; ++gc) {
              if constexpr (K % 2 == 1)
                wv[gc][h * 8 + p] = ~nm[gc] & nm[gc + 1] & 0x3F803F80u;  // p_{k-1} > 0 and p_k < 0
              else
                wv[gc][h * 8 + p] = (nm[gc] & 0x80008000u) | 0x3F803F80u;  // sign(p_m) as +-1
            }
          }
        }
#pragma unroll
        for (int gc = 0; gc < G; ++gc) {
          if constexpr (R == 16)
            ptx::tmem_st_x8(tw + lane_base + Sh::A2_OFF + gc * (R / 2),
                            *reinterpret_cast<const uint32_t(*)[8]>(wv[gc]));
          else
#pragma unroll
            for (int c = 0; c < R / 32; ++c)
              ptx::tmem_st_x16(tw + lane_base + Sh::A2_OFF + gc * (R / 2) + c * 16,
                               *reinterpret_cast<const uint32_t(*)[16]>(&wv[gc][c * 16]));
        }
        ptx::tmem_wait_st();
      }
      ptx::tc_fence_before();
      // D1 read and A2 written by the whole warpgroup; all leave together on failure
      if (ptx::named_barrier_or(1 + w, 128, bad)) break;
      // ---- the issuing thread: GEMM2(g), then GEMM1(g+1), then the stage of g+2
      uint32_t s1 = stage, p1 = sphase;
      stage_next(s1, p1);  // stage of tile g+1
      if (issuer) {
        ptx::tc_fence_after();
        const uint32_t b2 = wsm_s + stage * L::STAGE_BYTES + L::B2_OFF_IN_STAGE;
#pragma unroll
        for (int q = 0; q < Sh::KD2 / 16; ++q) {
          const uint32_t bstart = b2 + q * 2 * lbo_b2;
          const uint32_t sbo_b2 = (KCH == 2) ? 128u : (smem_base + L::ZERO_OFF - bstart);
          ptx::mma_bf16_ts(tw + Sh::D2_OFF, tw + Sh::A2_OFF + q * 8, ptx::smem_desc(bstart, lbo_b2, sbo_b2), idesc2,
                           (q > 0 || !first) ? 1u : 0u);
        }
        ptx::mma_commit(&empty_b[stage]);  // releases the stage (GEMM1(g) and GEMM2(g) read it)
        if (last) ptx::mma_commit(d2_ready);
        bool ok = true;
        if (has_next) {
          uint32_t nab = a1c & 1u;
          if (item_end) {  // the next tile opens the next item: wait for its directions
            nab ^= 1u;
            ok = ptx::mbar_wait(&a1_full[nab], ((a1c + 1) >> 1) & 1u, abort_flag, kWaitLimit);
          }
          // stage s1 was waited for one tile ago (or in the prologue): p1 is complete
          ok = ok && tc_issue_gemm1<L>(tw, wsm_s, smem_base, full_b, d1_full, s1, p1, nab, abort_flag, false);
          if (ok && (item_end ? 0 : j + 1) == (item_end ? next_ntile : ntile) - 1) ptx::mma_commit(&a1_empty[nab]);
          // does a tile g+2 exist?  (then wait for its stage while the MMAs run)
          bool has_next2;
          if (!item_end)
            has_next2 = (j + 2 < ntile) || next_ntile > 0;
          else
            has_next2 = next_ntile > 1 || tiles_of(item + 2 * workers) > 0;
          if (ok && has_next2) {
            uint32_t s2 = s1, p2 = p1;
            stage_next(s2, p2);
            ok = ptx::mbar_wait(&full_b[s2], p2, abort_flag, kWaitLimit);
          }
        }
        if (!ok) *abort_flag = 1;
      }
      // ---- fold the period's accumulator into the two-sum partials
      if (last) {
        bad = !warp_wait(d2_ready, pe & 1u, abort_flag, lane);
        if (!bad) {
          ptx::tc_fence_after();
          uint32_t dv[16];
          ptx::tmem_ld_x16(tw + lane_base + Sh::D2_OFF, dv);
          ptx::tmem_wait_ld();
          ptx::tc_fence_before();
          const int r2 = 2 * prm.r;
          double* out = partial + (chunk * prm.S_pad + ct * kTcM + row) * r2;
#pragma unroll
          for (int jj = 0; jj < 2 * kMaxRank; ++jj) {
            if (jj < r2) {
              float2 hl = acc[jj];
              float s, er;
              two_sum_f(hl.x, __uint_as_float(dv[jj]), s, er);
              hl.x = s;
              hl.y += er;
              if (item_end) {
                out[jj] = static_cast<double>(hl.x) + static_cast<double>(hl.y);
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
      stage = s1;
      sphase = p1;
      ++g;
      if (item_end) {
        ++a1c;
        item += workers;
        if (item < prm.num_items) {
          chunk = item / c_tiles;
          ct = item % c_tiles;
          ntile = next_ntile;
          next_ntile = tiles_of(item + workers);
        }
        j = 0;
      } else {
        ++j;
      }
    }
    if (bad || *abort_flag) {
      *abort_flag = 1;
      dev_fail(status, LRQ_ETIMEOUT);
    }
    // drain: the MMAs issued from this warp complete before TMEM is released
    if (lane == 0) {
      ptx::mma_commit(&drain_bar[qtr]);
      volatile int never = 0;
      ptx::mbar_wait(&drain_bar[qtr], 0u, &never, kWaitLimit);
    }
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
// Operand packing (run once per call): bf16 tiles in the exact shared-memory
// order the MMA descriptors expect, so each stage is one TMA box.
// ---------------------------------------------------------------------------
struct PackTables {
  float bcos[8], bsin[8];    // boundary directions theta_m, m < B_K
  float beta_r[8], beta_i[8];  // per-indicator coefficients
};

// augmented rows: tile t, chunk ch, row (b*ROWS + i) for boundary line
// line(b), 8 slots
template <int K, int KCH>
__global__ void pack_vaug_kernel(const float2* __restrict__ V, int64_t n, int r, int64_t n_tiles, PackTables tb,
                                 __nv_bfloat16* __restrict__ vt) {
  using Sh = TcShape<K>;
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
    const float bc = tb.bcos[m], bs = tb.bsin[m];
    for (int jj = 0; jj < r; ++jj) {
      float2 v = V[ig * r + jj];
      // rho_m V = (bc - i bs)(vr + i vi)
      slot[jj] = fmaf(bc, v.y, -bs * v.x);     // Im(rho_m V_ij)
      slot[r + jj] = fmaf(bc, v.x, bs * v.y);  // Re(rho_m V_ij)
    }
  }
#pragma unroll
  for (int ch = 0; ch < KCH; ++ch) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = __float2bfloat16_rn(slot[ch * 8 + k]);
    *reinterpret_cast<uint4*>(vt + ((t * KCH + ch) * Sh::N1 + rowin) * 8) = *reinterpret_cast<uint4*>(h);
  }
}

// GEMM2 B rows: tile t, K-chunk kc, output column nc: 8 reduction entries
template <int K, int KCH>
__global__ void pack_b2_kernel(const float2* __restrict__ V, int64_t n, int r, int64_t n_tiles, PackTables tb,
                               __nv_bfloat16* __restrict__ b2) {
  using Sh = TcShape<K>;
  using L = TcLayout<K, KCH>;
  const int64_t total = n_tiles * L::B2ROWS;
  int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int64_t t = q / L::B2ROWS;
  const int within = static_cast<int>(q % L::B2ROWS);
  const int kc = within / L::N2R, nc = within % L::N2R;
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int kk = kc * 8 + k;
    const int gc = kk / Sh::ROWS, i = kk % Sh::ROWS;
    const int64_t ig = t * Sh::ROWS + i;
    const int jj = nc >> 1;
    float val = 0.f;
    if (ig < n && jj < r) {
      float2 v = V[ig * r + jj];
      const float br = tb.beta_r[gc], bi = tb.beta_i[gc];
      // beta conj(V) = (br vr + bi vi) + i (bi vr - br vi)
      val = (nc & 1) ? fmaf(bi, v.x, -br * v.y) : fmaf(br, v.x, bi * v.y);
    }
    h[k] = __float2bfloat16_rn(val);
  }
  *reinterpret_cast<uint4*>(b2 + (t * L::B2ROWS + within) * 8) = *reinterpret_cast<uint4*>(h);
}

// directions: candidate tile ct, chunk ch, row s: slots [Re c, Im c, 0...]
template <int KCH>
__global__ void pack_dirs_kernel(const float2* __restrict__ C, int64_t S, int r, int64_t c_tiles,
                                 __nv_bfloat16* __restrict__ ctp) {
  const int64_t total = c_tiles * kTcM;
  int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int64_t ct = q / kTcM;
  const int row = static_cast<int>(q % kTcM);
  float slot[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) slot[k] = 0.f;
  if (q < S) {
    for (int jj = 0; jj < r; ++jj) {
      float2 c = C[q * r + jj];
      slot[jj] = c.x;
      slot[r + jj] = c.y;
    }
  }
#pragma unroll
  for (int ch = 0; ch < KCH; ++ch) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = __float2bfloat16_rn(slot[ch * 8 + k]);
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
static int pack_impl(const ScorePlan& p, const Alphabet& a, const float2* V, const float2* C, void* vt, void* b2,
                     void* ct, cudaStream_t st) {
  using Sh = TcShape<K>;
  using L = TcLayout<K, KCH>;
  PackTables tb = make_pack_tables(a);
  int64_t nv = p.n_tiles * Sh::N1;
  pack_vaug_kernel<K, KCH><<<static_cast<unsigned>(ceil_div(nv, 256)), 256, 0, st>>>(
      V, p.n, p.r, p.n_tiles, tb, static_cast<__nv_bfloat16*>(vt));
  count_launch();
  int64_t nb = p.n_tiles * L::B2ROWS;
  pack_b2_kernel<K, KCH><<<static_cast<unsigned>(ceil_div(nb, 256)), 256, 0, st>>>(
      V, p.n, p.r, p.n_tiles, tb, static_cast<__nv_bfloat16*>(b2));
  count_launch();
  int64_t nc = p.c_tiles * kTcM;
  pack_dirs_kernel<KCH><<<static_cast<unsigned>(ceil_div(nc, 256)), 256, 0, st>>>(C, p.S, p.r, p.c_tiles,
                                                                                  static_cast<__nv_bfloat16*>(ct));
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
static int score_impl(const ScorePlan& p, const void* vt, const void* b2, const void* ct, double* partial,
                      int32_t* status, cudaStream_t st) {
  using Sh = TcShape<K>;
  using L = TcLayout<K, KCH>;
  CUtensorMap m_vt, m_b2, m_ct;
  int e;
  if ((e = make_rows_map(&m_vt, vt, static_cast<size_t>(p.n_tiles) * L::B1_BYTES, L::B1_BYTES))) return e;
  if ((e = make_rows_map(&m_b2, b2, static_cast<size_t>(p.n_tiles) * L::B2_BYTES, L::B2_BYTES))) return e;
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
  score_tc_kernel<K, KCH><<<grid, Sh::THREADS, L::TOTAL, st>>>(m_vt, m_b2, m_ct, prm, partial, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "score_tc_kernel");
}

int tc_rows_per_tile(int K) {
  switch (K) {
    case 2: return TcShape<2>::ROWS;
    case 3: return TcShape<3>::ROWS;
    case 4: return TcShape<4>::ROWS;
    case 5: return TcShape<5>::ROWS;
    case 6: return TcShape<6>::ROWS;
    case 7: return TcShape<7>::ROWS;
    case 8: return TcShape<8>::ROWS;
    default: return 0;
  }
}

int tc_workers_per_cta(int K) {
  switch (K) {
    case 2: return TcShape<2>::NW;
    case 3: return TcShape<3>::NW;
    case 4: return TcShape<4>::NW;
    case 5: return TcShape<5>::NW;
    case 6: return TcShape<6>::NW;
    case 7: return TcShape<7>::NW;
    case 8: return TcShape<8>::NW;
    default: return 1;
  }
}

size_t tc_bytes_vaug(int K, int r, int64_t n_tiles) {
  int kch = r <= 4 ? 1 : 2;
  int n1 = 0;
  switch (K) {
    case 2: n1 = TcShape<2>::N1; break;
    case 3: n1 = TcShape<3>::N1; break;
    case 4: n1 = TcShape<4>::N1; break;
    case 5: n1 = TcShape<5>::N1; break;
    case 6: n1 = TcShape<6>::N1; break;
    case 7: n1 = TcShape<7>::N1; break;
    case 8: n1 = TcShape<8>::N1; break;
    default: return 0;
  }
  return static_cast<size_t>(n_tiles) * kch * n1 * 16;
}

size_t tc_bytes_b2(int K, int r, int64_t n_tiles) {
  int n2r = r <= 4 ? 8 : 16;
  int g = (K % 2 == 0) ? K / 2 : K - 1;
  return static_cast<size_t>(n_tiles) * (g * tc_rows_per_tile(K) / 8) * n2r * 16;
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

int launch_tc_pack(const ScorePlan& p, const Alphabet& a, const float2* V, const float2* C, void* vt, void* b2,
                   void* ct, cudaStream_t st) {
  LRQ_TC_DISPATCH(pack_impl, p, a, V, C, vt, b2, ct, st);
}

int launch_score_tc(const ScorePlan& p, const Alphabet& a, const void* vt, const void* b2, const void* ct,
                    double* partial, int32_t* status, cudaStream_t st) {
  (void)a;
  LRQ_TC_DISPATCH(score_impl, p, vt, b2, ct, partial, status, st);
}

}  // namespace lrq
