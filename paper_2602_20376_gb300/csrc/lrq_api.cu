// lrq_api.cu -- the extern "C" entry points of liblrq (declared in
// include/lrq.h): argument validation, workspace planning, alphabet tables
// and the launch sequence of each call.  No entry point allocates device
// memory or synchronises the stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "lrq_internal.h"

namespace lrq {

int tc_rows_per_tile(int K, int r);
int tc_workers_per_cta(int K, int r);
size_t tc_bytes_tiles(int K, int r, int64_t n_tiles);
size_t tc_bytes_indicator_scale(int K, int r, int64_t n_tiles);
size_t tc_bytes_dirs(int r, int64_t c_tiles);

static thread_local char g_last_error[512] = {0};
static std::atomic<uint64_t> g_launches{0};
static thread_local cudaEvent_t g_t_start = nullptr;
static thread_local cudaEvent_t g_t_stop = nullptr;

void count_launch(int k) { g_launches.fetch_add(static_cast<uint64_t>(k), std::memory_order_relaxed); }

void timing_start(cudaStream_t st) {
  if (g_t_start) cudaEventRecord(g_t_start, st);
}

void timing_stop(cudaStream_t st) {
  if (g_t_stop) cudaEventRecord(g_t_stop, st);
}

void set_error(const std::string& msg) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg.c_str());
}

int fail(int status, const std::string& msg) {
  set_error(msg);
  return status;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LRQ_OK;
  return fail(LRQ_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The MLP's GEMMs tile the batch rows 32 at a time on the grid's y axis
// (at most 65535 blocks).
constexpr int kMaxMlpBatch = 65535 * 32;

int num_sms_current() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

static double snap(double v) { return std::fabs(v) < 1e-15 ? 0.0 : v; }

Alphabet make_alphabet(int K) {
  Alphabet a;
  std::memset(&a, 0, sizeof(a));
  a.K = K;
  a.BK = (K % 2 == 0) ? K / 2 : K;
  a.G = (K % 2 == 0) ? K / 2 : K - 1;
  for (int m = 0; m < K && m < kMaxK; ++m) {
    double th = kPi * (2.0 * m + 1.0) / K;  // decision boundary theta_m
    a.bcos64[m] = snap(std::cos(th));
    a.bsin64[m] = snap(std::sin(th));
    a.bcos[m] = static_cast<float>(a.bcos64[m]);
    a.bsin[m] = static_cast<float>(a.bsin64[m]);
    double ph = 2.0 * kPi * m / K;  // root omega^m
    a.zr64[m] = snap(std::cos(ph));
    a.zi64[m] = snap(std::sin(ph));
    a.zr[m] = static_cast<float>(a.zr64[m]);
    a.zi[m] = static_cast<float>(a.zi64[m]);
  }
  for (int g = 0; g < a.G && g < kMaxK; ++g) {
    if (K % 2 == 1) {  // odd K: indicator of class g+1, coefficient omega^{g+1} - 1
      a.beta_r[g] = a.zr64[g + 1] - 1.0;
      a.beta_i[g] = a.zi64[g + 1];
    } else {  // even K: sign of boundary g, coefficient (omega^{g+1} - omega^g) / 2
      double r1 = snap(std::cos(2.0 * kPi * (g + 1) / K)), i1 = snap(std::sin(2.0 * kPi * (g + 1) / K));
      a.beta_r[g] = 0.5 * (r1 - a.zr64[g]);
      a.beta_i[g] = 0.5 * (i1 - a.zi64[g]);
    }
  }
  return a;
}

static size_t take(size_t& cursor, size_t bytes) {
  size_t off = cursor;
  cursor = align_up(cursor + bytes, 256);
  return off;
}

int plan_score(int64_t n, int r, int K, int64_t S, int mode, int top_m, int num_sms, ScorePlan* p, bool with_prep) {
  std::memset(p, 0, sizeof(*p));
  p->n = n;
  p->S = S;
  p->r = r;
  p->K = K;
  p->mode = mode;
  p->top_m = top_m;
  p->c_tiles = ceil_div(S, 128);
  const int64_t S_pad = p->c_tiles * 128;
  if (mode == LRQ_MODE_BF16_TC) {
    p->rows_per_tile = tc_rows_per_tile(K, r);
    p->n_tiles = ceil_div(n, p->rows_per_tile);
    // coordinate chunks: balance (chunk, candidate tile) items over the
    // workers (num_sms CTAs x workers per CTA); of the splits within 1% of
    // the best balance take the fewest chunks (each chunk writes S x 2r FP64
    // partial sums)
    const int64_t workers = static_cast<int64_t>(num_sms) * tc_workers_per_cta(K, r);
    double eff_of[65];
    double best_eff = -1.0;
    const int ns_max = static_cast<int>(std::min<int64_t>(64, p->n_tiles));
    for (int ns = 1; ns <= ns_max; ++ns) {
      int64_t tpc = ceil_div(p->n_tiles, ns);
      int64_t ns_eff = ceil_div(p->n_tiles, tpc);
      int64_t items = p->c_tiles * ns_eff;
      int64_t waves = ceil_div(items, workers);
      double eff = static_cast<double>(items) / static_cast<double>(waves * workers);
      // a longer chunk amortises the pipeline fill of an item
      eff *= static_cast<double>(tpc) / static_cast<double>(tpc + 2);
      eff_of[ns] = eff;
      best_eff = std::max(best_eff, eff);
    }
    int best_ns = 1;
    while (best_ns < ns_max && eff_of[best_ns] < best_eff - 0.01) ++best_ns;
    p->tiles_per_chunk = ceil_div(p->n_tiles, best_ns);
    p->nsplit = static_cast<int>(ceil_div(p->n_tiles, p->tiles_per_chunk));
    p->npart = p->nsplit;
  } else {
    p->fp32_block = 256;
    int64_t blocks_x = ceil_div(S, 256);
    int64_t want = std::max<int64_t>(1, ceil_div(int64_t(8) * num_sms, blocks_x));
    want = std::min<int64_t>(want, 64);
    int64_t rows = align_up(static_cast<size_t>(ceil_div(n, want)), 256);
    p->fp32_rows_per_chunk = std::max<int64_t>(rows, 256);
    p->nsplit = static_cast<int>(ceil_div(n, p->fp32_rows_per_chunk));
    p->npart = p->nsplit;
  }
  size_t cur = 0;
  p->sz_partial = static_cast<size_t>(p->npart) * S_pad * 2 * r * sizeof(double);
  p->off_partial = take(cur, p->sz_partial);
  if (with_prep) {
    p->sz_T = 2 * kMaxRank * sizeof(double);
    p->off_T = take(cur, p->sz_T);
    p->sz_Tpart = 256 * 2 * kMaxRank * sizeof(double);
    p->off_Tpart = take(cur, p->sz_Tpart);
  }
  if (mode == LRQ_MODE_BF16_TC) {
    if (with_prep) {
      p->sz_tiles = tc_bytes_tiles(K, r, p->n_tiles);
      p->off_tiles = take(cur, p->sz_tiles);
    }
    p->sz_ct = tc_bytes_dirs(r, p->c_tiles);
    p->off_ct = take(cur, p->sz_ct);
    if (with_prep) {
      p->sz_scale = 4 * sizeof(float);
      p->off_scale = take(cur, p->sz_scale);
      p->sz_iw = tc_bytes_indicator_scale(K, r, p->n_tiles);
      p->off_iw = take(cur, p->sz_iw);
    }
  }
  p->sz_scores = static_cast<size_t>(S) * sizeof(float);
  p->off_scores = take(cur, p->sz_scores);
  p->sz_keys = (static_cast<size_t>(S) + topm_scratch_keys(S, top_m)) * sizeof(uint64_t);
  p->off_keys = take(cur, p->sz_keys);
  p->total = cur;
  return LRQ_OK;
}

int plan_prepare(int64_t n, int r, int K, int mode, PrepLayout* L) {
  std::memset(L, 0, sizeof(*L));
  if (mode != LRQ_MODE_BF16_TC) return LRQ_OK;  // the FP32 path reads V itself
  L->n_tiles = ceil_div(n, tc_rows_per_tile(K, r));
  size_t cur = 0;
  L->off_T = take(cur, 2 * kMaxRank * sizeof(double));
  L->off_Tpart = take(cur, 256 * 2 * kMaxRank * sizeof(double));
  L->off_tiles = take(cur, tc_bytes_tiles(K, r, L->n_tiles));
  L->off_scale = take(cur, 4 * sizeof(float));
  L->off_iw = take(cur, tc_bytes_indicator_scale(K, r, L->n_tiles));
  L->total = cur;
  return LRQ_OK;
}

int plan_rescore(int64_t n, int r, int m, RescorePlan* p) {
  std::memset(p, 0, sizeof(*p));
  p->n = n;
  p->r = r;
  p->m = m;
  // blocks of (candidates x coordinate chunk): about four per SM, at most
  // 65536 rows per chunk (which bounds the scratch: m x nchunk x 2 kMaxRank
  // doubles), at least one staged tile of 256 rows per chunk
  const int64_t max_rows = int64_t(65536);
  const int64_t bx = rescore_blocks_x(m);
  int64_t nchunk = std::max<int64_t>(ceil_div(int64_t(4) * num_sms_current(), bx), ceil_div(n, max_rows));
  nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, std::max<int64_t>(1, ceil_div(n, 256))));
  nchunk = std::min<int64_t>(nchunk, 65535);  // grid y limit; longer chunks are fine (periodic FP64 flushes)
  p->rows_per_chunk = ceil_div(n, nchunk);
  p->nchunk = static_cast<int>(ceil_div(n, p->rows_per_chunk));
  size_t cur = 0;
  p->sz_part = static_cast<size_t>(m) * p->nchunk * 2 * kMaxRank * sizeof(double);
  p->off_part = take(cur, p->sz_part);
  p->total = cur;
  return LRQ_OK;
}

static int check_ws(const void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return LRQ_OK;
  if (ws == nullptr) return fail(LRQ_EWORKSPACE, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(LRQ_EWORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < need)
    return fail(LRQ_EWORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, got " +
                                    std::to_string(ws_bytes));
  return LRQ_OK;
}

static int check_score_args(int64_t n, int r, int K, int64_t S, int mode, int top_m) {
  if (n < 1) return fail(LRQ_EINVAL, "n must be >= 1");
  if (r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "r must be in [1, 8]");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (S < 1 || S >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "S must be in [1, 2^31)");
  if (mode != LRQ_MODE_FP32 && mode != LRQ_MODE_BF16_TC) return fail(LRQ_EINVAL, "unknown mode");
  if (top_m < 1 || top_m > kMaxTopM || top_m > S) return fail(LRQ_EINVAL, "top_m must be in [1, min(512, S)]");
  if (mode == LRQ_MODE_BF16_TC && K > kMaxTcK)
    return fail(LRQ_EUNSUPPORTED, "the tensor-core mode supports 2 <= K <= 8");
  if (n > (int64_t(1) << 40)) return fail(LRQ_EUNSUPPORTED, "n too large");
  return LRQ_OK;
}

// What scoring needs of one instance V, independent of the directions.
struct InstanceOperands {
  const float2* V;
  uint8_t* tiles;   // packed coordinate tiles (tensor-core mode)
  float* scale;     // GEMM2 operand scale
  uint8_t* iw;      // indicator magnitudes
  double* T;        // column sums of conj(V) (odd K, tensor-core mode)
  double* Tpart;    // their per-block partials
};

static int prepare_operands(const ScorePlan& p, const Alphabet& a, const InstanceOperands& io, int32_t* dev_status,
                            cudaStream_t st) {
  int e;
  if ((e = launch_check_finite(reinterpret_cast<const float*>(io.V), 2 * p.n * p.r, dev_status, st))) return e;
  if (p.mode != LRQ_MODE_BF16_TC) return LRQ_OK;
  if (p.K % 2 == 1) {
    int nb = static_cast<int>(std::min<int64_t>(256, std::max<int64_t>(1, ceil_div(p.n, 4096))));
    if ((e = launch_colsum(io.V, p.n, p.r, io.Tpart, io.T, nb, st))) return e;
  }
  return launch_tc_pack_v(p, a, io.V, io.tiles, io.scale, io.iw, st);
}

// Directions -> scores -> top-m, on prepared operands; w is the per-call
// workspace laid out by p.
static int score_directions(const ScorePlan& p, const Alphabet& a, const InstanceOperands& io, float2* Cf,
                            bool generate, uint64_t seed, uint8_t* w, float* scores_out, int64_t* top_idx_out,
                            float* top_f_out, int32_t* dev_status, cudaStream_t st) {
  int e;
  double* partial = reinterpret_cast<double*>(w + p.off_partial);
  float* scores = scores_out ? scores_out : reinterpret_cast<float*>(w + p.off_scores);
  uint64_t* keys = reinterpret_cast<uint64_t*>(w + p.off_keys);
  uint64_t* keys_scratch = keys + p.S;
  if (generate && (e = launch_sample_directions(seed, p.S, p.r, Cf, st))) return e;
  if ((e = launch_check_finite(reinterpret_cast<const float*>(Cf), 2 * p.S * p.r, dev_status, st))) return e;
  const double* Tuse = nullptr;
  if (p.mode == LRQ_MODE_BF16_TC) {
    if (p.K % 2 == 1) Tuse = io.T;
    if ((e = launch_tc_pack_dirs(p, Cf, w + p.off_ct, st))) return e;
    timing_start(st);
    if ((e = launch_score_tc(p, a, io.tiles, w + p.off_ct, io.scale, io.iw, partial, dev_status, st))) return e;
    timing_stop(st);
  } else {
    timing_start(st);
    if ((e = launch_score_fp32(p, a, io.V, Cf, partial, st))) return e;
    timing_stop(st);
  }
  if ((e = launch_finalize(p, a, partial, Tuse, scores, keys, st))) return e;
  return launch_topm(keys, p.S, p.top_m, keys_scratch, top_idx_out, top_f_out, st);
}

}  // namespace lrq

// A prepared instance (host object; its device buffer is the caller's).
struct lrq_prepared_v {
  int64_t n;
  int r, K, mode;
  lrq::PrepLayout L;
  const float2* V;
  uint8_t* buf;
  bool ready;
};

using namespace lrq;

extern "C" {

const char* lrq_status_string(int status) {
  switch (status) {
    case LRQ_OK: return "LRQ_OK";
    case LRQ_EINVAL: return "LRQ_EINVAL: invalid argument or non-finite input";
    case LRQ_EUNSUPPORTED: return "LRQ_EUNSUPPORTED: unsupported size, alphabet, rank or mode";
    case LRQ_ECUDA: return "LRQ_ECUDA: CUDA runtime error";
    case LRQ_ETIMEOUT: return "LRQ_ETIMEOUT: a bounded device wait ran out";
    case LRQ_ENOCONV: return "LRQ_ENOCONV: iterative solver did not converge";
    case LRQ_EWORKSPACE: return "LRQ_EWORKSPACE: workspace missing, misaligned or too small";
    default: return "LRQ_UNKNOWN";
  }
}

const char* lrq_last_error(void) { return g_last_error; }

int lrq_abi_version(void) { return 1; }

int lrq_sample_directions(uint64_t seed, int64_t S, int r, void* C_out, void* stream) {
  if (S < 0) return fail(LRQ_EINVAL, "S must be >= 0");
  if (r < 1 || r > kMaxK) return fail(LRQ_EINVAL, "r must be in [1, 64]");
  if (S > 0 && C_out == nullptr) return fail(LRQ_EINVAL, "C_out is NULL");
  return launch_sample_directions(seed, S, r, static_cast<float2*>(C_out), static_cast<cudaStream_t>(stream));
}

int lrq_sample_score_workspace_size(int64_t n, int r, int K, int64_t S, int mode, int top_m, size_t* bytes) {
  if (!bytes) return fail(LRQ_EINVAL, "bytes is NULL");
  int e = check_score_args(n, r, K, S, mode, top_m);
  if (e) return e;
  ScorePlan p;
  plan_score(n, r, K, S, mode, top_m, num_sms_current(), &p);
  *bytes = p.total;
  return LRQ_OK;
}

int lrq_sample_score(const void* V, int64_t n, int r, int K, void* C, int generate_C, uint64_t seed, int64_t S,
                     int mode, int top_m, float* scores_out, int64_t* top_idx_out, float* top_f_out, void* ws,
                     size_t ws_bytes, int32_t* dev_status, void* stream) {
  int e = check_score_args(n, r, K, S, mode, top_m);
  if (e) return e;
  if (!V || !C || !top_idx_out || !top_f_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  ScorePlan p;
  plan_score(n, r, K, S, mode, top_m, num_sms_current(), &p);
  if ((e = check_ws(ws, ws_bytes, p.total))) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(ws);
  InstanceOperands io{static_cast<const float2*>(V), w + p.off_tiles, reinterpret_cast<float*>(w + p.off_scale),
                      w + p.off_iw, reinterpret_cast<double*>(w + p.off_T), reinterpret_cast<double*>(w + p.off_Tpart)};
  const Alphabet a = make_alphabet(K);
  if ((e = prepare_operands(p, a, io, dev_status, st))) return e;
  return score_directions(p, a, io, static_cast<float2*>(C), generate_C != 0, seed, w, scores_out, top_idx_out,
                          top_f_out, dev_status, st);
}

int lrq_prepared_create(int64_t n, int r, int K, int mode, lrq_prepared_v** out) {
  if (!out) return fail(LRQ_EINVAL, "out is NULL");
  *out = nullptr;
  int e = check_score_args(n, r, K, 1, mode, 1);
  if (e) return e;
  lrq_prepared_v* h = new (std::nothrow) lrq_prepared_v();
  if (!h) return fail(LRQ_EINVAL, "host allocation failed");
  h->n = n;
  h->r = r;
  h->K = K;
  h->mode = mode;
  plan_prepare(n, r, K, mode, &h->L);
  h->V = nullptr;
  h->buf = nullptr;
  h->ready = false;
  *out = h;
  return LRQ_OK;
}

void lrq_prepared_destroy(lrq_prepared_v* h) { delete h; }

int lrq_prepared_size(const lrq_prepared_v* h, size_t* bytes) {
  if (!h || !bytes) return fail(LRQ_EINVAL, "NULL argument");
  *bytes = h->L.total;
  return LRQ_OK;
}

int lrq_prepare(lrq_prepared_v* h, const void* V, void* buf, size_t buf_bytes, int32_t* dev_status, void* stream) {
  if (!h || !V || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  int e = check_ws(buf, buf_bytes, h->L.total);
  if (e) return e;
  h->ready = false;
  ScorePlan p;
  plan_score(h->n, h->r, h->K, 1, h->mode, 1, num_sms_current(), &p, false);
  uint8_t* b = static_cast<uint8_t*>(buf);
  InstanceOperands io{static_cast<const float2*>(V), b + h->L.off_tiles, reinterpret_cast<float*>(b + h->L.off_scale),
                      b + h->L.off_iw, reinterpret_cast<double*>(b + h->L.off_T),
                      reinterpret_cast<double*>(b + h->L.off_Tpart)};
  if ((e = prepare_operands(p, make_alphabet(h->K), io, dev_status, static_cast<cudaStream_t>(stream)))) return e;
  h->V = static_cast<const float2*>(V);
  h->buf = b;
  h->ready = true;
  return LRQ_OK;
}

int lrq_sample_score_prepared_workspace_size(const lrq_prepared_v* h, int64_t S, int top_m, size_t* bytes) {
  if (!h || !bytes) return fail(LRQ_EINVAL, "NULL argument");
  int e = check_score_args(h->n, h->r, h->K, S, h->mode, top_m);
  if (e) return e;
  ScorePlan p;
  plan_score(h->n, h->r, h->K, S, h->mode, top_m, num_sms_current(), &p, false);
  *bytes = p.total;
  return LRQ_OK;
}

int lrq_sample_score_prepared(const lrq_prepared_v* h, void* C, int generate_C, uint64_t seed, int64_t S, int top_m,
                              float* scores_out, int64_t* top_idx_out, float* top_f_out, void* ws, size_t ws_bytes,
                              int32_t* dev_status, void* stream) {
  if (!h) return fail(LRQ_EINVAL, "handle is NULL");
  if (!h->ready) return fail(LRQ_EINVAL, "instance not prepared (call lrq_prepare first)");
  int e = check_score_args(h->n, h->r, h->K, S, h->mode, top_m);
  if (e) return e;
  if (!C || !top_idx_out || !top_f_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  ScorePlan p;
  plan_score(h->n, h->r, h->K, S, h->mode, top_m, num_sms_current(), &p, false);
  if ((e = check_ws(ws, ws_bytes, p.total))) return e;
  uint8_t* b = h->buf;
  InstanceOperands io{h->V, b + h->L.off_tiles, reinterpret_cast<float*>(b + h->L.off_scale), b + h->L.off_iw,
                      reinterpret_cast<double*>(b + h->L.off_T), reinterpret_cast<double*>(b + h->L.off_Tpart)};
  return score_directions(p, make_alphabet(h->K), io, static_cast<float2*>(C), generate_C != 0, seed,
                          static_cast<uint8_t*>(ws), scores_out, top_idx_out, top_f_out, dev_status,
                          static_cast<cudaStream_t>(stream));
}

int lrq_rescore_workspace_size(int64_t n, int r, int m, size_t* bytes) {
  if (!bytes) return fail(LRQ_EINVAL, "bytes is NULL");
  if (n < 1 || r < 1 || r > kMaxRank || m < 1 || m > kMaxRescoreM) return fail(LRQ_EINVAL, "bad sizes");
  RescorePlan p;
  plan_rescore(n, r, m, &p);
  *bytes = p.total;
  return LRQ_OK;
}

int lrq_rescore(const void* V, int64_t n, int r, int K, const void* C, int64_t S, const int64_t* idx, int m,
                double* f_out, uint8_t* z_out, int64_t* best_out, double* best_f_out, void* ws, size_t ws_bytes,
                int32_t* dev_status, void* stream) {
  if (n < 1) return fail(LRQ_EINVAL, "n must be >= 1");
  if (r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "r must be in [1, 8]");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (m < 1 || m > kMaxRescoreM) return fail(LRQ_EINVAL, "m must be in [1, 4096]");
  if (S < 1) return fail(LRQ_EINVAL, "S must be >= 1");
  if (!V || !C || !idx || !f_out || !best_out || !best_f_out || !dev_status)
    return fail(LRQ_EINVAL, "NULL pointer argument");
  RescorePlan p;
  plan_rescore(n, r, m, &p);
  int e = check_ws(ws, ws_bytes, p.total);
  if (e) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(ws);
  Alphabet a = make_alphabet(K);
  if ((e = launch_check_finite(reinterpret_cast<const float*>(V), 2 * n * r, dev_status, st))) return e;
  return launch_rescore(p, a, static_cast<const float2*>(V), static_cast<const float2*>(C), S, idx,
                        reinterpret_cast<double*>(w + p.off_part), f_out, z_out, best_out, best_f_out, dev_status,
                        st);
}

int lrq_truncate_workspace_size(const lrq_matrix* Q, int r, int max_iter, size_t* bytes) {
  if (!bytes) return fail(LRQ_EINVAL, "bytes is NULL");
  int e = truncate_check(Q, r, max_iter);
  if (e) return e;
  *bytes = truncate_workspace_bytes(Q, r, max_iter);
  return LRQ_OK;
}

int lrq_truncate(const lrq_matrix* Q, int r, double tol, int max_iter, uint64_t seed, void* V_out, void* V32_out,
                 double* lambda_out, int64_t* iters_out, void* ws, size_t ws_bytes, int32_t* dev_status,
                 void* stream) {
  int e = truncate_check(Q, r, max_iter);
  if (e) return e;
  if (!lambda_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  if (!(tol < 1.0) || tol != tol) return fail(LRQ_EINVAL, "tol must be below 1");
  if ((e = check_ws(ws, ws_bytes, truncate_workspace_bytes(Q, r, max_iter)))) return e;
  return launch_truncate(Q, r, tol, max_iter, seed, static_cast<double2*>(V_out), static_cast<float2*>(V32_out),
                         lambda_out, iters_out, ws, dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_proposal_num_features(int r) { return (r >= 1 && r <= kMaxRank) ? 5 * r + 4 : -1; }

int64_t lrq_proposal_num_params(int F) { return F >= 1 ? proposal_num_params(F) : -1; }

int lrq_proposal_features(const void* V, int B, int64_t n, int r, const double* lambda, void* Vg_out,
                          float* feat_out, int32_t* dev_status, void* stream) {
  if (B < 1 || n < 1 || r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "bad sizes");
  if (!V || !lambda || !Vg_out || !feat_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_features(static_cast<const float2*>(V), B, n, r, lambda, static_cast<float2*>(Vg_out), feat_out,
                         dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_mlp_forward(const float* params, int F, int B, const float* X, float* H1, float* H2, float* O, int bf16,
                    void* stream) {
  if (F < 1 || B < 1) return fail(LRQ_EINVAL, "bad sizes");
  if (B > kMaxMlpBatch) return fail(LRQ_EUNSUPPORTED, "at most 2097120 rows per MLP call");
  if (!params || !X || !H1 || !H2 || !O) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_mlp_forward(params, F, B, X, H1, H2, O, bf16 ? 1 : 0, static_cast<cudaStream_t>(stream));
}

int lrq_mlp_backward(const float* params, int F, int B, const float* X, const float* H1, const float* H2,
                     const float* dO, float* grads, float* scratch, int bf16, void* stream) {
  if (F < 1 || B < 1) return fail(LRQ_EINVAL, "bad sizes");
  if (B > kMaxMlpBatch) return fail(LRQ_EUNSUPPORTED, "at most 2097120 rows per MLP call");
  if (!params || !X || !H1 || !H2 || !dO || !grads || !scratch) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_mlp_backward(params, F, B, X, H1, H2, dO, grads, scratch, bf16 ? 1 : 0,
                             static_cast<cudaStream_t>(stream));
}

int lrq_vmf_nll(const float* O, int B, const float* targets, int T, double* loss_out, float* dO, void* stream) {
  if (B < 1 || T < 1) return fail(LRQ_EINVAL, "bad sizes");
  if (!O || !targets || !loss_out || !dO) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_vmf_nll(O, B, targets, T, loss_out, dO, static_cast<cudaStream_t>(stream));
}

int lrq_vmf_sample(const float* O, int B, int S, int K, uint64_t seed, void* C_out, int32_t* dev_status,
                   void* stream) {
  if (B < 1 || S < 1 || B > 65535) return fail(LRQ_EINVAL, "bad sizes");
  if (K < 1 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [1, 64]");
  if (!O || !C_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_vmf_sample(O, B, S, K, seed, static_cast<float2*>(C_out), dev_status,
                           static_cast<cudaStream_t>(stream));
}

int lrq_vmf_modes(const float* O, int B, void* C_out, void* stream) {
  if (B < 1) return fail(LRQ_EINVAL, "B must be >= 1");
  if (B > 65535) return fail(LRQ_EUNSUPPORTED, "B above 65535");
  if (!O || !C_out) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_vmf_modes(O, B, static_cast<float2*>(C_out), static_cast<cudaStream_t>(stream));
}

int lrq_adam_step(float* params, const float* grads, float* m, float* v, int64_t count, int t, float lr,
                  float beta1, float beta2, float eps, void* stream) {
  if (count < 0 || t < 1) return fail(LRQ_EINVAL, "count must be >= 0 and t >= 1");
  if (count > 0 && (!params || !grads || !m || !v)) return fail(LRQ_EINVAL, "NULL pointer argument");
  if (count == 0) return LRQ_OK;
  return launch_adam(params, grads, m, v, count, t, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream));
}

int lrq_proposal_targets(const void* C, int64_t S, int r, int K, const int64_t* idx, int64_t m, float* targets_out,
                         int32_t* dev_status, void* stream) {
  if (S < 1 || m < 0 || r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "bad sizes");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (m == 0) return LRQ_OK;
  if (!C || !idx || !targets_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_proposal_targets(static_cast<const float2*>(C), S, idx, m, r, K, targets_out, dev_status,
                                 static_cast<cudaStream_t>(stream));
}

int lrq_standardize_fit(const float* feat, int B, int F, float* mean_out, float* std_out, void* stream) {
  if (B < 1 || F < 1) return fail(LRQ_EINVAL, "bad sizes");
  if (!feat || !mean_out || !std_out) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_standardize_fit(feat, B, F, mean_out, std_out, static_cast<cudaStream_t>(stream));
}

int lrq_standardize(const float* feat, int B, int F, const float* mean, const float* std_dev, float* X_out,
                    void* stream) {
  if (B < 1 || F < 1) return fail(LRQ_EINVAL, "bad sizes");
  if (!feat || !mean || !std_dev || !X_out) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_standardize(feat, B, F, mean, std_dev, X_out, static_cast<cudaStream_t>(stream));
}

int lrq_rank1_workspace_size(int64_t n, size_t* bytes) {
  if (!bytes) return fail(LRQ_EINVAL, "bytes is NULL");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "n must be in [1, 2^31)");
  *bytes = rank1_workspace_bytes(n);
  return LRQ_OK;
}

int lrq_rank1_sweep(const void* q, int64_t n, int K, uint8_t* z_out, double* f_out, const int32_t* rowptr,
                    const int32_t* colidx, int64_t nnz, int64_t* cut_out, uint8_t* zcut_out, void* ws,
                    size_t ws_bytes, int32_t* dev_status, void* stream) {
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "n must be in [1, 2^31)");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (!q || !z_out || !f_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  if (rowptr && (!colidx || !cut_out || !zcut_out || nnz < 0)) return fail(LRQ_EINVAL, "incomplete graph arguments");
  int e = check_ws(ws, ws_bytes, rank1_workspace_bytes(n));
  if (e) return e;
  return launch_rank1(static_cast<const double2*>(q), n, K, z_out, f_out, rowptr, colidx, nnz, cut_out, zcut_out,
                      ws, dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_two_eigvec_q(const void* V, int64_t n, int r, const double* lambda, void* q_out, void* stream) {
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "n must be in [1, 2^31)");
  if (r < 2) return fail(LRQ_EINVAL, "r must be >= 2");
  if (!V || !lambda || !q_out) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_two_eigvec_q(static_cast<const double2*>(V), n, r, lambda, static_cast<double2*>(q_out),
                             static_cast<cudaStream_t>(stream));
}

int lrq_sample_null_directions(const void* V, int64_t n, int r, int K, uint64_t seed, int64_t S, void* C_out,
                               int64_t* draws_out, int32_t* dev_status, void* stream) {
  if (n < 1 || S < 1 || S >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "need n >= 1 and 1 <= S < 2^31");
  if (r < 1 || r > kMaxRank) return fail(LRQ_EINVAL, "r must be in [1, 8]");
  if (K < 2 || K > kMaxK) return fail(LRQ_EINVAL, "K must be in [2, 64]");
  if (n * static_cast<int64_t>(K) < 2 * r - 1) return fail(LRQ_EINVAL, "fewer augmented rows than 2r - 1");
  if (!V || !C_out || !draws_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_null_sample(static_cast<const float2*>(V), n, r, K, seed, S, static_cast<float2*>(C_out), draws_out,
                            dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_spectral_energy(const lrq_matrix* Q, const double* lambda, int r, double* trace_out, double* rho_out,
                        int32_t* dev_status, void* stream) {
  if (!Q) return fail(LRQ_EINVAL, "Q is NULL");
  if (Q->kind != LRQ_MATRIX_DENSE_C128 && Q->kind != LRQ_MATRIX_CSR_LAPLACIAN)
    return fail(LRQ_EINVAL, "unknown matrix kind");
  if (Q->n < 1 || Q->n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "n must be in [1, 2^31)");
  if (r < 0) return fail(LRQ_EINVAL, "r must be >= 0");
  if ((r > 0 && !lambda) || !trace_out || !rho_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  if (Q->kind == LRQ_MATRIX_DENSE_C128) {
    if (!Q->values || Q->ld < Q->n) return fail(LRQ_EINVAL, "dense values NULL or ld < n");
  } else {
    if (!Q->rowptr || (Q->nnz > 0 && !Q->colidx)) return fail(LRQ_EINVAL, "CSR pointer is NULL");
    if (Q->nnz < 0 || Q->nnz >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "nnz must be in [0, 2^31)");
  }
  return launch_spectral_energy(Q, lambda, r, trace_out, rho_out, dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_greedy_workspace_size(int64_t n, size_t* bytes) {
  if (!bytes) return fail(LRQ_EINVAL, "bytes is NULL");
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "n must be in [1, 2^31)");
  *bytes = greedy_workspace_bytes(n);
  return LRQ_OK;
}

int lrq_greedy_cut(const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz, int K, uint8_t* z,
                   int64_t max_rounds, int64_t* cut_out, int64_t* rounds_out, int64_t* moves_out,
                   int32_t* converged_out, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream) {
  if (n < 1 || n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "n must be in [1, 2^31)");
  if (K < 2 || K > 8) return fail(LRQ_EINVAL, "K must be in [2, 8]");
  if (nnz < 0 || max_rounds < 0) return fail(LRQ_EINVAL, "nnz and max_rounds must be >= 0");
  if (!rowptr || (nnz > 0 && !colidx) || !z || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  int e = check_ws(ws, ws_bytes, greedy_workspace_bytes(n));
  if (e) return e;
  return launch_greedy(rowptr, colidx, n, nnz, K, z, max_rounds, cut_out, rounds_out, moves_out, converged_out, ws,
                       dev_status, static_cast<cudaStream_t>(stream));
}

int lrq_enumerate_workspace_size(int64_t n, int r, int K, size_t* bytes) {
  if (!bytes) return fail(LRQ_EINVAL, "bytes is NULL");
  int e = enumerate_check(n, r, K, 1e300);
  if (e) return e;
  *bytes = enum_workspace_bytes(n, r);
  return LRQ_OK;
}

int lrq_enumerate(const void* V, int64_t n, int r, int K, double budget, uint8_t* z_out, double* f_out,
                  int64_t* n_sets_out, void* ws, size_t ws_bytes, int32_t* dev_status, void* stream) {
  int e = enumerate_check(n, r, K, budget);
  if (e) return e;
  if (!V || !z_out || !f_out || !dev_status) return fail(LRQ_EINVAL, "NULL pointer argument");
  if ((e = check_ws(ws, ws_bytes, enum_workspace_bytes(n, r)))) return e;
  return launch_enumerate(static_cast<const double2*>(V), n, r, K, z_out, f_out, n_sets_out, ws, dev_status,
                          static_cast<cudaStream_t>(stream));
}

int lrq_cut_count(const int32_t* rowptr, const int32_t* colidx, int64_t n, const uint8_t* z, int64_t* cut_out,
                  void* stream) {
  if (n < 0) return fail(LRQ_EINVAL, "n must be >= 0");
  if (!cut_out || (n > 0 && (!rowptr || !colidx || !z))) return fail(LRQ_EINVAL, "NULL pointer argument");
  return launch_cut_count(rowptr, colidx, n, z, cut_out, static_cast<cudaStream_t>(stream));
}

int lrq_set_timing_events(void* start_event, void* stop_event) {
  if ((start_event == nullptr) != (stop_event == nullptr))
    return fail(LRQ_EINVAL, "pass both timing events or neither");
  g_t_start = static_cast<cudaEvent_t>(start_event);
  g_t_stop = static_cast<cudaEvent_t>(stop_event);
  return LRQ_OK;
}

uint64_t lrq_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
