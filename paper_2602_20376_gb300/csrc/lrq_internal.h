// lrq_internal.h -- shared declarations of the CUDA library (not part of the
// public ABI).  Host launch helpers for every kernel translation unit, the
// workspace planner, device status helpers and the alphabet tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lrq.h"  // include/ is on the compiler include path

namespace lrq {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kMaxRank = 8;         // r supported by the scoring kernels
constexpr int kMaxK = 64;           // alphabet sizes supported by FP32 / FP64 paths
constexpr int kMaxTcK = 8;          // alphabet sizes supported by the tensor-core path
constexpr int kMaxTopM = 512;
constexpr int kMaxRescoreM = 4096;

// Thread-local error message (lrq_last_error).
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);

// First device-side error wins.
__device__ __forceinline__ void dev_fail(int32_t* status, int code) {
  if (status) atomicCAS(reinterpret_cast<int*>(status), 0, code);
}

// Alphabet A_K and its decision boundaries (Sec. 2.3).  theta_m = pi(2m+1)/K,
// m = 0..B_K-1, with B_K = K/2 for even K and K for odd K (Definition 2.1).
// The boundary projection of w is p_m = Im(exp(-i theta_m) w)
//   = y cos(theta_m) - x sin(theta_m), positive on the counter-clockwise side.
struct Alphabet {
  int K;
  int BK;                  // distinct boundary lines
  int G;                   // tensor-core indicator columns per coordinate (K-1 odd, K/2 even)
  float bcos[kMaxK], bsin[kMaxK];     // boundary line directions, FP32 (|v| < 1e-7 -> 0)
  double bcos64[kMaxK], bsin64[kMaxK];
  float zr[kMaxK], zi[kMaxK];         // omega^k, FP32
  double zr64[kMaxK], zi64[kMaxK];    // omega^k, FP64
  double beta_r[kMaxK], beta_i[kMaxK];  // per-indicator coefficients (tensor path)
};
Alphabet make_alphabet(int K);

// Byte offsets into the caller's workspace.
struct ScorePlan {
  int64_t n, S;
  int r, K, mode, top_m;
  // tensor-core tiling
  int rows_per_tile;       // coordinates per pipeline stage
  int64_t n_tiles;         // ceil(n / rows_per_tile)
  int64_t c_tiles;         // ceil(S / 128)
  int nsplit;              // coordinate chunks
  int npart;               // partial-sum slabs (chunks x producers per chunk)
  int64_t tiles_per_chunk;
  // FP32 tiling
  int fp32_block;          // candidates per block
  int64_t fp32_rows_per_chunk;
  // workspace layout
  size_t off_partial, sz_partial;   // npart x S_pad x 2r doubles
  size_t off_T, sz_T;               // 2r doubles (column sums of conj(V), odd K)
  size_t off_Tpart, sz_Tpart;       // per-block partial column sums
  size_t off_tiles, sz_tiles;       // packed coordinate tiles: augmented rows (bf16) | class rows (FP8 hi | lo)
  size_t off_ct, sz_ct;             // packed directions (bf16)
  size_t off_scale, sz_scale;       // GEMM2 operand scale {2^g, 2^-g, max|V component|}
  size_t off_iw, sz_iw;             // per-coordinate indicator magnitudes (E4M3, 1 byte per coordinate)
  size_t off_scores, sz_scores;     // S floats (when the caller passes none)
  size_t off_keys, sz_keys;         // selection keys
  size_t total;
};
// with_prep = false leaves out the instance's operands (T, tiles, scale,
// indicator magnitudes): a prepared instance holds them (PrepLayout).
int plan_score(int64_t n, int r, int K, int64_t S, int mode, int top_m, int num_sms, ScorePlan* p,
               bool with_prep = true);

// Byte offsets into a prepared instance's buffer: what scoring needs of V
// that does not depend on the directions.
struct PrepLayout {
  int64_t n_tiles;
  size_t off_T, off_Tpart, off_tiles, off_scale, off_iw;
  size_t total;
};
int plan_prepare(int64_t n, int r, int K, int mode, PrepLayout* L);

struct RescorePlan {
  int64_t n;
  int r, m, nchunk;
  int64_t rows_per_chunk;
  size_t off_part, sz_part;  // m x nchunk x 2r doubles
  size_t total;
};
int plan_rescore(int64_t n, int r, int m, RescorePlan* p);
int rescore_blocks_x(int m);  // candidate blocks of the re-scoring grid

int num_sms_current();

// Kernel-launch accounting (lrq_kernel_launches) and the timing hook.
void count_launch(int k = 1);
void timing_start(cudaStream_t st);
void timing_stop(cudaStream_t st);

// ---- launch helpers (return lrq_status; never synchronise) -----------------
int launch_sample_directions(uint64_t seed, int64_t S, int r, float2* C, cudaStream_t st);
int launch_check_finite(const float* x, int64_t count, int32_t* status, cudaStream_t st);
int launch_colsum(const float2* V, int64_t n, int r, double* Tpart, double* T, int nblocks,
                  cudaStream_t st);
int launch_score_fp32(const ScorePlan& p, const Alphabet& a, const float2* V, const float2* C,
                      double* partial, cudaStream_t st);
int launch_finalize(const ScorePlan& p, const Alphabet& a, const double* partial, const double* T,
                    float* scores, uint64_t* keys, cudaStream_t st);
int launch_topm(const uint64_t* keys_in, int64_t count, int m, uint64_t* scratch, int64_t* top_idx,
                float* top_f, cudaStream_t st);
size_t topm_scratch_keys(int64_t count, int m);
int launch_rescore(const RescorePlan& p, const Alphabet& a, const float2* V, const float2* C,
                   int64_t S, const int64_t* idx, double* part, double* f_out, uint8_t* z_out,
                   int64_t* best_out, double* best_f_out, int32_t* status, cudaStream_t st);
int launch_cut_count(const int32_t* rowptr, const int32_t* colidx, int64_t n, const uint8_t* z,
                     int64_t* cut_out, cudaStream_t st);
// spectral truncation (FP64 Lanczos)
int truncate_check(const lrq_matrix* Q, int r, int max_iter);
size_t truncate_workspace_bytes(const lrq_matrix* Q, int r, int max_iter);
int launch_truncate(const lrq_matrix* Q, int r, double tol, int max_iter, uint64_t seed, double2* V, float2* V32,
                    double* lambda_out, int64_t* iters_out, void* ws, int32_t* status, cudaStream_t st);
// learned proposal
int64_t proposal_num_params(int F);
int launch_features(const float2* V, int B, int64_t n, int r, const double* lambda, float2* Vg, float* feat,
                    int32_t* status, cudaStream_t st);
int launch_mlp_forward(const float* params, int F, int B, const float* X, float* H1, float* H2, float* O, int bf16,
                       cudaStream_t st);
// C = act(op(A) op(B) + bias) (* mask > 0), BF16 operands, FP32 accumulation, tcgen05
void launch_mlp_gemm_tc(cudaStream_t st, int M, int N, int K, const float* A, int lda, int ta, const float* Bm,
                        int ldb, int tb, const float* bias, int relu, const float* mask, float* C, int ldc);
int launch_mlp_backward(const float* params, int F, int B, const float* X, const float* H1, const float* H2,
                        const float* dO, float* grads, float* scratch, int bf16, cudaStream_t st);
int launch_vmf_nll(const float* O, int B, const float* X, int T, double* loss, float* dO, cudaStream_t st);
int launch_vmf_sample(const float* O, int B, int S, int K, uint64_t seed, float2* C, int32_t* status,
                      cudaStream_t st);
int launch_vmf_modes(const float* O, int B, float2* C, cudaStream_t st);
int launch_adam(float* p, const float* g, float* m, float* v, int64_t count, int t, float lr, float b1, float b2,
                float eps, cudaStream_t st);
int launch_proposal_targets(const float2* C, int64_t S, const int64_t* idx, int64_t m, int r, int K, float* out,
                            int32_t* status, cudaStream_t st);
int launch_standardize_fit(const float* feat, int B, int F, float* mean, float* sd, cudaStream_t st);
int launch_standardize(const float* feat, int B, int F, const float* mean, const float* sd, float* X,
                       cudaStream_t st);
// exact rank-1 sweep (FP64)
size_t rank1_workspace_bytes(int64_t n);
int launch_rank1(const double2* q, int64_t n, int K, uint8_t* z_out, double* f_out, const int32_t* rowptr,
                 const int32_t* colidx, int64_t nnz, int64_t* cut_out, uint8_t* zcut_out, void* ws, int32_t* status,
                 cudaStream_t st);
int launch_two_eigvec_q(const double2* V, int64_t n, int r, const double* lambda, double2* q, cudaStream_t st);
// null-vector direction sampler
int launch_null_sample(const float2* V, int64_t n, int r, int K, uint64_t seed, int64_t S, float2* C,
                       int64_t* draws_out, int32_t* status, cudaStream_t st);
// spectral energy ratio
int launch_spectral_energy(const lrq_matrix* Q, const double* lambda, int r, double* trace_out, double* rho_out,
                           int32_t* status, cudaStream_t st);
// greedy local search (Max-K-Cut)
size_t greedy_workspace_bytes(int64_t n);
int launch_greedy(const int32_t* rowptr, const int32_t* colidx, int64_t n, int64_t nnz, int K, uint8_t* z,
                  int64_t max_rounds, int64_t* cut_out, int64_t* rounds_out, int64_t* moves_out,
                  int32_t* converged_out, void* ws, int32_t* status, cudaStream_t st);
// vertex enumeration (FP64)
int enumerate_check(int64_t n, int r, int K, double budget);
size_t enum_workspace_bytes(int64_t n, int r);
int launch_enumerate(const double2* V, int64_t n, int r, int K, uint8_t* z_out, double* f_out, int64_t* n_sets_out,
                     void* ws, int32_t* status, cudaStream_t st);
// tensor-core path
int launch_tc_pack_v(const ScorePlan& p, const Alphabet& a, const float2* V, void* tiles, void* scale, void* iw,
                     cudaStream_t st);
int launch_tc_pack_dirs(const ScorePlan& p, const float2* C, void* ct, cudaStream_t st);
int launch_score_tc(const ScorePlan& p, const Alphabet& a, const void* tiles, const void* ct, const void* scale,
                    const void* iw, double* partial, int32_t* status, cudaStream_t st);

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace lrq
