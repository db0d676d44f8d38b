// k_learned.cu -- the learned proposal: spectral features, a 3-layer MLP
// (forward, backward, Adam), and a mixture of von Mises-Fisher densities on
// S^7 (negative log-likelihood with its gradient, and sampling).  The paper
// has no learned component; the sampling it replaces is uniform on the
// sphere (Sec. 4.2), and the K-fold equivalence of directions (Sec. 2.3)
// lets targets live in one canonical window.
//
// Layouts: V is B x n x r complex64 (instance-major); parameters are one
// flat FP32 array W1 (F x 256), b1, W2 (256 x 256), b2, W3 (256 x 160), b3,
// each W row-major (in x out) so that a layer is y = x W + b.  In BF16 mode
// every GEMM operand is rounded to bfloat16 (round to nearest even) as it is
// staged in shared memory and the products accumulate in FP32, on the tensor
// cores (k_mlp_tc.cu); FP32 mode runs the CUDA-core GEMM below.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kWidth = 256;
constexpr int kComp = 16;
constexpr int kHead = 10;
constexpr int kOut = kComp * kHead;  // 160
constexpr int kDim = 8;              // S^7 in R^8 = C^4

// ---------------------------------------------------------------------------
// features (FP64): gauge, then eigenvalue shares and moments
// ---------------------------------------------------------------------------
__device__ double block_sum_f64(double v, double* red) {
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

// one block (256 threads) per instance
__global__ void __launch_bounds__(256) features_kernel(const float2* __restrict__ V, int64_t n, int r,
                                                       const double* __restrict__ lambda, float2* __restrict__ Vg,
                                                       float* __restrict__ feat, int32_t* status) {
  __shared__ double red[8];
  __shared__ unsigned long long red_key[8];
  __shared__ double s_ph_re[kMaxRank], s_ph_im[kMaxRank];
  const int b = blockIdx.x;
  const float2* Vb = V + static_cast<int64_t>(b) * n * r;
  const double* lam = lambda + static_cast<int64_t>(b) * r;
  const int F = 5 * r + 4;
  float* fo = feat + static_cast<int64_t>(b) * F;
  double total = 0.0;
  for (int j = 0; j < r; ++j) total += lam[j];
  if (!(total > 0.0)) {
    if (threadIdx.x == 0) dev_fail(status, LRQ_EINVAL);
    return;
  }
  // gauge: per column the entry of largest modulus (lowest row on ties)
  for (int j = 0; j < r; ++j) {
    // argmax of |V_ij|^2 with ties to the lower row
    double best = -1.0;
    int64_t brow = n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const float2 v = Vb[i * r + j];
      const double m2 = static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
      if (m2 > best) {
        best = m2;
        brow = i;
      }
    }
    for (int m = 16; m > 0; m >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, m);
      const int64_t orow = __shfl_xor_sync(0xffffffffu, brow, m);
      if (ob > best || (ob == best && orow < brow)) {
        best = ob;
        brow = orow;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = best;
      red_key[threadIdx.x >> 5] = static_cast<unsigned long long>(brow);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = red[0];
      int64_t br = static_cast<int64_t>(red_key[0]);
      for (int k = 1; k < static_cast<int>(blockDim.x >> 5); ++k) {
        const int64_t rr = static_cast<int64_t>(red_key[k]);
        if (red[k] > bb || (red[k] == bb && rr < br)) {
          bb = red[k];
          br = rr;
        }
      }
      const float2 a = Vb[br * r + j];
      const double am = sqrt(static_cast<double>(a.x) * a.x + static_cast<double>(a.y) * a.y);
      // multiply the column by |a| / a = conj(a) / |a|
      s_ph_re[j] = am > 0.0 ? a.x / am : 1.0;
      s_ph_im[j] = am > 0.0 ? -a.y / am : 0.0;
    }
    __syncthreads();
  }
  // gauge-fixed copy
  float2* Vo = Vg + static_cast<int64_t>(b) * n * r;
  for (int64_t t = threadIdx.x; t < n * r; t += blockDim.x) {
    const int j = static_cast<int>(t % r);
    const float2 v = Vb[t];
    const double re = v.x * s_ph_re[j] - v.y * s_ph_im[j];
    const double im = v.x * s_ph_im[j] + v.y * s_ph_re[j];
    Vo[t] = make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  if (threadIdx.x < r) fo[threadIdx.x] = static_cast<float>(lam[threadIdx.x] / total);
  // moments of a_i = ||V_i||^2 n / total and b_ij = |V_ij|^2 n / lambda_j:
  // q = 0 is a, q = 1 + j is column j
  for (int q = 0; q <= r; ++q) {
    const double scale = q == 0 ? static_cast<double>(n) / total : static_cast<double>(n) / lam[q - 1];
    double s1 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      double a = 0.0;
      for (int j = (q == 0 ? 0 : q - 1); j < (q == 0 ? r : q); ++j) {
        const float2 v = Vb[i * r + j];
        a += static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
      }
      s1 += a * scale;
    }
    const double mean = block_sum_f64(s1, red) / static_cast<double>(n);
    double s2 = 0.0, s3 = 0.0, s4 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      double a = 0.0;
      for (int j = (q == 0 ? 0 : q - 1); j < (q == 0 ? r : q); ++j) {
        const float2 v = Vb[i * r + j];
        a += static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y;
      }
      const double d = a * scale - mean;
      s2 += d * d;
      s3 += d * d * d;
      s4 += d * d * d * d;
    }
    const double var = block_sum_f64(s2, red) / static_cast<double>(n);
    const double m3 = block_sum_f64(s3, red) / static_cast<double>(n);
    const double m4 = block_sum_f64(s4, red) / static_cast<double>(n);
    if (threadIdx.x == 0) {
      float* o = fo + r + 4 * q;
      o[0] = static_cast<float>(mean);
      o[1] = static_cast<float>(var);
      o[2] = var > 0.0 ? static_cast<float>(m3 / (var * sqrt(var))) : 0.f;
      o[3] = var > 0.0 ? static_cast<float>(m4 / (var * var) - 3.0) : 0.f;
    }
  }
}

// ---------------------------------------------------------------------------
// GEMM for the MLP: C = act(op(A) op(B) + bias) [* mask > 0]
//   op(A): M x K (A stored M x K, or K x M when ta), op(B): K x N (B stored
//   K x N, or N x K when tb).  32 x 32 tiles, 256 threads, 2 x 2 per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(256) mlp_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       int ta, const float* __restrict__ Bm, int ldb, int tb,
                                                       const float* __restrict__ bias, int relu,
                                                       const float* __restrict__ mask, float* __restrict__ C,
                                                       int ldc, int bf16) {
  __shared__ float As[32][33], Bs[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int t = threadIdx.x; t < 32 * 32; t += 256) {
      const int i = t >> 5, k = t & 31;
      const int gr = row0 + i, gk = k0 + k;
      float a = 0.f;
      if (gr < M && gk < K) a = ta ? A[static_cast<int64_t>(gk) * lda + gr] : A[static_cast<int64_t>(gr) * lda + gk];
      As[i][k] = bf16 ? bf16_round(a) : a;
      const int gc = col0 + i;  // reuse i as the column for B
      float bv = 0.f;
      if (gc < N && gk < K) bv = tb ? Bm[static_cast<int64_t>(gc) * ldb + gk] : Bm[static_cast<int64_t>(gk) * ldb + gc];
      Bs[k][i] = bf16 ? bf16_round(bv) : bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float a0 = As[ty * 2][k], a1 = As[ty * 2 + 1][k];
      const float b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int gr = row0 + ty * 2 + u, gc = col0 + tx * 2 + v;
      if (gr >= M || gc >= N) continue;
      float x = acc[u][v] + (bias ? bias[gc] : 0.f);
      if (relu) x = fmaxf(x, 0.f);
      if (mask && !(mask[static_cast<int64_t>(gr) * ldc + gc] > 0.f)) x = 0.f;
      C[static_cast<int64_t>(gr) * ldc + gc] = x;
    }
}

// out[j] = sum_b G[b, j] (bias gradients), a thread per column, rows in order
__global__ void colsum_f32_kernel(const float* __restrict__ G, int B, int N, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += G[static_cast<int64_t>(b) * N + j];
  out[j] = s;
}

// ---------------------------------------------------------------------------
// vMF normaliser on S^7 (FP64): log I_nu by its power series for kappa <= 30
// and by the large-argument expansion above
// ---------------------------------------------------------------------------
__device__ double log_bessel_i_dev(int nu, double kappa) {
  if (kappa <= 30.0) {
    const double half = 0.5 * kappa;
    double fact = 1.0;
    for (int k = 2; k <= nu; ++k) fact *= k;
    double t = pow(half, static_cast<double>(nu)) / fact;
    double s = t;
    for (int k = 0; k < 500; ++k) {
      t *= half * half / (static_cast<double>(k + 1) * static_cast<double>(k + 1 + nu));
      s += t;
      if (t < 1e-18 * s) break;
    }
    return log(s);
  }
  const double mu = 4.0 * nu * nu;
  double s = 1.0, t = 1.0;
  for (int j = 1; j < 12; ++j) {
    const double o = 2.0 * j - 1.0;
    t *= -(mu - o * o) / (j * 8.0 * kappa);
    s += t;
  }
  return kappa - 0.5 * log(2.0 * kPi * kappa) + log(s);
}

struct CompParams {
  double mu[kComp][kDim];
  double unorm[kComp];
  double kappa[kComp];
  double sig[kComp];     // softplus'
  double logpi[kComp];
  double pi[kComp];
  double logc[kComp];
  double a8[kComp];
};

// threads 0..15 fill one component each; thread 0 normalises the weights
__device__ void head_params(const float* __restrict__ O, CompParams& cp) {
  const int m = threadIdx.x;
  if (m < kComp) {
    const float* o = O + m * kHead;
    double nrm = 0.0;
    for (int d = 0; d < kDim; ++d) nrm += static_cast<double>(o[d]) * o[d];
    nrm = sqrt(nrm);
    cp.unorm[m] = nrm;
    for (int d = 0; d < kDim; ++d) cp.mu[m][d] = nrm > 0.0 ? o[d] / nrm : (d == 0 ? 1.0 : 0.0);
    const double x = o[kDim];
    const double kap = x > 20.0 ? x : log1p(exp(x));
    cp.kappa[m] = kap;
    cp.sig[m] = 1.0 / (1.0 + exp(-x));
    const double li3 = log_bessel_i_dev(3, kap), li4 = log_bessel_i_dev(4, kap);
    cp.logc[m] = 3.0 * log(kap) - 4.0 * log(2.0 * kPi) - li3;
    cp.a8[m] = exp(li4 - li3);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = -INFINITY;
    for (int k = 0; k < kComp; ++k) mx = fmax(mx, static_cast<double>(O[k * kHead + kDim + 1]));
    double s = 0.0;
    for (int k = 0; k < kComp; ++k) s += exp(static_cast<double>(O[k * kHead + kDim + 1]) - mx);
    const double lse = mx + log(s);
    for (int k = 0; k < kComp; ++k) {
      cp.logpi[k] = O[k * kHead + kDim + 1] - lse;
      cp.pi[k] = exp(cp.logpi[k]);
    }
  }
  __syncthreads();
}

// Loss and gradient of the mean negative log-likelihood, one block per
// instance; gradient contributions summed in shared memory (FP64).
__global__ void __launch_bounds__(128) vmf_nll_kernel(const float* __restrict__ O, int B, const float* __restrict__ X,
                                                      int T, double* __restrict__ loss, float* __restrict__ dO) {
  __shared__ CompParams cp;
  __shared__ double g[kOut];
  __shared__ double lred[4];
  const int b = blockIdx.x;
  const float* Ob = O + static_cast<int64_t>(b) * kOut;
  for (int k = threadIdx.x; k < kOut; k += blockDim.x) g[k] = 0.0;
  head_params(Ob, cp);
  double lsum = 0.0;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const float* x = X + (static_cast<int64_t>(b) * T + t) * kDim;
    double xv[kDim];
    for (int d = 0; d < kDim; ++d) xv[d] = x[d];
    double dots[kComp], ell[kComp], mx = -INFINITY;
    for (int m = 0; m < kComp; ++m) {
      double s = 0.0;
      for (int d = 0; d < kDim; ++d) s += cp.mu[m][d] * xv[d];
      dots[m] = s;
      ell[m] = cp.logpi[m] + cp.logc[m] + cp.kappa[m] * s;
      mx = fmax(mx, ell[m]);
    }
    double se = 0.0;
    for (int m = 0; m < kComp; ++m) se += exp(ell[m] - mx);
    lsum += -(mx + log(se));
    for (int m = 0; m < kComp; ++m) {
      const double gam = exp(ell[m] - mx) / se;
      atomicAdd(&g[m * kHead + kDim + 1], cp.pi[m] - gam);
      atomicAdd(&g[m * kHead + kDim], -gam * (dots[m] - cp.a8[m]) * cp.sig[m]);
      const double c = -gam * cp.kappa[m] / cp.unorm[m];
      for (int d = 0; d < kDim; ++d) atomicAdd(&g[m * kHead + d], c * (xv[d] - dots[m] * cp.mu[m][d]));
    }
  }
  const double ls = block_sum_f64(lsum, lred);
  __syncthreads();
  const double inv = 1.0 / (static_cast<double>(B) * T);
  for (int k = threadIdx.x; k < kOut; k += blockDim.x) dO[static_cast<int64_t>(b) * kOut + k] = static_cast<float>(g[k] * inv);
  if (threadIdx.x == 0) atomicAdd(loss, ls * inv);
}

// ---------------------------------------------------------------------------
// sampling: component by its weight, Wood's rejection step for the cosine
// to mu, a uniform direction orthogonal to mu, then a random omega^k
// ---------------------------------------------------------------------------
struct VmfRng {
  uint64_t seed;
  uint32_t s, b, ctr;
  __device__ double2 uniform2() {  // two 53-bit uniforms in (0, 1)
    PhiloxOut o = philox4x32_10(s, b, ctr++, 0x564D46u, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    return make_double2(uniform53(o.w[0], o.w[1]), uniform53(o.w[2], o.w[3]));
  }
  __device__ double2 normal2() {
    const double2 u = uniform2();
    const double rad = sqrt(-2.0 * log(u.x));
    double sn, cs;
    sincospi(2.0 * u.y, &sn, &cs);
    return make_double2(rad * cs, rad * sn);
  }
  // Gamma(7/2) = Gamma(3) + Gamma(1/2): -log(u1 u2 u3) + n^2 / 2
  __device__ double gamma35() {
    const double2 a = uniform2(), c = uniform2();
    const double2 nn = normal2();
    return -log(a.x * a.y * c.x) + 0.5 * nn.x * nn.x;
  }
};

__global__ void __launch_bounds__(128) vmf_sample_kernel(const float* __restrict__ O, int B, int S, int K,
                                                         uint64_t seed, float2* __restrict__ C,
                                                         int32_t* status) {
  __shared__ CompParams cp;
  __shared__ double wb[kComp], wx0[kComp], wc[kComp], cdf[kComp];
  const int b = blockIdx.y;
  head_params(O + static_cast<int64_t>(b) * kOut, cp);
  if (threadIdx.x < kComp) {
    const int m = threadIdx.x;
    const double kap = cp.kappa[m];
    const double p1 = kDim - 1.0;
    const double bb = p1 / (2.0 * kap + sqrt(4.0 * kap * kap + p1 * p1));  // = (-2k + sqrt(4k^2 + p1^2)) / p1
    const double x0 = (1.0 - bb) / (1.0 + bb);
    wb[m] = bb;
    wx0[m] = x0;
    wc[m] = kap * x0 + p1 * log(1.0 - x0 * x0);
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int m = 0; m < kComp; ++m) {
      s += cp.pi[m];
      cdf[m] = s;
    }
  }
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  VmfRng rng{seed, static_cast<uint32_t>(s), static_cast<uint32_t>(b), 0u};
  const double2 u0 = rng.uniform2();
  int m = 0;
  const double target = u0.x * cdf[kComp - 1];
  while (m < kComp - 1 && cdf[m] < target) ++m;
  const double kap = cp.kappa[m], bb = wb[m], x0 = wx0[m], cc = wc[m];
  double w = 1.0;
  bool ok = false;
  for (int tries = 0; tries < 1000; ++tries) {
    const double g1 = rng.gamma35(), g2 = rng.gamma35();
    const double z = g1 / (g1 + g2);  // Beta(7/2, 7/2)
    w = (1.0 - (1.0 + bb) * z) / (1.0 - (1.0 - bb) * z);
    const double u = rng.uniform2().x;
    if (kap * w + (kDim - 1.0) * log(1.0 - x0 * w) - cc >= log(u)) {
      ok = true;
      break;
    }
  }
  if (!ok) dev_fail(status, LRQ_ETIMEOUT);
  double v[kDim], dot = 0.0;
  for (int d = 0; d < kDim; d += 2) {
    const double2 nn = rng.normal2();
    v[d] = nn.x;
    v[d + 1] = nn.y;
  }
  for (int d = 0; d < kDim; ++d) dot += v[d] * cp.mu[m][d];
  double nv = 0.0;
  for (int d = 0; d < kDim; ++d) {
    v[d] -= dot * cp.mu[m][d];
    nv += v[d] * v[d];
  }
  nv = nv > 0.0 ? 1.0 / sqrt(nv) : 0.0;
  const double sw = sqrt(fmax(0.0, 1.0 - w * w));
  double x[kDim];
  for (int d = 0; d < kDim; ++d) x[d] = w * cp.mu[m][d] + sw * v[d] * nv;
  // random member of the K-fold equivalence class
  const int k = min(K - 1, static_cast<int>(u0.y * K));
  double sn, cs;
  sincospi(2.0 * k / static_cast<double>(K), &sn, &cs);
  float2* out = C + (static_cast<int64_t>(b) * S + s) * (kDim / 2);
  for (int j = 0; j < kDim / 2; ++j) {
    const double re = x[2 * j], im = x[2 * j + 1];
    out[j] = make_float2(static_cast<float>(re * cs - im * sn), static_cast<float>(re * sn + im * cs));
  }
}

// The mixture's component means, ordered by weight (largest logit first,
// lower component index on ties): the most probable directions of the
// proposal, as directions of C^4.  A component with u = 0 gives e_1, the
// same convention as the sampler.  One warp per instance.
__global__ void vmf_modes_kernel(const float* __restrict__ O, int B, float2* __restrict__ C) {
  const int b = blockIdx.x;
  const int m = threadIdx.x;
  if (b >= B || m >= kComp) return;
  const float* Ob = O + static_cast<int64_t>(b) * kOut;
  const float lm = Ob[m * kHead + kDim + 1];
  int rank = 0;
  for (int k = 0; k < kComp; ++k) {
    const float lk = Ob[k * kHead + kDim + 1];
    rank += (lk > lm || (lk == lm && k < m)) ? 1 : 0;
  }
  double nrm = 0.0;
  for (int d = 0; d < kDim; ++d) nrm += static_cast<double>(Ob[m * kHead + d]) * Ob[m * kHead + d];
  nrm = sqrt(nrm);
  float2* out = C + (static_cast<int64_t>(b) * kComp + rank) * (kDim / 2);
  for (int j = 0; j < kDim / 2; ++j) {
    const double re = nrm > 0.0 ? Ob[m * kHead + 2 * j] / nrm : (j == 0 ? 1.0 : 0.0);
    const double im = nrm > 0.0 ? Ob[m * kHead + 2 * j + 1] / nrm : 0.0;
    out[j] = make_float2(static_cast<float>(re), static_cast<float>(im));
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba) with bias correction
// ---------------------------------------------------------------------------
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int64_t proposal_num_params(int F) {
  return static_cast<int64_t>(F) * kWidth + kWidth + kWidth * kWidth + kWidth + kWidth * kOut + kOut;
}

int launch_features(const float2* V, int B, int64_t n, int r, const double* lambda, float2* Vg, float* feat,
                    int32_t* status, cudaStream_t st) {
  features_kernel<<<B, 256, 0, st>>>(V, n, r, lambda, Vg, feat, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "features_kernel");
}

// BF16 mode on the tensor cores (k_mlp_tc.cu); FP32 mode on the CUDA cores
static void gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, int ta, const float* Bm, int ldb,
                 int tb, const float* bias, int relu, const float* mask, float* C, int ldc, int bf16) {
  if (bf16) {
    launch_mlp_gemm_tc(st, M, N, K, A, lda, ta, Bm, ldb, tb, bias, relu, mask, C, ldc);
    return;
  }
  dim3 grid(static_cast<unsigned>(ceil_div(N, 32)), static_cast<unsigned>(ceil_div(M, 32)));
  mlp_gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, lda, ta, Bm, ldb, tb, bias, relu, mask, C, ldc, 0);
  count_launch();
}

int launch_mlp_forward(const float* params, int F, int B, const float* X, float* H1, float* H2, float* O, int bf16,
                       cudaStream_t st) {
  const float* W1 = params;
  const float* b1 = W1 + static_cast<int64_t>(F) * kWidth;
  const float* W2 = b1 + kWidth;
  const float* b2 = W2 + kWidth * kWidth;
  const float* W3 = b2 + kWidth;
  const float* b3 = W3 + kWidth * kOut;
  gemm(st, B, kWidth, F, X, F, 0, W1, kWidth, 0, b1, 1, nullptr, H1, kWidth, bf16);
  gemm(st, B, kWidth, kWidth, H1, kWidth, 0, W2, kWidth, 0, b2, 1, nullptr, H2, kWidth, bf16);
  gemm(st, B, kOut, kWidth, H2, kWidth, 0, W3, kOut, 0, b3, 0, nullptr, O, kOut, bf16);
  return cuda_check(cudaGetLastError(), "mlp forward");
}

int launch_mlp_backward(const float* params, int F, int B, const float* X, const float* H1, const float* H2,
                        const float* dO, float* grads, float* scratch, int bf16, cudaStream_t st) {
  const float* W2 = params + static_cast<int64_t>(F) * kWidth + kWidth;
  const float* W3 = W2 + kWidth * kWidth + kWidth;
  float* dW1 = grads;
  float* db1 = dW1 + static_cast<int64_t>(F) * kWidth;
  float* dW2 = db1 + kWidth;
  float* db2 = dW2 + kWidth * kWidth;
  float* dW3 = db2 + kWidth;
  float* db3 = dW3 + kWidth * kOut;
  float* dH2 = scratch;
  float* dH1 = scratch + static_cast<int64_t>(B) * kWidth;
  // layer 3
  gemm(st, kWidth, kOut, B, H2, kWidth, 1, dO, kOut, 0, nullptr, 0, nullptr, dW3, kOut, bf16);
  colsum_f32_kernel<<<1, 256, 0, st>>>(dO, B, kOut, db3);
  gemm(st, B, kWidth, kOut, dO, kOut, 0, W3, kOut, 1, nullptr, 0, H2, dH2, kWidth, bf16);
  // layer 2
  gemm(st, kWidth, kWidth, B, H1, kWidth, 1, dH2, kWidth, 0, nullptr, 0, nullptr, dW2, kWidth, bf16);
  colsum_f32_kernel<<<1, 256, 0, st>>>(dH2, B, kWidth, db2);
  gemm(st, B, kWidth, kWidth, dH2, kWidth, 0, W2, kWidth, 1, nullptr, 0, H1, dH1, kWidth, bf16);
  // layer 1
  gemm(st, F, kWidth, B, X, F, 1, dH1, kWidth, 0, nullptr, 0, nullptr, dW1, kWidth, bf16);
  colsum_f32_kernel<<<1, 256, 0, st>>>(dH1, B, kWidth, db1);
  count_launch(3);
  return cuda_check(cudaGetLastError(), "mlp backward");
}

int launch_vmf_nll(const float* O, int B, const float* X, int T, double* loss, float* dO, cudaStream_t st) {
  int e = cuda_check(cudaMemsetAsync(loss, 0, sizeof(double), st), "reset loss");
  if (e) return e;
  vmf_nll_kernel<<<B, 128, 0, st>>>(O, B, X, T, loss, dO);
  count_launch();
  return cuda_check(cudaGetLastError(), "vmf_nll_kernel");
}

int launch_vmf_sample(const float* O, int B, int S, int K, uint64_t seed, float2* C, int32_t* status,
                      cudaStream_t st) {
  dim3 grid(static_cast<unsigned>(ceil_div(S, 128)), static_cast<unsigned>(B));
  vmf_sample_kernel<<<grid, 128, 0, st>>>(O, B, S, K, seed, C, status);
  count_launch();
  return cuda_check(cudaGetLastError(), "vmf_sample_kernel");
}

int launch_vmf_modes(const float* O, int B, float2* C, cudaStream_t st) {
  vmf_modes_kernel<<<B, 32, 0, st>>>(O, B, C);
  count_launch();
  return cuda_check(cudaGetLastError(), "vmf_modes_kernel");
}

int launch_adam(float* p, const float* g, float* m, float* v, int64_t count, int t, float lr, float b1, float b2,
                float eps, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, static_cast<float>(t)), c2 = 1.f - powf(b2, static_cast<float>(t));
  const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(count, 256), 152 * 8));
  adam_kernel<<<blocks, 256, 0, st>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2);
  count_launch();
  return cuda_check(cudaGetLastError(), "adam_kernel");
}

}  // namespace lrq
