// lrq_device.cuh -- device helpers shared by the CUDA kernels of liblrq:
// the Philox4x32-10 generator, the decision rule in FP32 and FP64, and the
// ABI status helper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lrq_internal.h"

namespace lrq {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Round: two 32x32->64
// multiplies of counter words 0 and 2, outputs xor-ed with counter words 1, 3
// and the key; the key is advanced by the golden-ratio Weyl increments before
// every round but the first.
// ---------------------------------------------------------------------------
struct PhiloxOut {
  uint32_t w[4];
};

__device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t lo0 = M0 * c0, hi0 = __umulhi(M0, c0);
    uint32_t lo1 = M1 * c2, hi1 = __umulhi(M1, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  PhiloxOut o;
  o.w[0] = c0;
  o.w[1] = c1;
  o.w[2] = c2;
  o.w[3] = c3;
  return o;
}

// 53-bit uniform in (0, 1) from two words (top 53 bits of hi:lo, centred).
__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
  uint64_t x = ((static_cast<uint64_t>(hi) << 32) | lo) >> 11;
  return (static_cast<double>(x) + 0.5) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Uniform directions on the complex unit sphere (Sec. 4.2; App. E, Lemma
// "innerIsBeta": c = Z/||Z||, Z ~ CN(0, I_r)).  One thread per candidate; the
// Philox counter of component j of candidate s is (lo32 s, hi32 s, j, 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sphere_component(uint64_t seed, int64_t s, int j, double* zr, double* zi) {
  PhiloxOut o = philox4x32_10(static_cast<uint32_t>(s), static_cast<uint32_t>(static_cast<uint64_t>(s) >> 32),
                              static_cast<uint32_t>(j), 0u, static_cast<uint32_t>(seed),
                              static_cast<uint32_t>(seed >> 32));
  double u1 = uniform53(o.w[0], o.w[1]);
  double u2 = uniform53(o.w[2], o.w[3]);
  double rad = sqrt(-log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  *zr = rad * cs;
  *zi = rad * sn;
}

// ---------------------------------------------------------------------------
// Decision rule (Sec. 3, Eq. 9) from boundary-line signs.
// s_m = [p_m > 0] with p_m = Im(exp(-i theta_m) w), theta_m = pi(2m+1)/K.
//   even K (B_K = K/2 lines): c = #{m : s_m}, k = s_0 ? c : (K - c) mod K;
//   odd K  (B_K = K lines):   k = the j in [1, K) with s_{j-1} and not s_j,
//                             or 0 if there is none.
// Both read the sector of w off the half-planes of the lines through the
// origin; no trigonometry runs per coordinate.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ int decide_from_signs(uint32_t s) {
  if constexpr (K % 2 == 0) {
    int c = __popc(s);
    return (s & 1u) ? c : (c == 0 ? 0 : K - c);
  } else {
    // bit j-1 set and bit j clear, for j in [1, K)
    uint32_t t = s & ~(s >> 1) & ((1u << (K - 1)) - 1u);
    return t ? (__ffs(t)) : 0;
  }
}

template <int K>
__device__ __forceinline__ int decide_fp32(float x, float y, const float* bcos, const float* bsin) {
  constexpr int BK = (K % 2 == 0) ? K / 2 : K;
  uint32_t s = 0;
#pragma unroll
  for (int m = 0; m < BK; ++m) {
    float p = fmaf(y, bcos[m], -x * bsin[m]);
    s |= (p > 0.0f ? 1u : 0u) << m;
  }
  return decide_from_signs<K>(s);
}

// Generic K (> 8): nearest root from the angle, k = round(K arg(w) / 2pi) mod K.
__device__ __forceinline__ int decide_fp32_generic(float x, float y, int K) {
  if (x == 0.0f && y == 0.0f) return 0;
  float t = atan2f(y, x) * (static_cast<float>(K) * 0.15915494309189535f);
  int k = __float2int_rn(t);
  k %= K;
  if (k < 0) k += K;
  return k;
}

__device__ __forceinline__ int decide_fp64(double x, double y, int K, const double* bcos,
                                           const double* bsin) {
  if (K <= 8) {
    const int BK = (K % 2 == 0) ? K / 2 : K;
    uint32_t s = 0;
    for (int m = 0; m < BK; ++m) {
      double p = fma(y, bcos[m], -x * bsin[m]);
      s |= (p > 0.0 ? 1u : 0u) << m;
    }
    if (K % 2 == 0) {
      int c = __popc(s);
      return (s & 1u) ? c : (c == 0 ? 0 : K - c);
    }
    uint32_t t = s & ~(s >> 1) & ((1u << (K - 1)) - 1u);
    return t ? __ffs(t) : 0;
  }
  if (x == 0.0 && y == 0.0) return 0;
  double t = atan2(y, x) * (static_cast<double>(K) / (2.0 * kPi));
  long long k = __double2ll_rn(t);
  k %= K;
  if (k < 0) k += K;
  return static_cast<int>(k);
}

// ---------------------------------------------------------------------------
// Null vector (unit norm) of the m x (m+1) matrix H (row-major, modified;
// m <= kMaxRows); returns false if the rank is below m.  FP64 Gaussian
// elimination with full pivoting: a largest remaining pivot at or below
// 1e-10 max|H| rejects.  The null space's generator solves the triangular
// system with the last (permuted) unknown set to 1.
template <int kMaxRows>
__device__ bool null_vector_fp64(double* H, int m, double* c) {
  const int nc = m + 1;
  int colperm[kMaxRows + 1];
  for (int j = 0; j < nc; ++j) colperm[j] = j;
  double scale = 0.0;
  for (int t = 0; t < m * nc; ++t) scale = fmax(scale, fabs(H[t]));
  if (scale == 0.0) return false;
  for (int k = 0; k < m; ++k) {
    int pr = k, pc = k;
    double best = -1.0;
    for (int i = k; i < m; ++i)
      for (int j = k; j < nc; ++j)
        if (fabs(H[i * nc + j]) > best) {
          best = fabs(H[i * nc + j]);
          pr = i;
          pc = j;
        }
    if (best <= 1e-10 * scale) return false;
    if (pr != k)
      for (int j = 0; j < nc; ++j) {
        double t = H[k * nc + j];
        H[k * nc + j] = H[pr * nc + j];
        H[pr * nc + j] = t;
      }
    if (pc != k) {
      for (int i = 0; i < m; ++i) {
        double t = H[i * nc + k];
        H[i * nc + k] = H[i * nc + pc];
        H[i * nc + pc] = t;
      }
      int t = colperm[k];
      colperm[k] = colperm[pc];
      colperm[pc] = t;
    }
    for (int i = k + 1; i < m; ++i) {
      double f = H[i * nc + k] / H[k * nc + k];
      for (int j = k; j < nc; ++j) H[i * nc + j] -= f * H[k * nc + j];
    }
  }
  // free variable: permuted column m = 1, back-substitute
  double y[kMaxRows + 1];
  y[m] = 1.0;
  for (int k = m - 1; k >= 0; --k) {
    double s = H[k * nc + m];
    for (int j = k + 1; j < m; ++j) s += H[k * nc + j] * y[j];
    y[k] = -s / H[k * nc + k];
  }
  double nrm = 0.0;
  for (int j = 0; j < nc; ++j) nrm += y[j] * y[j];
  nrm = 1.0 / sqrt(nrm);
  for (int j = 0; j < nc; ++j) c[colperm[j]] = y[j] * nrm;
  return true;
}

}  // namespace lrq
