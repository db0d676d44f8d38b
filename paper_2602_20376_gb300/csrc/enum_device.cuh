// enum_device.cuh -- device side of the exact rank-r solver by vertex
// enumeration (Sec. 3, Algorithm 2; Theorem 3.2), shared by the standalone
// solver (k_enum.cu) and the exact sub-batch of the batched launch
// (k_batched.cu).
//
// For an index set I of 2d-1 rows of the augmented real matrix (Eq. 6; rows
// h_(i,m) = [Im(rho_m V_i), Re(rho_m V_i)], rho_m = exp(-i pi (2m+1)/K),
// m < B_K, at most two rows per coordinate group) with rank 2d-1, its null
// vector c~ gives the vertex c = +-(c~[:d] + i c~[d:]); every coordinate
// takes the codes of the cells that touch the vertex (all K where w_i = 0,
// both neighbours within 1e-9 rad of a boundary, else the decision code of
// Eq. 9), and every combination is scored on the full V (||V^H z||^2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kEnumMaxD = 4;      // r <= 4
constexpr int kEnumMaxRows = 2 * kEnumMaxD - 1;
constexpr int kEnumMaxBranch = 12;
constexpr unsigned long long kEnumMaxCombos = 1ull << 16;

struct EnumTables {
  int K, BK;
  double rho_c[kMaxTcK], rho_s[kMaxTcK];  // cos, sin of theta_m (rho_m = cos - i sin)
  double bcos[kMaxTcK], bsin[kMaxTcK];    // all K boundaries for margins
  double zr[kMaxTcK], zi[kMaxTcK];        // omega^k
};

struct EnumBest {
  double f;
  int level;
  int sign;
  unsigned long long rank;
  unsigned long long choice;
};

__host__ __device__ inline unsigned long long binom(int nn, int k) {
  if (k < 0 || k > nn) return 0ull;
  unsigned long long b = 1;
  for (int t = 1; t <= k; ++t) b = b * static_cast<unsigned long long>(nn - k + t) / static_cast<unsigned long long>(t);
  return b;
}

// combinatorial number system: rank = sum_k C(idx[k], k + 1) -> sorted
// combination idx[0] < ... < idx[m-1] of [0, N) (colexicographic order)
__host__ __device__ inline void unrank(unsigned long long rank, int N, int m, int* idx) {
  int hi = N;
  for (int pos = m; pos >= 1; --pos) {
    int c = hi - 1;
    while (c >= pos - 1 && binom(c, pos) > rank) --c;
    idx[pos - 1] = c;
    rank -= binom(c, pos);
    hi = c;
  }
}

// successor in the same (colexicographic) order as unrank
__host__ __device__ inline bool next_comb(int N, int m, int* idx) {
  for (int pos = 0; pos < m; ++pos) {
    const int lim = (pos + 1 < m) ? idx[pos + 1] : N;
    if (idx[pos] + 1 < lim) {
      ++idx[pos];
      for (int q = 0; q < pos; ++q) idx[q] = q;
      return true;
    }
  }
  return false;
}

// Read access to V (n x r, row-major) in FP64: complex128 with precomputed
// row norms, or complex64 with the norms computed on the fly.
struct EnumV64 {
  const double2* V;
  int r;
  const double* rown2;  // squared row norms
  __device__ double re(int i, int j) const { return V[static_cast<int64_t>(i) * r + j].x; }
  __device__ double im(int i, int j) const { return V[static_cast<int64_t>(i) * r + j].y; }
  __device__ double rownorm2(int i) const { return rown2[i]; }
};

struct EnumV32 {
  const float2* V;
  int r;
  __device__ double re(int i, int j) const { return V[static_cast<int64_t>(i) * r + j].x; }
  __device__ double im(int i, int j) const { return V[static_cast<int64_t>(i) * r + j].y; }
  __device__ double rownorm2(int i) const {
    double s = 0.0;
    for (int j = 0; j < r; ++j) s += re(i, j) * re(i, j) + im(i, j) * im(i, j);
    return s;
  }
};

// Decision code and code set of coordinate value (x, y) for the superset rule.
// Returns the number of options written to opt (1, 2 or K).
// Thresholds in squares (no division or square root, both slow in FP64):
// |w| <= 1e-9 ||V_i||  <=>  |w|^2 <= 1e-18 ||V_i||^2, and the sine of the
// angle to a boundary |p| / |w| <= 1e-9  <=>  p^2 <= 1e-18 |w|^2.
__device__ inline int code_options(double x, double y, double rownorm2, bool dbl, const EnumTables& tb, int* opt) {
  const int K = tb.K;
  if (rownorm2 == 0.0) {  // a zero row of V: its code does not change f; fixed at 0
    opt[0] = 0;
    return 1;
  }
  const double aw2 = x * x + y * y;
  if (dbl || aw2 <= 1e-18 * rownorm2) {
    for (int k = 0; k < K; ++k) opt[k] = k;
    return K;
  }
  const int k = decide_fp64(x, y, K, tb.bcos, tb.bsin);
  // angular distance to the two boundaries of sector k: |p| / |w| = sin(dist)
  const int mlo = (k == 0) ? K - 1 : k - 1;
  const double plo = y * tb.bcos[mlo] - x * tb.bsin[mlo];
  const double phi = y * tb.bcos[k] - x * tb.bsin[k];
  const double lim = 1e-18 * aw2;
  if (plo * plo <= lim) {
    opt[0] = mlo;   // sector below boundary mlo is mlo, above is mlo + 1 = k
    opt[1] = k;
    return 2;
  }
  if (phi * phi <= lim) {
    opt[0] = k;
    opt[1] = (k + 1) % K;
    return 2;
  }
  opt[0] = k;
  return 1;
}

// Evaluate every candidate of one (level, index set, sign); keep the best.
// If `want` >= 0 the choice `want` is decoded into z instead.
template <class VA>
__device__ void eval_vertex(const VA& va, int n, int r, int d, const int* I, int m, const double* ct, int sign,
                            const EnumTables& tb, EnumBest& best, unsigned long long rank,
                            long long want, uint8_t* z_out, double* f_out, int32_t* status) {
  const int BK = tb.BK;
  double cr[kEnumMaxD], ci[kEnumMaxD];
  for (int j = 0; j < d; ++j) {
    cr[j] = sign * ct[j];
    ci[j] = sign * ct[d + j];
  }
  // groups of I: doubles
  int grp[kEnumMaxRows];
  for (int t = 0; t < m; ++t) grp[t] = I[t] / BK;
  double sr[2 * kMaxRank], si[2 * kMaxRank];
  for (int j = 0; j < r; ++j) sr[j] = si[j] = 0.0;
  int bidx[kEnumMaxBranch], bopt[kEnumMaxBranch][kMaxTcK], bcnt[kEnumMaxBranch], nb = 0;
  bool overflow = false;
  for (int i = 0; i < n; ++i) {
    double x = 0.0, y = 0.0;
    for (int j = 0; j < d; ++j) {
      x += va.re(i, j) * cr[j] - va.im(i, j) * ci[j];
      y += va.re(i, j) * ci[j] + va.im(i, j) * cr[j];
    }
    int cnt_in = 0;
    for (int t = 0; t < m; ++t) cnt_in += (grp[t] == i);
    int opt[kMaxK];
    const int no = code_options(x, y, va.rownorm2(i), cnt_in >= 2, tb, opt);
    const int k0 = opt[0];
    if (no > 1) {
      if (nb < kEnumMaxBranch && no <= kMaxTcK) {
        bidx[nb] = i;
        bcnt[nb] = no;
        for (int q = 0; q < no; ++q) bopt[nb][q] = opt[q];
        ++nb;
      } else {
        overflow = true;
      }
    }
    if (z_out && no == 1) z_out[i] = static_cast<uint8_t>(k0);
    // base sum with the first option
    for (int j = 0; j < r; ++j) {
      const double vr = va.re(i, j), vi = va.im(i, j);
      sr[j] += vr * tb.zr[k0] + vi * tb.zi[k0];
      si[j] += vr * tb.zi[k0] - vi * tb.zr[k0];
    }
  }
  unsigned long long total = 1;
  for (int b = 0; b < nb; ++b) total *= static_cast<unsigned long long>(bcnt[b]);
  if (overflow || total > kEnumMaxCombos) {
    // a vertex where more coordinates touch boundaries than the branch budget
    // allows (a degenerate, highly structured V): the result could not be
    // certified exact, so the call reports LRQ_EUNSUPPORTED
    dev_fail(status, LRQ_EUNSUPPORTED);
    return;
  }
  for (unsigned long long ch = 0; ch < total; ++ch) {
    if (want >= 0 && ch != static_cast<unsigned long long>(want)) continue;
    double tr[2 * kMaxRank], ti[2 * kMaxRank];
    for (int j = 0; j < r; ++j) {
      tr[j] = sr[j];
      ti[j] = si[j];
    }
    unsigned long long rem = ch;
    for (int b = 0; b < nb; ++b) {
      const int q = static_cast<int>(rem % bcnt[b]);
      rem /= bcnt[b];
      const int i = bidx[b];
      const int k0 = bopt[b][0], k1 = bopt[b][q];
      if (z_out) z_out[i] = static_cast<uint8_t>(k1);
      if (q == 0) continue;
      const double dzr = tb.zr[k1] - tb.zr[k0], dzi = tb.zi[k1] - tb.zi[k0];
      for (int j = 0; j < r; ++j) {
        const double vr = va.re(i, j), vi = va.im(i, j);
        tr[j] += vr * dzr + vi * dzi;
        ti[j] += vr * dzi - vi * dzr;
      }
    }
    double f = 0.0;
    for (int j = 0; j < r; ++j) f += tr[j] * tr[j] + ti[j] * ti[j];
    if (want >= 0) {
      if (f_out) *f_out = f;
      return;
    }
    if (f > best.f) {
      best.f = f;
      best.level = d;
      best.sign = sign;
      best.rank = rank;
      best.choice = ch;
    }
  }
}

template <class VA>
__device__ void build_rows(const VA& va, int r, int d, const int* I, int m, const EnumTables& tb, double* H) {
  const int nc = 2 * d;
  for (int t = 0; t < m; ++t) {
    const int i = I[t] / tb.BK, mm = I[t] % tb.BK;
    const double c = tb.rho_c[mm], s = tb.rho_s[mm];
    for (int j = 0; j < d; ++j) {
      const double vr = va.re(i, j), vi = va.im(i, j);
      // rho V = (c - i s)(vr + i vi) = (c vr + s vi) + i (c vi - s vr)
      H[t * nc + j] = c * vi - s * vr;       // Im(rho V_ij)
      H[t * nc + d + j] = c * vr + s * vi;   // Re(rho V_ij)
    }
  }
}

__host__ __device__ inline bool valid_set(const int* I, int m, int BK) {
  for (int t = 0; t + 2 < m; ++t)
    if (I[t] / BK == I[t + 2] / BK) return false;  // three rows of one group (sorted)
  return true;
}

// The decision tables of A_K for the solver (host; K <= 8).
inline EnumTables make_enum_tables(int K) {
  EnumTables tb;
  memset(&tb, 0, sizeof(tb));
  tb.K = K;
  tb.BK = (K % 2 == 0) ? K / 2 : K;
  const Alphabet a = make_alphabet(K);
  for (int mm = 0; mm < tb.BK; ++mm) {
    tb.rho_c[mm] = a.bcos64[mm];
    tb.rho_s[mm] = a.bsin64[mm];
  }
  for (int k = 0; k < K; ++k) {
    tb.bcos[k] = a.bcos64[k];
    tb.bsin[k] = a.bsin64[k];
    tb.zr[k] = a.zr64[k];
    tb.zi[k] = a.zi64[k];
  }
  return tb;
}

// Deterministic order of candidates: larger f first, then the higher level,
// the smaller index-set rank, the + sign, the smaller choice.
__host__ __device__ inline bool enum_better(const EnumBest& o, const EnumBest& me) {
  return o.f > me.f || (o.f == me.f && o.f >= 0.0 &&
                        (o.level > me.level ||
                         (o.level == me.level &&
                          (o.rank < me.rank ||
                           (o.rank == me.rank && (o.sign > me.sign || (o.sign == me.sign && o.choice < me.choice)))))));
}

}  // namespace lrq
