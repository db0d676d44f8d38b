// k_lanczos.cu -- spectral truncation Q ~= V V^H, V = [sqrt(lambda_j) u_j]
// (Sec. 4.1, Algorithm 3): the r largest (algebraic) eigenpairs of a
// Hermitian operator by FP64 Lanczos on the GPU.
//
// Operators: a dense Hermitian complex128 matrix, or the Laplacian
// L = D - A of a graph given as symmetric CSR (optional edge weights),
// applied matrix-free (self loops cancel in D - A and are skipped).
//
// Method (the paper calls ARPACK; this is a Lanczos of our own design):
//   * Lanczos with full reorthogonalisation: after w = Q u_j, w is projected
//     off u_j and u_{j-1} (the three-term step, which removes its large
//     components) and then off every stored vector (one classical
//     Gram-Schmidt pass over components of rounding size); alpha_j =
//     u_j^H Q u_j is the sum of the two projections onto u_j, and
//     beta_j = ||w||.  The tridiagonal T_J is real for Hermitian Q.
//   * Convergence: eigenvalues of T_J by multisection on Sturm counts, their
//     eigenvectors by inverse iteration (Gaussian elimination with partial
//     pivoting), residual ||Q y - theta y|| = beta_{J-1} |x_{J-1}|.
//   * Locking: converged Ritz vectors are stored in front of the Krylov
//     basis and every later vector is orthogonalised against them, so that a
//     new run (fresh random start) sees only the rest of the spectrum.  A
//     single-vector Krylov space holds one vector per eigenspace; "check"
//     runs repeat until the largest remaining eigenvalue is not above the
//     r-th locked one, which recovers every copy of a repeated eigenvalue
//     that belongs to the top r.
// Vectors are stored column-major (each basis vector contiguous, n doubles
// or complex doubles); the projections are tall-skinny GEMV pairs over
// row chunks with a fixed-order reduction (deterministic).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "lrq_device.cuh"
#include "lrq_internal.h"

namespace lrq {

constexpr int kLzThreads = 256;
constexpr int kLzChunkMax = 4096;  // rows per block in the projection kernels (at most)
constexpr int kLzGroup = 8;        // basis vectors per block in the projection kernels
constexpr int kLzWant = kMaxRank;  // at most 8 wanted pairs per run
constexpr int kLzMaxIter = 4096;
constexpr int kLzDefaultIter = 500;
constexpr int kLzLag = 2;          // Lanczos steps run while a convergence check is in flight

// ---------------------------------------------------------------------------
// scalar helpers: real (graph Laplacian) and complex (dense Hermitian) paths
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lz_cdot(double a, double b) { return a * b; }
__device__ __forceinline__ double2 lz_cdot(double2 a, double2 b) {  // conj(a) b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double lz_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 lz_mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double lz_scale(double a, double s) { return a * s; }
__device__ __forceinline__ double2 lz_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ void lz_add(double& a, double b) { a += b; }
__device__ __forceinline__ void lz_add(double2& a, double2 b) {
  a.x += b.x;
  a.y += b.y;
}
__device__ __forceinline__ void lz_sub(double& a, double b) { a -= b; }
__device__ __forceinline__ void lz_sub(double2& a, double2 b) {
  a.x -= b.x;
  a.y -= b.y;
}
__device__ __forceinline__ double lz_abs2(double a) { return a * a; }
__device__ __forceinline__ double lz_abs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double lz_re(double a) { return a; }
__device__ __forceinline__ double lz_re(double2 a) { return a.x; }
template <typename T>
__device__ __forceinline__ T lz_zero();
template <>
__device__ __forceinline__ double lz_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ double2 lz_zero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double lz_shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double2 lz_shfl_xor(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <typename T>
__device__ __forceinline__ T lz_warp_sum(T v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) lz_add(v, lz_shfl_xor(v, m));
  return v;
}
__device__ __forceinline__ double2 lz_as_complex(double a) { return make_double2(a, 0.0); }
__device__ __forceinline__ double2 lz_as_complex(double2 a) { return a; }
__device__ __forceinline__ double lz_real_or_gauss(double, double g0, double) { return g0; }
__device__ __forceinline__ double2 lz_real_or_gauss(double2, double g0, double g1) { return make_double2(g0, g1); }

// Device state of one Lanczos run.
struct LzState {
  int stop;        // set on breakdown (invariant subspace reached)
  int jdone;       // Lanczos vectors whose alpha and beta are known
  double tnorm;    // running estimate of ||T||
  double inv_beta;
};

// Result of a convergence check (copied to the host).
struct LzCheck {
  int J;
  int converged;
  int breakdown;
  int nvalid;
  double tnorm;
  double theta[kLzWant];
  double res[kLzWant];
};

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------
// y = L x = D x - A x for the graph Laplacian, a thread per row: the
// weighted degrees D are precomputed (lz_degree), so a row costs one FP64
// add or FMA per stored edge (GB300's FP64 rate, not memory, bounds this
// operator).  Self loops are skipped, out-of-range columns ignored (they are
// reported by lz_check_csr).
__global__ void __launch_bounds__(kLzThreads) lz_matvec_laplacian(const int32_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ colidx,
                                                                  const double* __restrict__ wts,
                                                                  const double* __restrict__ deg, int64_t n,
                                                                  int64_t nnz, const double* __restrict__ x,
                                                                  double* __restrict__ y, const LzState* st) {
  if (st->stop) return;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
    k0 = k0 < 0 ? 0 : (k0 > nnz ? nnz : k0);
    k1 = k1 < k0 ? k0 : (k1 > nnz ? nnz : k1);
    double acc = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t j = colidx[k];
      if (j < 0 || j >= n || j == i) continue;
      acc = wts ? fma(wts[k], x[j], acc) : acc + x[j];
    }
    y[i] = fma(deg[i], x[i], -acc);
  }
}

// deg[i] = sum of the row's edge weights (self loops and invalid columns
// skipped), once per truncation
__global__ void __launch_bounds__(kLzThreads) lz_degree(const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ colidx,
                                                        const double* __restrict__ wts, int64_t n, int64_t nnz,
                                                        double* __restrict__ deg) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
    k0 = k0 < 0 ? 0 : (k0 > nnz ? nnz : k0);
    k1 = k1 < k0 ? k0 : (k1 > nnz ? nnz : k1);
    double d = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t j = colidx[k];
      if (j < 0 || j >= n || j == i) continue;
      d += wts ? wts[k] : 1.0;
    }
    deg[i] = d;
  }
}

// y = Q x for dense Hermitian Q (row-major, leading dimension ld): a warp
// per row.
__global__ void __launch_bounds__(kLzThreads) lz_matvec_dense(const double2* __restrict__ Q, int64_t n, int64_t ld,
                                                              const double2* __restrict__ x, double2* __restrict__ y,
                                                              const LzState* st) {
  if (st->stop) return;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const double2* row = Q + i * ld;
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    int64_t j = lane;
    for (; j + 32 < n; j += 64) {
      lz_add(a0, lz_mul(row[j], x[j]));
      lz_add(a1, lz_mul(row[j + 32], x[j + 32]));
    }
    if (j < n) lz_add(a0, lz_mul(row[j], x[j]));
    lz_add(a0, a1);
    a0 = lz_warp_sum(a0);
    if (lane == 0) y[i] = a0;
  }
}

// ---------------------------------------------------------------------------
// projections
// ---------------------------------------------------------------------------
// partial[c * nch + chunk] = sum over the chunk's rows of conj(U_c) w, for
// basis vectors c in [0, nc).  grid = (nch, ceil(nc / 8)).
template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_dots(const T* __restrict__ U, int64_t n, int nc,
                                                      const T* __restrict__ w, T* __restrict__ partial, int nch,
                                                      int chunk_rows, const LzState* st) {
  if (st->stop) return;
  __shared__ T red[kLzGroup][kLzThreads / 32];
  const int chunk = blockIdx.x;
  const int cg = blockIdx.y * kLzGroup;
  const int64_t i0 = static_cast<int64_t>(chunk) * chunk_rows;
  const int64_t i1 = min(n, i0 + chunk_rows);
  T acc[kLzGroup];
#pragma unroll
  for (int q = 0; q < kLzGroup; ++q) acc[q] = lz_zero<T>();
  const int ncols = min(kLzGroup, nc - cg);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const T wi = w[i];
#pragma unroll
    for (int q = 0; q < kLzGroup; ++q)
      if (q < ncols) lz_add(acc[q], lz_cdot(U[static_cast<int64_t>(cg + q) * n + i], wi));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kLzGroup; ++q) {
    T v = lz_warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < ncols) {
    T s = lz_zero<T>();
    for (int k = 0; k < kLzThreads / 32; ++k) lz_add(s, red[threadIdx.x][k]);
    partial[static_cast<int64_t>(cg + threadIdx.x) * nch + chunk] = s;
  }
}

// h[c] = sum_chunk partial[c * nch + chunk] in chunk order (a warp per c).
template <typename T>
__global__ void lz_reduce(const T* __restrict__ partial, int nc, int nch, T* __restrict__ h, const LzState* st) {
  if (st->stop) return;
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= nc) return;  // whole warps leave together
  T s = lz_zero<T>();
  for (int k = lane; k < nch; k += 32) lz_add(s, partial[static_cast<int64_t>(c) * nch + k]);
  s = lz_warp_sum(s);
  if (lane == 0) h[c] = s;
}

// w -= sum_c U_c h[c]: a block takes 32 rows, its 8 warps take every 8th
// basis vector (coalesced 32-row loads), and the 8 partial sums of a row are
// added in warp order (deterministic).
template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_update(const T* __restrict__ U, int64_t n, int nc,
                                                        const T* __restrict__ h, T* __restrict__ w,
                                                        const LzState* st) {
  if (st->stop) return;
  __shared__ T part[kLzThreads / 32][32];
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  constexpr int NS = kLzThreads / 32;
  for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32; r0 < n; r0 += static_cast<int64_t>(gridDim.x) * 32) {
    const int64_t i = r0 + lane;
    T s0 = lz_zero<T>(), s1 = lz_zero<T>();
    if (i < n) {
      int c = slice;
      for (; c + NS < nc; c += 2 * NS) {
        lz_add(s0, lz_mul(U[static_cast<int64_t>(c) * n + i], h[c]));
        lz_add(s1, lz_mul(U[static_cast<int64_t>(c + NS) * n + i], h[c + NS]));
      }
      if (c < nc) lz_add(s0, lz_mul(U[static_cast<int64_t>(c) * n + i], h[c]));
    }
    lz_add(s0, s1);
    part[slice][lane] = s0;
    __syncthreads();
    if (slice == 0 && i < n) {
      T t = part[0][lane];
      for (int k = 1; k < NS; ++k) lz_add(t, part[k][lane]);
      T v = w[i];
      lz_sub(v, t);
      w[i] = v;
    }
    __syncthreads();
  }
}

// npart[chunk] = sum over the chunk of |w_i|^2
template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_norm_partial(const T* __restrict__ w, int64_t n,
                                                              double* __restrict__ npart, int chunk_rows,
                                                              const LzState* st) {
  if (st->stop) return;
  __shared__ double red[kLzThreads / 32];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * chunk_rows;
  const int64_t i1 = min(n, i0 + chunk_rows);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += lz_abs2(w[i]);
  s = lz_warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kLzThreads / 32; ++k) t += red[k];
    npart[blockIdx.x] = t;
  }
}

// Close step j: beta_j = ||w||, alpha_j = Re(h1[c] + h2[c]) (c = column of
// u_j), breakdown test.  mode 1 = normalising a start vector (no alpha).
template <typename T>
__global__ void lz_finish(const double* __restrict__ npart, int nch, const T* __restrict__ h1,
                          const T* __restrict__ h2, int c, int j, int mode, double* __restrict__ alpha,
                          double* __restrict__ beta, LzState* st) {
  if (blockIdx.x != 0 || st->stop) return;
  // the chunk norms, lane-strided then a fixed shuffle tree (deterministic)
  double s = 0.0;
  for (int k = threadIdx.x; k < nch; k += 32) s += npart[k];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (threadIdx.x != 0) return;
  const double b = sqrt(s);
  if (mode == 1) {
    // start vector: b is its norm after projection; a zero vector means the
    // locked vectors already span the space
    if (!(b > 0.0)) {
      st->stop = 2;
      return;
    }
    st->inv_beta = 1.0 / b;
    return;
  }
  const double a = lz_re(h1[c]) + lz_re(h2[c]);
  alpha[j] = a;
  beta[j] = b;
  const double bprev = j > 0 ? beta[j - 1] : 0.0;
  st->tnorm = fmax(st->tnorm, fabs(a) + b + bprev);
  st->jdone = j + 1;
  if (!(b > 1e-12 * st->tnorm)) {
    st->stop = 1;  // invariant subspace: the Ritz values of T_{j+1} are exact
    return;
  }
  st->inv_beta = 1.0 / b;
}

template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_scale_into(const T* __restrict__ w, int64_t n, T* __restrict__ u,
                                                            const LzState* st) {
  if (st->stop) return;
  const double s = st->inv_beta;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    u[i] = lz_scale(w[i], s);
}

// Gaussian start vector from Philox4x32-10: key = seed, counter =
// (lo32 i, hi32 i, run, 0x4C5A) (Box-Muller on two 53-bit uniforms).
template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_start(T* __restrict__ w, int64_t n, uint64_t seed, int run,
                                                       const LzState* st) {
  if (st->stop) return;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    PhiloxOut o = philox4x32_10(static_cast<uint32_t>(i), static_cast<uint32_t>(static_cast<uint64_t>(i) >> 32),
                                static_cast<uint32_t>(run), 0x4C5Au, static_cast<uint32_t>(seed),
                                static_cast<uint32_t>(seed >> 32));
    const double u1 = uniform53(o.w[0], o.w[1]), u2 = uniform53(o.w[2], o.w[3]);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    w[i] = lz_real_or_gauss(T(), rad * cs, rad * sn);
  }
}

// ---------------------------------------------------------------------------
// tridiagonal eigenproblem of T_J (one block)
// ---------------------------------------------------------------------------
// Number of eigenvalues of T_J below x (Sturm sequence of the LDL^T pivots).
__device__ int lz_sturm(const double* __restrict__ a, const double* __restrict__ b, int J, double x, double pivmin) {
  int cnt = 0;
  double d = a[0] - x;
  if (fabs(d) < pivmin) d = -pivmin;
  cnt += d < 0.0;
  for (int i = 1; i < J; ++i) {
    d = (a[i] - x) - b[i - 1] * b[i - 1] / d;
    if (fabs(d) < pivmin) d = -pivmin;
    cnt += d < 0.0;
  }
  return cnt;
}

// One solve of (T - theta I) x = rhs by Gaussian elimination with partial
// pivoting; x overwrites rhs.  Work arrays D, DL, DU, DU2, PV of length J.
__device__ void lz_tri_solve(const double* __restrict__ a, const double* __restrict__ b, int J, double theta,
                             double pivtol, double* D, double* DL, double* DU, double* DU2, double* PV,
                             double* x) {
  for (int i = 0; i < J; ++i) {
    D[i] = a[i] - theta;
    if (i + 1 < J) {
      DL[i] = b[i];
      DU[i] = b[i];
    }
    DU2[i] = 0.0;
  }
  for (int i = 0; i + 1 < J; ++i) {
    if (fabs(D[i]) >= fabs(DL[i])) {
      if (fabs(D[i]) < pivtol) D[i] = D[i] < 0.0 ? -pivtol : pivtol;
      const double f = DL[i] / D[i];
      DL[i] = f;
      D[i + 1] -= f * DU[i];
      PV[i] = 0.0;
    } else {
      const double f = D[i] / DL[i];
      D[i] = DL[i];
      DL[i] = f;
      const double t = DU[i];
      DU[i] = D[i + 1];
      D[i + 1] = t - f * D[i + 1];
      if (i + 2 < J) {
        DU2[i] = DU[i + 1];
        DU[i + 1] = -f * DU[i + 1];
      }
      PV[i] = 1.0;
    }
  }
  if (fabs(D[J - 1]) < pivtol) D[J - 1] = D[J - 1] < 0.0 ? -pivtol : pivtol;
  for (int i = 0; i + 1 < J; ++i) {
    if (PV[i] != 0.0) {
      const double t = x[i];
      x[i] = x[i + 1];
      x[i + 1] = t;
    }
    x[i + 1] -= DL[i] * x[i];
  }
  x[J - 1] /= D[J - 1];
  if (J > 1) x[J - 2] = (x[J - 2] - DU[J - 2] * x[J - 1]) / D[J - 2];
  for (int i = J - 3; i >= 0; --i) x[i] = (x[i] - DU[i] * x[i + 1] - DU2[i] * x[i + 2]) / D[i];
}

__device__ void lz_normalize(double* x, int J) {
  double s = 0.0, mx = 0.0;
  for (int i = 0; i < J; ++i) mx = fmax(mx, fabs(x[i]));
  if (!(mx > 0.0)) {
    x[0] = 1.0;
    return;
  }
  for (int i = 0; i < J; ++i) {
    x[i] /= mx;
    s += x[i] * x[i];
  }
  s = 1.0 / sqrt(s);
  for (int i = 0; i < J; ++i) x[i] *= s;
}

// p largest eigenvalues of T_J, their eigenvectors X[w * ldx + k], residual
// bounds and the convergence verdict.  256 threads; warp w < p bisects the
// w-th largest eigenvalue with 32-point multisection.
__global__ void __launch_bounds__(256) lz_tridiag(const double* __restrict__ alpha, const double* __restrict__ beta,
                                                  int p, double tol, int ldx, double* __restrict__ X,
                                                  double* __restrict__ work, const LzState* st,
                                                  LzCheck* __restrict__ out) {
  __shared__ double s_lo, s_hi, s_theta[kLzWant];
  __shared__ double red_lo[8], red_hi[8];
  const int J = st->jdone;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (J <= 0) {
    if (tid == 0) {
      out->J = 0;
      out->converged = 0;
      out->breakdown = st->stop;
      out->nvalid = 0;
    }
    return;
  }
  // Gershgorin interval of T_J
  double lo = INFINITY, hi = -INFINITY;
  for (int i = tid; i < J; i += blockDim.x) {
    const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < J ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  for (int m = 16; m > 0; m >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, m));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, m));
  }
  if (lane == 0) {
    red_lo[warp] = lo;
    red_hi[warp] = hi;
  }
  __syncthreads();
  if (tid == 0) {
    double a = red_lo[0], c = red_hi[0];
    for (int k = 1; k < 8; ++k) {
      a = fmin(a, red_lo[k]);
      c = fmax(c, red_hi[k]);
    }
    s_lo = a;
    s_hi = c;
  }
  __syncthreads();
  const double tn = fmax(fmax(fabs(s_lo), fabs(s_hi)), DBL_MIN);
  const double pivmin = DBL_MIN * fmax(1.0, tn * tn);
  const int nwant = min(p, J);
  if (warp < nwant) {
    const int k = J - 1 - warp;  // 0-based ascending index
    double l = s_lo - 1e-12 * tn - pivmin, h = s_hi + 1e-12 * tn + pivmin;
    for (int round = 0; round < 64; ++round) {
      if (h - l <= 4.0 * DBL_EPSILON * fmax(fabs(l), fabs(h)) + pivmin) break;
      const double x = l + (h - l) * static_cast<double>(lane + 1) / 33.0;
      const int cnt = lz_sturm(alpha, beta, J, x, pivmin);
      double nl = cnt <= k ? x : -INFINITY;
      double nh = cnt >= k + 1 ? x : INFINITY;
      for (int m = 16; m > 0; m >>= 1) {
        nl = fmax(nl, __shfl_xor_sync(0xffffffffu, nl, m));
        nh = fmin(nh, __shfl_xor_sync(0xffffffffu, nh, m));
      }
      if (nl > l) l = nl;
      if (nh < h) h = nh;
    }
    if (lane == 0) s_theta[warp] = 0.5 * (l + h);
  }
  __syncthreads();
  // inverse iteration, three rounds, with Gram-Schmidt inside clusters
  const double pivtol = DBL_EPSILON * tn;
  for (int it = 0; it < 3; ++it) {
    if (tid < nwant) {
      double* x = X + static_cast<int64_t>(tid) * ldx;
      double* wk = work + static_cast<int64_t>(tid) * 5 * ldx;
      if (it == 0)
        for (int i = 0; i < J; ++i) x[i] = 1.0 + 0.01 * static_cast<double>((i * 7 + tid * 3) % 11);
      const double shift = s_theta[tid] + 2.0 * DBL_EPSILON * tn;
      lz_tri_solve(alpha, beta, J, shift, pivtol, wk, wk + ldx, wk + 2 * ldx, wk + 3 * ldx, wk + 4 * ldx, x);
      lz_normalize(x, J);
    }
    __syncthreads();
    if (tid == 0) {
      for (int a = 1; a < nwant; ++a)
        for (int c = 0; c < a; ++c) {
          if (fabs(s_theta[a] - s_theta[c]) > 1e-3 * tn) continue;
          double* xa = X + static_cast<int64_t>(a) * ldx;
          const double* xc = X + static_cast<int64_t>(c) * ldx;
          double d = 0.0;
          for (int i = 0; i < J; ++i) d += xa[i] * xc[i];
          for (int i = 0; i < J; ++i) xa[i] -= d * xc[i];
          lz_normalize(xa, J);
        }
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double bJ = beta[J - 1];
    int conv = 1;
    for (int a = 0; a < nwant; ++a) {
      const double r = fabs(bJ) * fabs(X[static_cast<int64_t>(a) * ldx + J - 1]);
      out->theta[a] = s_theta[a];
      out->res[a] = r;
      if (!(r <= tol * tn)) conv = 0;
    }
    out->J = J;
    out->nvalid = nwant;
    out->breakdown = st->stop;
    out->converged = conv && nwant == p;
    out->tnorm = tn;
  }
}

// Y[a] = sum_k U_{c0+k} X[a][k] for a < p (Ritz vectors), a thread per row.
template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_ritz(const T* __restrict__ U, int64_t n, int c0, int J,
                                                      const double* __restrict__ X, int ldx, int p,
                                                      T* __restrict__ Y) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    T acc[kLzWant];
#pragma unroll
    for (int a = 0; a < kLzWant; ++a) acc[a] = lz_zero<T>();
    for (int k = 0; k < J; ++k) {
      const T u = U[static_cast<int64_t>(c0 + k) * n + i];
#pragma unroll
      for (int a = 0; a < kLzWant; ++a)
        if (a < p) lz_add(acc[a], lz_scale(u, X[static_cast<int64_t>(a) * ldx + k]));
    }
#pragma unroll
    for (int a = 0; a < kLzWant; ++a)
      if (a < p) Y[static_cast<int64_t>(a) * n + i] = acc[a];
  }
}

struct LzOutput {
  int r;
  int col[kLzWant];
  double lam[kLzWant];
};

// V[i, j] = sqrt(lambda_j) u_j[i] for lambda_j > 0, else 0 (row-major n x r).
template <typename T>
__global__ void __launch_bounds__(kLzThreads) lz_output(const T* __restrict__ U, int64_t n,
                                                        const __grid_constant__ LzOutput o, double2* __restrict__ V,
                                                        float2* __restrict__ V32) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int j = 0; j < o.r; ++j) {
      double2 v = make_double2(0.0, 0.0);
      if (o.col[j] >= 0 && o.lam[j] > 0.0) {
        const double s = sqrt(o.lam[j]);
        const T u = U[static_cast<int64_t>(o.col[j]) * n + i];
        v = lz_mul(make_double2(s, 0.0), lz_as_complex(u));
      }
      if (V) V[i * o.r + j] = v;
      if (V32) V32[i * o.r + j] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
    }
  }
}

// ---------------------------------------------------------------------------
// input checks
// ---------------------------------------------------------------------------
__global__ void lz_check_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                             const double* __restrict__ wts, int64_t n, int64_t nnz, int32_t* status) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  bool bad = false;
  if (t0 == 0) bad |= rowptr[0] != 0 || static_cast<int64_t>(rowptr[n]) != nnz;
  for (int64_t i = t0; i < n; i += stride) bad |= rowptr[i] > rowptr[i + 1];
  for (int64_t k = t0; k < nnz; k += stride) {
    bad |= colidx[k] < 0 || colidx[k] >= n;
    if (wts) bad |= !isfinite(wts[k]);
  }
  if (bad) dev_fail(status, LRQ_EINVAL);
}

__global__ void lz_check_dense(const double2* __restrict__ Q, int64_t n, int64_t ld, int32_t* status) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n * n; t += stride) {
    const double2 q = Q[(t / n) * ld + (t % n)];
    bad |= !isfinite(q.x) || !isfinite(q.y);
  }
  if (bad) dev_fail(status, LRQ_EINVAL);
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
namespace {

struct LzPlan {
  int64_t n;
  int r, maxit, lmax, cap, nch, chunk, ldx;
  size_t esz;
  size_t off_U, off_w, off_Y, off_part, off_h1, off_h2, off_npart, off_alpha, off_beta, off_state, off_check, off_X,
      off_work, off_deg, off_snap, total;
};

size_t lz_take(size_t& cur, size_t bytes) {
  size_t o = cur;
  cur = align_up(cur + bytes, 256);
  return o;
}

void lz_plan(int64_t n, int r, int maxit, bool cplx, LzPlan* p) {
  p->n = n;
  p->r = r;
  p->maxit = maxit;
  p->lmax = 2 * r + 8;                    // locked vectors (repeated eigenvalues need extra slots)
  p->cap = p->lmax + maxit + 1;           // basis columns
  // about two row chunks per SM, 256 to 4096 rows each
  p->chunk = static_cast<int>(std::min<int64_t>(
      kLzChunkMax, std::max<int64_t>(256, static_cast<int64_t>(align_up(ceil_div(n, 2 * 152), 256)))));
  p->nch = static_cast<int>(ceil_div(n, p->chunk));
  p->ldx = maxit + 1;
  p->esz = cplx ? sizeof(double2) : sizeof(double);
  size_t cur = 0;
  p->off_U = lz_take(cur, static_cast<size_t>(n) * p->cap * p->esz);
  p->off_w = lz_take(cur, static_cast<size_t>(n) * p->esz);
  p->off_Y = lz_take(cur, static_cast<size_t>(n) * kLzWant * p->esz);
  p->off_part = lz_take(cur, static_cast<size_t>(p->cap) * p->nch * p->esz);
  p->off_h1 = lz_take(cur, static_cast<size_t>(p->cap) * p->esz);
  p->off_h2 = lz_take(cur, static_cast<size_t>(p->cap) * p->esz);
  p->off_npart = lz_take(cur, static_cast<size_t>(p->nch) * sizeof(double));
  p->off_alpha = lz_take(cur, static_cast<size_t>(p->ldx) * sizeof(double));
  p->off_beta = lz_take(cur, static_cast<size_t>(p->ldx) * sizeof(double));
  p->off_state = lz_take(cur, sizeof(LzState));
  p->off_check = lz_take(cur, sizeof(LzCheck));
  p->off_X = lz_take(cur, static_cast<size_t>(kLzWant) * p->ldx * sizeof(double));
  p->off_work = lz_take(cur, static_cast<size_t>(kLzWant) * 5 * p->ldx * sizeof(double));
  p->off_deg = lz_take(cur, cplx ? 0 : static_cast<size_t>(n) * sizeof(double));  // Laplacian degrees
  p->off_snap = lz_take(cur, sizeof(LzState));  // the state a convergence check reads
  p->total = cur;
}

int lz_rows_grid(int64_t rows) { return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, kLzThreads), 152 * 8))); }

template <typename T>
struct LzRun {
  // operator
  bool dense;
  const double2* Q;
  int64_t ld;
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* wts;
  int64_t nnz;
  // problem
  int64_t n;
  double tol;
  uint64_t seed;
  LzPlan p;
  uint8_t* ws;
  int32_t* status;
  cudaStream_t st;
  cudaStream_t side;  // convergence checks run here, beside the next Lanczos steps
  cudaEvent_t ev;     // step done (the check waits for it)
  cudaEvent_t done;   // check done (the host polls it)

  T* U() const { return reinterpret_cast<T*>(ws + p.off_U); }
  T* col(int c) const { return U() + static_cast<int64_t>(c) * n; }
  T* w() const { return reinterpret_cast<T*>(ws + p.off_w); }
  T* Y() const { return reinterpret_cast<T*>(ws + p.off_Y); }
  T* part() const { return reinterpret_cast<T*>(ws + p.off_part); }
  T* h1() const { return reinterpret_cast<T*>(ws + p.off_h1); }
  T* h2() const { return reinterpret_cast<T*>(ws + p.off_h2); }
  double* npart() const { return reinterpret_cast<double*>(ws + p.off_npart); }
  double* alpha() const { return reinterpret_cast<double*>(ws + p.off_alpha); }
  double* beta() const { return reinterpret_cast<double*>(ws + p.off_beta); }
  LzState* state() const { return reinterpret_cast<LzState*>(ws + p.off_state); }
  LzCheck* check() const { return reinterpret_cast<LzCheck*>(ws + p.off_check); }
  double* X() const { return reinterpret_cast<double*>(ws + p.off_X); }
  double* work() const { return reinterpret_cast<double*>(ws + p.off_work); }
  double* deg() const { return reinterpret_cast<double*>(ws + p.off_deg); }
  LzState* snap() const { return reinterpret_cast<LzState*>(ws + p.off_snap); }

  void matvec(const T* x, T* y) const;
  void prepare() const;  // operator set-up once per truncation (Laplacian degrees)

  // w -= U[:, first:first+nc] (U[:, first:first+nc]^H w), projections into
  // h[first:first+nc]
  void project(int first, int nc, T* h) const {
    if (nc <= 0) return;
    dim3 g(p.nch, static_cast<unsigned>(ceil_div(nc, kLzGroup)));
    lz_dots<T><<<g, kLzThreads, 0, st>>>(col(first), n, nc, w(), part(), p.nch, p.chunk, state());
    lz_reduce<T><<<static_cast<unsigned>(ceil_div(static_cast<int64_t>(nc) * 32, 256)), 256, 0, st>>>(
        part(), nc, p.nch, h + first, state());
    lz_update<T><<<static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 32), 152 * 16)), kLzThreads, 0, st>>>(
        col(first), n, nc, h + first, w(), state());
    count_launch(3);
  }
  // normalise w into column c; mode 0 closes Lanczos step j (column c - 1)
  void close(int c, int j, int mode) const {
    lz_norm_partial<T><<<p.nch, kLzThreads, 0, st>>>(w(), n, npart(), p.chunk, state());
    lz_finish<T><<<1, 32, 0, st>>>(npart(), p.nch, h1(), h2(), c - 1, j, mode, alpha(), beta(), state());
    lz_scale_into<T><<<lz_rows_grid(n), kLzThreads, 0, st>>>(w(), n, col(c), state());
    count_launch(3);
  }
  // A convergence check reads alpha, beta and a snapshot of the state of
  // step J and runs on the side stream, so the next Lanczos steps (which
  // only append to alpha, beta and the basis) proceed meanwhile; its verdict
  // is read kLzLag steps later: the host waits for it with those steps
  // queued, so the GPU is not left idle and at most kLzLag steps run past
  // convergence.
  int launch_check(int p_want) const {
    int e = cuda_check(cudaMemcpyAsync(snap(), state(), sizeof(LzState), cudaMemcpyDeviceToDevice, st),
                       "snapshot state");
    if (e) return e;
    if ((e = cuda_check(cudaEventRecord(ev, st), "record step event"))) return e;
    if ((e = cuda_check(cudaStreamWaitEvent(side, ev, 0), "order check after step"))) return e;
    lz_tridiag<<<1, 256, 0, side>>>(alpha(), beta(), p_want, tol, p.ldx, X(), work(), snap(), check());
    count_launch();
    if ((e = cuda_check(cudaGetLastError(), "lz_tridiag"))) return e;
    return cuda_check(cudaEventRecord(done, side), "record check event");
  }
  int finish_check(LzCheck* hc) const {
    int32_t hs = 0;
    int e = cuda_check(cudaEventSynchronize(done), "wait for the check");
    if (e) return e;
    if ((e = cuda_check(cudaMemcpyAsync(hc, check(), sizeof(LzCheck), cudaMemcpyDeviceToHost, side), "copy check")))
      return e;
    if (e) return e;
    if ((e = cuda_check(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, side),
                        "copy status")))
      return e;
    if ((e = cuda_check(cudaStreamSynchronize(side), "lanczos sync"))) return e;
    if (hs != 0) return fail(hs, "lrq_truncate: the device reported an invalid input or error");
    return LRQ_OK;
  }

  // One Lanczos run against the L locked vectors; wants the p largest
  // eigenpairs of the deflated operator.
  int run(int L, int p_want, int run_id, LzCheck* hc, int64_t* steps) const {
    int e = cuda_check(cudaMemsetAsync(state(), 0, sizeof(LzState), st), "memset state");
    if (e) return e;
    lz_start<T><<<lz_rows_grid(n), kLzThreads, 0, st>>>(w(), n, seed, run_id, state());
    count_launch();
    project(0, L, h1());
    project(0, L, h2());
    close(L, 0, 1);
    int pending = 0, since = 0;  // a check in flight, and steps taken since it started
    // the verdict of the check in flight: 1 = this run is over, 0 = go on
    auto verdict = [&](int* over) -> int {
      pending = 0;
      int e2 = finish_check(hc);
      if (e2) return e2;
      if (hc->breakdown == 2) hc->nvalid = 0;  // the start vector had no part outside the locked space
      *over = hc->breakdown || hc->converged || L + hc->J >= n;
      return LRQ_OK;
    };
    for (int j = 0; j < p.maxit && L + j < n; ++j) {
      const int c = L + j;
      matvec(col(c), w());
      // the three-term step: the large components of w = Q u_j lie along u_j
      // and u_{j-1}; taking them out first leaves components of rounding size
      // along every other stored vector, which one full Gram-Schmidt pass then
      // removes (alpha_j = h1[c] + h2[c])
      if (j > 0)
        project(c - 1, 2, h1());
      else
        project(c, 1, h1());
      project(0, c + 1, h2());
      close(c + 1, j, 0);
      ++*steps;
      ++since;
      const int J = j + 1;
      const bool last = J == p.maxit || L + J >= n;
      const int every = J < 16 ? 2 : (J < 64 ? 4 : 8);
      const bool due = J >= p_want && J % every == 0;
      int over = 0;
      if (pending && (due || last || since >= kLzLag)) {
        if ((e = verdict(&over))) return e;
        if (over) return LRQ_OK;
      }
      if (due || last) {
        if ((e = launch_check(p_want))) return e;
        pending = J;
        since = 0;
      }
      if (last) {
        if ((e = verdict(&over))) return e;
        if (over) return LRQ_OK;
        return fail(LRQ_ENOCONV, "lrq_truncate: Lanczos did not converge within max_iter steps");
      }
    }
    return fail(LRQ_ENOCONV, "lrq_truncate: Lanczos did not converge within max_iter steps");
  }

  int solve(int r, double* lambda_out, double2* V, float2* V32, int64_t* iters_out) const {
    std::vector<double> vals;
    int L = 0, run_id = 0;
    int64_t steps = 0;
    bool verify = false;
    double tn = 0.0;
    int e;
    prepare();
    while (L < n) {
      if (!verify && L >= r) verify = true;
      const int p_want = verify ? 1 : static_cast<int>(std::min<int64_t>(r - L, n - L));
      LzCheck hc;
      if ((e = run(L, p_want, run_id++, &hc, &steps))) return e;
      if (hc.nvalid <= 0) break;
      tn = std::max(tn, hc.tnorm);
      if (verify) {
        std::vector<double> sorted = vals;
        std::sort(sorted.begin(), sorted.end(), [](double a, double b) { return a > b; });
        // a further copy of the r-th value changes no value of the top r (and
        // that eigenspace has no unique r-dimensional part): stop unless the
        // deflated operator still has an eigenvalue above the r-th one
        if (!(hc.theta[0] > sorted[r - 1] + 1e-8 * tn)) break;
      }
      const int q = verify ? 1 : hc.nvalid;
      if (L + q > p.lmax) return fail(LRQ_ENOCONV, "lrq_truncate: more repeated eigenvalues than locking slots");
      lz_ritz<T><<<lz_rows_grid(n), kLzThreads, 0, st>>>(U(), n, L, hc.J, X(), p.ldx, q, Y());
      count_launch();
      if ((e = cuda_check(cudaMemcpyAsync(col(L), Y(), static_cast<size_t>(q) * n * sizeof(T),
                                          cudaMemcpyDeviceToDevice, st),
                          "copy Ritz vectors")))
        return e;
      for (int a = 0; a < q; ++a) vals.push_back(hc.theta[a]);
      L += q;
    }
    // the r largest locked pairs, descending
    std::vector<int> order(vals.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int>(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return vals[a] > vals[b]; });
    LzOutput o;
    std::memset(&o, 0, sizeof(o));
    o.r = r;
    double lam_host[kLzWant];
    for (int j = 0; j < r; ++j) {
      if (j < static_cast<int>(order.size())) {
        o.col[j] = order[j];
        o.lam[j] = vals[order[j]];
      } else {
        o.col[j] = -1;
        o.lam[j] = 0.0;
      }
      lam_host[j] = o.lam[j];
    }
    if (V || V32) {
      lz_output<T><<<lz_rows_grid(n), kLzThreads, 0, st>>>(U(), n, o, V, V32);
      count_launch();
    }
    if ((e = cuda_check(cudaMemcpyAsync(lambda_out, lam_host, r * sizeof(double), cudaMemcpyHostToDevice, st),
                        "copy eigenvalues")))
      return e;
    if ((e = cuda_check(cudaStreamSynchronize(st), "lanczos sync"))) return e;
    if (iters_out) *iters_out = steps;
    return LRQ_OK;
  }
};

template <>
void LzRun<double>::matvec(const double* x, double* y) const {
  lz_matvec_laplacian<<<lz_rows_grid(n), kLzThreads, 0, st>>>(rowptr, colidx, wts, deg(), n, nnz, x, y, state());
  count_launch();
}

template <>
void LzRun<double>::prepare() const {
  lz_degree<<<lz_rows_grid(n), kLzThreads, 0, st>>>(rowptr, colidx, wts, n, nnz, deg());
  count_launch();
}

template <>
void LzRun<double2>::prepare() const {}

template <>
void LzRun<double2>::matvec(const double2* x, double2* y) const {
  const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8), 152 * 16)));
  lz_matvec_dense<<<blocks, kLzThreads, 0, st>>>(Q, n, ld, x, y, state());
  count_launch();
}

}  // namespace

int truncate_check(const lrq_matrix* Q, int r, int max_iter) {
  if (!Q) return fail(LRQ_EINVAL, "Q is NULL");
  if (Q->kind != LRQ_MATRIX_DENSE_C128 && Q->kind != LRQ_MATRIX_CSR_LAPLACIAN)
    return fail(LRQ_EINVAL, "unknown matrix kind");
  if (Q->n < 1) return fail(LRQ_EINVAL, "n must be >= 1");
  if (r < 1 || r > kLzWant || r > Q->n) return fail(LRQ_EINVAL, "r must be in [1, min(8, n)]");
  if (max_iter < 0 || max_iter > kLzMaxIter) return fail(LRQ_EINVAL, "max_iter must be in [0, 4096]");
  if (Q->kind == LRQ_MATRIX_DENSE_C128) {
    if (!Q->values) return fail(LRQ_EINVAL, "dense values pointer is NULL");
    if (Q->ld < Q->n) return fail(LRQ_EINVAL, "ld must be >= n");
    if (Q->n > (int64_t(1) << 20)) return fail(LRQ_EUNSUPPORTED, "dense n above 2^20");
  } else {
    if (!Q->rowptr || (Q->nnz > 0 && !Q->colidx)) return fail(LRQ_EINVAL, "CSR pointer is NULL");
    if (Q->nnz < 0 || Q->nnz >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "nnz must be in [0, 2^31)");
    if (Q->n >= (int64_t(1) << 31)) return fail(LRQ_EINVAL, "CSR n must be below 2^31");
  }
  return LRQ_OK;
}

size_t truncate_workspace_bytes(const lrq_matrix* Q, int r, int max_iter) {
  LzPlan p;
  const int it = static_cast<int>(std::min<int64_t>(max_iter > 0 ? max_iter : kLzDefaultIter, Q->n));
  lz_plan(Q->n, r, it, Q->kind == LRQ_MATRIX_DENSE_C128, &p);
  return p.total;
}

namespace {
// the side stream and event of one truncation call, released on every path
struct LzSide {
  cudaStream_t side = nullptr;
  cudaEvent_t ev = nullptr, done = nullptr;
  int init() {
    int e = cuda_check(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking), "create check stream");
    if (e) return e;
    if ((e = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "create step event"))) return e;
    return cuda_check(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "create check event");
  }
  ~LzSide() {
    if (side) cudaStreamSynchronize(side);
    if (done) cudaEventDestroy(done);
    if (ev) cudaEventDestroy(ev);
    if (side) cudaStreamDestroy(side);
  }
};
}  // namespace

int launch_truncate(const lrq_matrix* Q, int r, double tol, int max_iter, uint64_t seed, double2* V, float2* V32,
                    double* lambda_out, int64_t* iters_out, void* ws, int32_t* status, cudaStream_t st) {
  const int it = static_cast<int>(std::min<int64_t>(max_iter > 0 ? max_iter : kLzDefaultIter, Q->n));
  const double t = tol > 0.0 ? tol : 1e-10;
  LzSide sd;
  int e = sd.init();
  if (e) return e;
  if (Q->kind == LRQ_MATRIX_DENSE_C128) {
    LzRun<double2> R;
    R.dense = true;
    R.Q = static_cast<const double2*>(Q->values);
    R.ld = Q->ld;
    R.rowptr = nullptr;
    R.colidx = nullptr;
    R.wts = nullptr;
    R.nnz = 0;
    R.n = Q->n;
    R.tol = t;
    R.seed = seed;
    lz_plan(Q->n, r, it, true, &R.p);
    R.ws = static_cast<uint8_t*>(ws);
    R.status = status;
    R.st = st;
    R.side = sd.side;
    R.ev = sd.ev;
    R.done = sd.done;
    lz_check_dense<<<lz_rows_grid(Q->n * Q->n), kLzThreads, 0, st>>>(R.Q, Q->n, Q->ld, status);
    count_launch();
    return R.solve(r, lambda_out, V, V32, iters_out);
  }
  LzRun<double> R;
  R.dense = false;
  R.Q = nullptr;
  R.ld = 0;
  R.rowptr = Q->rowptr;
  R.colidx = Q->colidx;
  R.wts = Q->weights;
  R.nnz = Q->nnz;
  R.n = Q->n;
  R.tol = t;
  R.seed = seed;
  lz_plan(Q->n, r, it, false, &R.p);
  R.ws = static_cast<uint8_t*>(ws);
  R.status = status;
  R.st = st;
  R.side = sd.side;
  R.ev = sd.ev;
  R.done = sd.done;
  lz_check_csr<<<lz_rows_grid(std::max<int64_t>(Q->n, Q->nnz)), kLzThreads, 0, st>>>(Q->rowptr, Q->colidx,
                                                                                     Q->weights, Q->n, Q->nnz,
                                                                                     status);
  count_launch();
  return R.solve(r, lambda_out, V, V32, iters_out);
}

}  // namespace lrq
