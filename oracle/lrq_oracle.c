/*
 * lrq_oracle.c -- plain, slow, FP64 CPU oracle for the low-rank discrete
 * quadratic maximisation method of arXiv 2602.20376
 * ("Exploiting Low-Rank Objective Structure in Discrete Quadratic Optimization").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs use it.  It shares no code with the CUDA
 * library (no headers, no helpers, no tables).
 *
 * Every function below computes the plain definition of what the paper
 * states, in FP64, with no blocking, fusion or reordering beyond what the
 * definition needs:
 *
 *   alphabet       A_K = { exp(2 pi i k / K) }                     (Sec. 1, Eq. 2)
 *   objective      z^H Q z = || V^H z ||^2 with Q = V V^H          (Sec. 2.2, Eq. 3)
 *   decision rule  k_i = argmin_k | 2 pi k / K - arg(V_i c) |_mod 2pi   (Sec. 3, Eq. 9)
 *                  computed as argmax_k Re(conj(omega^k) V_i c), which is the
 *                  same index (cos is decreasing in the angular distance);
 *                  ties keep the smallest k, w = 0 gives k = 0.
 *   sampled score  f(c) = || V^H z(c) ||^2                         (Sec. 4.2, Eq. 10)
 *   Max-K-Cut      cut(z) = #{ edges {i,j} : k_i != k_j }           (Sec. 1)
 *   sampler        c = Z / ||Z||, Z ~ CN(0, I_r)  (Lemma "innerIsBeta", App. E)
 *                  with Z drawn by Philox4x32-10 (Salmon et al., SC'11) and
 *                  the Box-Muller transform.
 *
 * Sums over the n coordinates use pairwise (binary-tree) summation, built
 * leaf by leaf with an O(log n) stack, so that the FP64 rounding error is
 * O(log n * eps).
 *
 * Complex arrays are interleaved (re, im) doubles, row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Pairwise summation of vectors of `dim` doubles.                           */
/* Leaves are pushed one at a time; two partial sums of equal height are     */
/* merged, which reproduces the balanced binary tree of pairwise summation.  */
/* ------------------------------------------------------------------------ */
#define PW_MAX_LEVELS 64
#define PW_MAX_DIM 32
typedef struct {
  int top;
  int dim;
  int height[PW_MAX_LEVELS];
  double val[PW_MAX_LEVELS][PW_MAX_DIM];
} pairwise_t;

static void pw_init(pairwise_t* p, int dim) {
  p->top = 0;
  p->dim = dim;
}

static void pw_push(pairwise_t* p, const double* leaf) {
  int t = p->top;
  memcpy(p->val[t], leaf, sizeof(double) * p->dim);
  p->height[t] = 0;
  p->top = t + 1;
  while (p->top >= 2 && p->height[p->top - 1] == p->height[p->top - 2]) {
    int a = p->top - 2, b = p->top - 1;
    for (int d = 0; d < p->dim; ++d) p->val[a][d] += p->val[b][d];
    p->height[a] += 1;
    p->top -= 1;
  }
}

static void pw_result(pairwise_t* p, double* out) {
  for (int d = 0; d < p->dim; ++d) out[d] = 0.0;
  /* fold the remaining (unequal-height) partial sums, smallest first */
  for (int t = p->top - 1; t >= 0; --t)
    for (int d = 0; d < p->dim; ++d) out[d] += p->val[t][d];
}

/* ------------------------------------------------------------------------ */
/* Decision rule (Eq. 9): nearest K-th root of unity in angle.               */
/* ------------------------------------------------------------------------ */
int oracle_decide(double x, double y, int K) {
  int best = 0;
  double best_val = x; /* k = 0: Re(w) */
  for (int k = 1; k < K; ++k) {
    double a = 2.0 * ORACLE_PI * (double)k / (double)K;
    double v = x * cos(a) + y * sin(a); /* Re(conj(omega^k) * w) */
    if (v > best_val) {
      best_val = v;
      best = k;
    }
  }
  return best;
}

/* Angular distance of arg(w) to the nearest decision boundary
 * theta_m = pi (2m+1) / K (Sec. 2.3).  w = 0 lies on every boundary and
 * reports 0. */
double oracle_boundary_margin(double x, double y, int K) {
  if (x == 0.0 && y == 0.0) return 0.0;
  double th = atan2(y, x); /* (-pi, pi] */
  double best = INFINITY;
  for (int m = 0; m < K; ++m) {
    double b = ORACLE_PI * (double)(2 * m + 1) / (double)K;
    double d = fmod(fabs(th - b), 2.0 * ORACLE_PI);
    if (d > ORACLE_PI) d = 2.0 * ORACLE_PI - d;
    if (d < best) best = d;
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* Objective || V^H z ||^2 for codes z (Eq. 3).                              */
/* ------------------------------------------------------------------------ */
double oracle_objective(const double* V, int64_t n, int r, int K, const uint8_t* z) {
  pairwise_t pw;
  pw_init(&pw, 2 * r);
  double leaf[PW_MAX_DIM];
  for (int64_t i = 0; i < n; ++i) {
    double a = 2.0 * ORACLE_PI * (double)z[i] / (double)K;
    double zr = cos(a), zi = sin(a);
    for (int j = 0; j < r; ++j) {
      double vr = V[2 * (i * r + j)], vi = V[2 * (i * r + j) + 1];
      /* conj(V_ij) * z_i */
      leaf[2 * j] = vr * zr + vi * zi;
      leaf[2 * j + 1] = vr * zi - vi * zr;
    }
    pw_push(&pw, leaf);
  }
  double s[PW_MAX_DIM];
  pw_result(&pw, s);
  double f = 0.0;
  for (int j = 0; j < 2 * r; ++j) f += s[j] * s[j];
  return f;
}

/* ------------------------------------------------------------------------ */
/* Candidate scoring (Eq. 9 + Eq. 10): for each direction c_s,              */
/*   w_i = V_i c_s,  k_i = decide(w_i),  f_s = || V^H z ||^2.               */
/* z_out (optional, S x n codes) receives the assignments.                   */
/* ------------------------------------------------------------------------ */
int oracle_score(const double* V, int64_t n, int r, int K, const double* C, int64_t S,
                 double* f_out, uint8_t* z_out, int nthreads) {
  if (r < 1 || 2 * r > PW_MAX_DIM || K < 2) return 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t s = 0; s < S; ++s) {
    const double* c = C + 2 * s * r;
    pairwise_t pw;
    pw_init(&pw, 2 * r);
    double leaf[PW_MAX_DIM];
    for (int64_t i = 0; i < n; ++i) {
      const double* v = V + 2 * i * r;
      double x = 0.0, y = 0.0;
      for (int j = 0; j < r; ++j) {
        x += v[2 * j] * c[2 * j] - v[2 * j + 1] * c[2 * j + 1];
        y += v[2 * j] * c[2 * j + 1] + v[2 * j + 1] * c[2 * j];
      }
      int k = oracle_decide(x, y, K);
      if (z_out) z_out[s * n + i] = (uint8_t)k;
      double a = 2.0 * ORACLE_PI * (double)k / (double)K;
      double zr = cos(a), zi = sin(a);
      for (int j = 0; j < r; ++j) {
        leaf[2 * j] = v[2 * j] * zr + v[2 * j + 1] * zi;
        leaf[2 * j + 1] = v[2 * j] * zi - v[2 * j + 1] * zr;
      }
      pw_push(&pw, leaf);
    }
    double acc[PW_MAX_DIM];
    pw_result(&pw, acc);
    double f = 0.0;
    for (int j = 0; j < 2 * r; ++j) f += acc[j] * acc[j];
    f_out[s] = f;
  }
  return 0;
}

/* Decision rule applied to arrays of (x, y) pairs. */
void oracle_decide_array(const double* x, const double* y, int64_t m, int K, uint8_t* k_out) {
  for (int64_t t = 0; t < m; ++t) k_out[t] = (uint8_t)oracle_decide(x[t], y[t], K);
}

/* Angle margin of every (candidate, coordinate) entry; used by the parity
 * tests to exclude entries that sit within a tolerance of a boundary. */
int oracle_margins(const double* V, int64_t n, int r, int K, const double* C, int64_t S,
                   double* margin_out, double* absw_out) {
  for (int64_t s = 0; s < S; ++s) {
    const double* c = C + 2 * s * r;
    for (int64_t i = 0; i < n; ++i) {
      const double* v = V + 2 * i * r;
      double x = 0.0, y = 0.0;
      for (int j = 0; j < r; ++j) {
        x += v[2 * j] * c[2 * j] - v[2 * j + 1] * c[2 * j + 1];
        y += v[2 * j] * c[2 * j + 1] + v[2 * j + 1] * c[2 * j];
      }
      margin_out[s * n + i] = oracle_boundary_margin(x, y, K);
      if (absw_out) absw_out[s * n + i] = hypot(x, y);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Brute force over all K^n assignments (the definition of OPT, Eq. 1).     */
/* ------------------------------------------------------------------------ */
double oracle_bruteforce(const double* V, int64_t n, int r, int K, uint8_t* z_best) {
  uint8_t* z = (uint8_t*)calloc((size_t)n, 1);
  double best = -1.0;
  for (;;) {
    double f = oracle_objective(V, n, r, K, z);
    if (f > best) {
      best = f;
      memcpy(z_best, z, (size_t)n);
    }
    /* next assignment in base-K counting order */
    int64_t i = 0;
    while (i < n) {
      z[i] += 1;
      if (z[i] < K) break;
      z[i] = 0;
      ++i;
    }
    if (i == n) break;
  }
  free(z);
  return best;
}

/* Brute force of the quadratic form z^H Q z for a dense Hermitian Q (n x n
 * interleaved complex), used to pin the factorised objective and the
 * Laplacian/cut identity on tiny instances. */
double oracle_quadform(const double* Q, int64_t n, int K, const uint8_t* z) {
  double acc = 0.0;
  for (int64_t a = 0; a < n; ++a) {
    double ta = 2.0 * ORACLE_PI * (double)z[a] / (double)K;
    double za_r = cos(ta), za_i = sin(ta);
    for (int64_t b = 0; b < n; ++b) {
      double tb = 2.0 * ORACLE_PI * (double)z[b] / (double)K;
      double zb_r = cos(tb), zb_i = sin(tb);
      double qr = Q[2 * (a * n + b)], qi = Q[2 * (a * n + b) + 1];
      /* conj(z_a) * Q_ab * z_b, real part */
      double t_r = qr * zb_r - qi * zb_i;
      double t_i = qr * zb_i + qi * zb_r;
      acc += za_r * t_r + za_i * t_i;
    }
  }
  return acc;
}

double oracle_quadform_bruteforce(const double* Q, int64_t n, int K, uint8_t* z_best) {
  uint8_t* z = (uint8_t*)calloc((size_t)n, 1);
  double best = -INFINITY;
  for (;;) {
    double f = oracle_quadform(Q, n, K, z);
    if (f > best) {
      best = f;
      memcpy(z_best, z, (size_t)n);
    }
    int64_t i = 0;
    while (i < n) {
      z[i] += 1;
      if (z[i] < K) break;
      z[i] = 0;
      ++i;
    }
    if (i == n) break;
  }
  free(z);
  return best;
}

/* ------------------------------------------------------------------------ */
/* Max-K-Cut count on a symmetric CSR graph (Sec. 1: K = 3 with a Laplacian  */
/* objective is Max-3-Cut).  Each undirected edge is stored twice; it is    */
/* counted once, from its lower endpoint.  Self loops never count.          */
/* ------------------------------------------------------------------------ */
int64_t oracle_cut_count(const int32_t* rowptr, const int32_t* colidx, int64_t n, const uint8_t* z) {
  int64_t cut = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int64_t j = colidx[e];
      if (j > i && z[i] != z[j]) ++cut;
    }
  return cut;
}

/* z^H L z for the unit-weight Laplacian L = D - A of a symmetric CSR graph,
 * computed as sum over stored entries of the definition of L.            */
double oracle_laplacian_quadform(const int32_t* rowptr, const int32_t* colidx, int64_t n, int K,
                                 const uint8_t* z) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double ti = 2.0 * ORACLE_PI * (double)z[i] / (double)K;
    double zr_i = cos(ti), zi_i = sin(ti);
    double deg = (double)(rowptr[i + 1] - rowptr[i]);
    acc += deg; /* |z_i|^2 D_ii */
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int64_t j = colidx[e];
      double tj = 2.0 * ORACLE_PI * (double)z[j] / (double)K;
      /* - Re(conj(z_i) z_j) for A_ij = 1 */
      acc -= zr_i * cos(tj) + zi_i * sin(tj);
    }
  }
  return acc;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): 10 rounds of a multiply-xor round function on  */
/* a 128-bit counter under a 64-bit key; the key advances by the Weyl       */
/* constants before every round after the first.                            */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Uniform (0,1) double from two 32-bit words: top 53 bits, centred. */
static double u53(uint32_t hi, uint32_t lo) {
  uint64_t x = (((uint64_t)hi << 32) | (uint64_t)lo) >> 11;
  return ((double)x + 0.5) * (1.0 / 9007199254740992.0);
}

/* Uniform directions on the complex unit sphere of C^r.
 * Candidate s, component j: one Philox block with counter
 * (lo32(s), hi32(s), j, 0) and key (lo32(seed), hi32(seed)); words 0,1 give
 * u1, words 2,3 give u2; Z_j = sqrt(-ln u1) * exp(2 pi i u2), so that
 * Re Z_j, Im Z_j ~ N(0, 1/2) independently (complex Gaussian CN(0,1)).
 * c_s = Z / ||Z||, written as doubles. */
void oracle_sphere_sample(uint64_t seed, int64_t S, int r, double* C_out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t s = 0; s < S; ++s) {
    double zr[64], zi[64];
    double nrm2 = 0.0;
    for (int j = 0; j < r; ++j) {
      uint32_t ctr[4] = {(uint32_t)s, (uint32_t)((uint64_t)s >> 32), (uint32_t)j, 0u};
      uint32_t o[4];
      oracle_philox4x32_10(ctr, key, o);
      double u1 = u53(o[0], o[1]);
      double u2 = u53(o[2], o[3]);
      double rad = sqrt(-log(u1));
      zr[j] = rad * cos(2.0 * ORACLE_PI * u2);
      zi[j] = rad * sin(2.0 * ORACLE_PI * u2);
      nrm2 += zr[j] * zr[j] + zi[j] * zi[j];
    }
    double inv = 1.0 / sqrt(nrm2);
    for (int j = 0; j < r; ++j) {
      C_out[2 * (s * r + j)] = zr[j] * inv;
      C_out[2 * (s * r + j) + 1] = zi[j] * inv;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Exact rank-1 sweep (Sec. 2.5, Algorithm 1, Theorem 2.1).                 */
/* For q in C^n: theta_i = arg q_i; the assignment at phi = -pi/K is        */
/* k_i = floor(K theta_i / 2pi) mod K; coordinate i changes to k_i + 1 when */
/* phi passes its boundary point                                             */
/*   phi_i = (2pi/K) (1/2 + floor(K theta_i/2pi) - K theta_i/2pi).           */
/* Visiting the boundary points in increasing order gives the n+1 cells;    */
/* the best of the n+1 assignments under |z^H q|^2 is returned.             */
/* ------------------------------------------------------------------------ */
typedef struct {
  double phi;
  int64_t idx;
} phi_idx_t;

static int cmp_phi(const void* a, const void* b) {
  double x = ((const phi_idx_t*)a)->phi, y = ((const phi_idx_t*)b)->phi;
  if (x < y) return -1;
  if (x > y) return 1;
  int64_t i = ((const phi_idx_t*)a)->idx, j = ((const phi_idx_t*)b)->idx;
  return (i > j) - (i < j);
}

double oracle_rank1_sweep(const double* q, int64_t n, int K, uint8_t* z_best) {
  phi_idx_t* bp = (phi_idx_t*)malloc(sizeof(phi_idx_t) * (size_t)n);
  uint8_t* k = (uint8_t*)malloc((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    double th = atan2(q[2 * i + 1], q[2 * i]);
    double t = (double)K * th / (2.0 * ORACLE_PI);
    double fl = floor(t);
    bp[i].phi = (2.0 * ORACLE_PI / (double)K) * (0.5 + fl - t);
    bp[i].idx = i;
    long kk = ((long)fl) % K;
    if (kk < 0) kk += K;
    k[i] = (uint8_t)kk;
  }
  qsort(bp, (size_t)n, sizeof(phi_idx_t), cmp_phi);
  /* q as an n x 1 factor: objective |z^H q|^2 = || q^H z ||^2 */
  double best = oracle_objective(q, n, 1, K, k);
  memcpy(z_best, k, (size_t)n);
  for (int64_t l = 0; l < n; ++l) {
    int64_t i = bp[l].idx;
    k[i] = (uint8_t)((k[i] + 1) % K);
    double f = oracle_objective(q, n, 1, K, k);
    if (f > best) {
      best = f;
      memcpy(z_best, k, (size_t)n);
    }
  }
  free(bp);
  free(k);
  return best;
}

/* --------------------------------------------------------------------------
 * Sequential steepest ascent for Max-K-Cut (App. "Hybrid Warm-Start" names
 * steepest ascent without fixing how moves are grouped): repeatedly take the
 * single vertex with the largest gain g_i = n_i(z_i) - min_{c != z_i} n_i(c)
 * (n_i(c): neighbours of i with label c over the CSR adjacency, self loops
 * ignored, parallel edges with multiplicity; ties to the smaller index) and
 * move it to the smallest label attaining the minimum, until no vertex gains
 * or max_moves moves were made (max_moves < 0: no limit).  The cut rises by
 * g_i with each move.  A binary max-heap of (gain, index) keys with lazy
 * deletion finds the steepest vertex.  Returns the number of moves, or -1 on
 * a label outside [0, K) or an allocation failure; z is updated in place.
 * ------------------------------------------------------------------------ */
static int64_t gs_key(int64_t gain, int64_t i) { return (gain << 32) | (int64_t)(0xFFFFFFFFu - (uint32_t)i); }

static int gs_push(int64_t** heap, int64_t* size, int64_t* cap, int64_t key) {
  if (*size == *cap) {
    int64_t nc = *cap * 2 + 16;
    int64_t* nh = (int64_t*)realloc(*heap, (size_t)nc * sizeof(int64_t));
    if (!nh) return -1;
    *heap = nh;
    *cap = nc;
  }
  int64_t* h = *heap;
  int64_t k = (*size)++;
  h[k] = key;
  while (k > 0) {
    int64_t p = (k - 1) / 2;
    if (h[p] >= h[k]) break;
    int64_t t = h[p];
    h[p] = h[k];
    h[k] = t;
    k = p;
  }
  return 0;
}

static int64_t gs_pop(int64_t* h, int64_t* size) {
  int64_t top = h[0];
  h[0] = h[--(*size)];
  int64_t k = 0;
  for (;;) {
    int64_t l = 2 * k + 1, r = l + 1, m = k;
    if (l < *size && h[l] > h[m]) m = l;
    if (r < *size && h[r] > h[m]) m = r;
    if (m == k) break;
    int64_t t = h[m];
    h[m] = h[k];
    h[k] = t;
    k = m;
  }
  return top;
}

static int64_t gs_gain(const int32_t* cnt, int K, int zi, int* best) {
  int b = -1;
  for (int c = 0; c < K; ++c)
    if (c != zi && (b < 0 || cnt[c] < cnt[b])) b = c;
  *best = b;
  return (int64_t)cnt[zi] - cnt[b];
}

int64_t oracle_greedy_sequential(const int32_t* rowptr, const int32_t* colidx, int64_t n, int K, uint8_t* z,
                                 int64_t max_moves) {
  if (K < 2 || n < 0) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (z[i] >= K) return -1;
  int32_t* cnt = (int32_t*)calloc((size_t)(n > 0 ? n : 1) * K, sizeof(int32_t));
  int64_t* gain = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t cap = n + 16, size = 0;
  int64_t* heap = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
  if (!cnt || !gain || !heap) {
    free(cnt);
    free(gain);
    free(heap);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (colidx[e] != i) cnt[i * K + z[colidx[e]]] += 1;
  int64_t rc = 0;
  for (int64_t i = 0; i < n && rc == 0; ++i) {
    int b;
    gain[i] = gs_gain(cnt + i * K, K, z[i], &b);
    if (gain[i] > 0) rc = gs_push(&heap, &size, &cap, gs_key(gain[i], i));
  }
  int64_t moves = 0;
  while (rc == 0 && size > 0 && (max_moves < 0 || moves < max_moves)) {
    const int64_t key = gs_pop(heap, &size);
    const int64_t g = key >> 32;
    const int64_t i = 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFF);
    if (g != gain[i] || g <= 0) continue;  // a stale entry
    int b;
    gs_gain(cnt + i * K, K, z[i], &b);
    const int old = z[i];
    z[i] = (uint8_t)b;
    ++moves;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t j = colidx[e];
      if (j == i) continue;
      cnt[j * K + old] -= 1;
      cnt[j * K + b] += 1;
    }
    int bi;
    gain[i] = gs_gain(cnt + i * K, K, z[i], &bi);
    if (gain[i] > 0) rc = gs_push(&heap, &size, &cap, gs_key(gain[i], i));
    for (int32_t e = rowptr[i]; e < rowptr[i + 1] && rc == 0; ++e) {
      const int64_t j = colidx[e];
      if (j == i) continue;
      int bj;
      const int64_t gj = gs_gain(cnt + j * K, K, z[j], &bj);
      if (gj != gain[j]) {
        gain[j] = gj;
        if (gj > 0) rc = gs_push(&heap, &size, &cap, gs_key(gj, j));
      }
    }
  }
  free(cnt);
  free(gain);
  free(heap);
  return rc == 0 ? moves : -1;
}
