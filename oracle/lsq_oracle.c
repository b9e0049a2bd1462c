/*
 * lsq_oracle.c -- plain, slow, FP64 CPU oracle for the randomized-preconditioned
 * least-squares method of Lacotte & Pilanci, "Faster Least Squares Optimization"
 * (arXiv 1911.02675).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the CUDA
 * path: every routine below is written from the paper (and, for the random number
 * generator, from its published definition) in the most direct form available.
 *
 * Problem (Section 1, eq. eqnconvexquadratic): x* = argmin 1/2 <x,Hx> - <b,x>,
 * H = A^T A, A n-by-d (row-major, contiguous rows of stride ld), b in R^d.
 *
 * Conventions fixed here where the paper is silent (each one is listed with its
 * reason in the design notes of the repository):
 *   - every sketch is scaled so that E[S^T S] = I_n;
 *   - Philox4x32-10 key = (seed lo, seed hi); counter word 2 = sketch instance t,
 *     counter word 3 = a stream tag (1 Gaussian, 2 SRHT sign, 3 SRHT sample key,
 *     4 SJLT position, 5 SJLT sign);
 *   - SRHT rows: the m smallest 64-bit sample keys (ties by index), stored in
 *     ascending row order; Hadamard in natural (Sylvester) order, zero padding to
 *     the next power of two N, scale 1/sqrt(m) on the +-1 matrix;
 *   - SJLT positions: Lemire's bounded integer from successive Philox words,
 *     duplicates skipped, until s distinct rows; sign k = bit k of one more word;
 *   - Gaussian entry z(j,i) of sketch row j, data row i: Box-Muller on the words of
 *     Philox(i, j/2, t, 1); even j takes the cosine branch, odd j the sine branch.
 *
 * Every floating-point routine is FP64 (double-double where it says so).
 * Parity status: every function here is pinned by a test in tests/test_oracle_*.py
 * against values or identities that do not come from this file (see each header).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TAG_GAUSS 1u
#define ORC_TAG_SIGN 2u
#define ORC_TAG_SAMPLE 3u
#define ORC_TAG_SJLT 4u
#define ORC_TAG_SJLT_SIGN 5u

/* status codes, same meaning as the library's */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_RANK 2
#define ORC_ERR_BREAKDOWN 3
#define ORC_ERR_MAXIT 4

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the  */
/* published multipliers, key bumped by the published Weyl constants.         */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_at(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t t, uint32_t tag, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, t, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

void orc_philox_batch(int64_t count, const uint32_t* ctrs, const uint32_t key[2], uint32_t* out) {
  for (int64_t k = 0; k < count; ++k) orc_philox4x32_10(ctrs + 4 * k, key, out + 4 * k);
}

/* ------------------------------------------------------------------------ */
/* Gaussian embedding, Section 2: iid N(0, 1/m) entries.                     */
/* ------------------------------------------------------------------------ */
static double unit_open(uint32_t hi, uint32_t lo) {
  /* 53 random bits -> the open interval (0,1): (k + 1/2) 2^-53 */
  uint64_t k = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
  return ((double)k + 0.5) * (1.0 / 9007199254740992.0);
}

/* standard normal z(j,i) by Box-Muller (Box & Muller 1958) */
double orc_gauss_z(uint64_t seed, uint32_t t, int64_t j, int64_t i) {
  uint32_t w[4];
  philox_at(seed, (uint32_t)i, (uint32_t)(j >> 1), t, ORC_TAG_GAUSS, w);
  double u1 = unit_open(w[0], w[1]);
  double u2 = unit_open(w[2], w[3]);
  double radius = sqrt(-2.0 * log(u1));
  double angle = 2.0 * M_PI * u2;
  return (j & 1) ? radius * sin(angle) : radius * cos(angle);
}

/* explicit S (m x n, row-major): S[j,i] = z(j,i)/sqrt(m) */
void orc_gauss_matrix(int64_t m, int64_t n, uint64_t seed, uint32_t t, double* S) {
  double scale = 1.0 / sqrt((double)m);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < n; ++i) S[j * n + i] = scale * orc_gauss_z(seed, t, j, i);
}

/* SA = S A with S generated entry by entry; plain triple loop (a matmul). */
void orc_sketch_gauss(const double* A, int64_t n, int64_t d, int64_t ld, int64_t m, uint64_t seed,
                      uint32_t t, double* SA) {
  double scale = 1.0 / sqrt((double)m);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < m; ++j) {
    double* out = SA + j * d;
    for (int64_t c = 0; c < d; ++c) out[c] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = scale * orc_gauss_z(seed, t, j, i);
      const double* a = A + i * ld;
      for (int64_t c = 0; c < d; ++c) out[c] += s * a[c];
    }
  }
}

/* Rows `rows[0..k-1]` of SA = S A for the m x n Gaussian S above (the same entries
   z(j,i)/sqrt(m)), without the other rows: a row sample of the sketch, for checks and timing
   of the sketch at sizes where all m rows would take too long. */
void orc_sketch_gauss_rows(const double* A, int64_t n, int64_t d, int64_t ld, int64_t m, uint64_t seed,
                           uint32_t t, const int64_t* rows, int64_t k, double* SA_rows) {
  double scale = 1.0 / sqrt((double)m);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < k; ++r) {
    int64_t j = rows[r];
    double* out = SA_rows + r * d;
    for (int64_t c = 0; c < d; ++c) out[c] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = scale * orc_gauss_z(seed, t, j, i);
      const double* a = A + i * ld;
      for (int64_t c = 0; c < d; ++c) out[c] += s * a[c];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* SRHT, Section 2: S = R H E (row sampling without replacement, Hadamard,   */
/* random signs), zero padding of n to N = 2^ceil(log2 n) (footnote there).   */
/* ------------------------------------------------------------------------ */
int64_t orc_next_pow2(int64_t n) {
  int64_t N = 1;
  while (N < n) N <<= 1;
  return N;
}

/* E: sign_i = +1 if bit 0 of the first word of Philox(i, 0, t, 2) is 0, else -1 */
void orc_srht_signs(int64_t N, uint64_t seed, uint32_t t, int8_t* sgn) {
  for (int64_t i = 0; i < N; ++i) {
    uint32_t w[4];
    philox_at(seed, (uint32_t)i, (uint32_t)(i >> 32), t, ORC_TAG_SIGN, w);
    sgn[i] = (w[0] & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

typedef struct {
  uint64_t key;
  int64_t idx;
} keyed_row;

static int cmp_keyed(const void* a, const void* b) {
  const keyed_row* x = (const keyed_row*)a;
  const keyed_row* y = (const keyed_row*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* R: the m rows (of N) with the smallest (key, index), key = 64-bit Philox word
   pair of Philox(i, 0, t, 3); returned sorted ascending. A uniformly random m-subset. */
void orc_srht_rows(int64_t N, int64_t m, uint64_t seed, uint32_t t, int64_t* rows) {
  keyed_row* all = (keyed_row*)malloc(sizeof(keyed_row) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    uint32_t w[4];
    philox_at(seed, (uint32_t)i, (uint32_t)(i >> 32), t, ORC_TAG_SAMPLE, w);
    all[i].key = (((uint64_t)w[0]) << 32) | (uint64_t)w[1];
    all[i].idx = i;
  }
  qsort(all, (size_t)N, sizeof(keyed_row), cmp_keyed);
  for (int64_t r = 0; r < m; ++r) rows[r] = all[r].idx;
  qsort(rows, (size_t)m, sizeof(int64_t), cmp_i64);
  free(all);
}

/* unnormalised Sylvester Hadamard transform along the rows of X (N x d):
   for each column, the length-N fast Walsh-Hadamard transform */
void orc_fwht_rows(double* X, int64_t N, int64_t d) {
  for (int64_t h = 1; h < N; h <<= 1) {
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < N; blk += 2 * h) {
      for (int64_t i = blk; i < blk + h; ++i) {
        double* u = X + i * d;
        double* v = X + (i + h) * d;
        for (int64_t c = 0; c < d; ++c) {
          double a = u[c], b = v[c];
          u[c] = a + b;
          v[c] = a - b;
        }
      }
    }
  }
}

int orc_sketch_srht(const double* A, int64_t n, int64_t d, int64_t ld, int64_t m, uint64_t seed,
                    uint32_t t, double* SA) {
  int64_t N = orc_next_pow2(n);
  if (m < 1 || m > N) return ORC_ERR_ARG;
  double* X = (double*)calloc((size_t)(N * d), sizeof(double));
  int8_t* sgn = (int8_t*)malloc((size_t)N);
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  if (!X || !sgn || !rows) { free(X); free(sgn); free(rows); return ORC_ERR_ARG; }
  orc_srht_signs(N, seed, t, sgn);
  /* E A (zero rows beyond n) */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < d; ++c) X[i * d + c] = (double)sgn[i] * A[i * ld + c];
  /* H E A */
  orc_fwht_rows(X, N, d);
  /* R H E A, scaled so that E[S^T S] = I */
  orc_srht_rows(N, m, seed, t, rows);
  double scale = 1.0 / sqrt((double)m);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t c = 0; c < d; ++c) SA[r * d + c] = scale * X[rows[r] * d + c];
  free(X); free(sgn); free(rows);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SJLT, Section 2: for each column of S (one data row i), s rows chosen      */
/* uniformly without replacement, entries +-1/sqrt(s).                        */
/* ------------------------------------------------------------------------ */

/* Lemire, "Fast random integer generation in an interval" (ACM TOMACS 2019):
   returns 1 and the value in [0, range) if word x is accepted, 0 if rejected. */
static int lemire_accept(uint32_t x, uint32_t range, uint32_t* value) {
  uint64_t prod = (uint64_t)x * (uint64_t)range;
  uint32_t low = (uint32_t)prod;
  if (low < range) {
    uint32_t threshold = (uint32_t)(-range) % range;
    if (low < threshold) return 0;
  }
  *value = (uint32_t)(prod >> 32);
  return 1;
}

/* positions h (n x s, each row ascending) and signs (n x s, +-1) */
int orc_sjlt_hash(int64_t n, int64_t m, int s, uint64_t seed, uint32_t t, int32_t* h, int8_t* sg) {
  if (s < 1 || s > 32 || s > m || m > 0x7fffffff) return ORC_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int32_t picked[32];
    int got = 0;
    for (uint32_t draw = 0; got < s; ++draw) {
      uint32_t w[4];
      philox_at(seed, (uint32_t)i, draw, t, ORC_TAG_SJLT, w);
      for (int k = 0; k < 4 && got < s; ++k) {
        uint32_t v;
        if (!lemire_accept(w[k], (uint32_t)m, &v)) continue;
        int dup = 0;
        for (int q = 0; q < got; ++q) dup |= (picked[q] == (int32_t)v);
        if (!dup) picked[got++] = (int32_t)v;
      }
    }
    uint32_t sw[4];
    philox_at(seed, (uint32_t)i, 0u, t, ORC_TAG_SJLT_SIGN, sw);
    int8_t sign_of[32];
    for (int k = 0; k < s; ++k) sign_of[k] = ((sw[0] >> k) & 1u) ? (int8_t)-1 : (int8_t)1;
    /* store sorted by position (insertion sort keeps each sign with its row) */
    for (int a = 1; a < s; ++a) {
      int32_t pv = picked[a];
      int8_t sv = sign_of[a];
      int b = a - 1;
      while (b >= 0 && picked[b] > pv) { picked[b + 1] = picked[b]; sign_of[b + 1] = sign_of[b]; --b; }
      picked[b + 1] = pv;
      sign_of[b + 1] = sv;
    }
    for (int k = 0; k < s; ++k) { h[i * s + k] = picked[k]; sg[i * s + k] = sign_of[k]; }
  }
  return ORC_OK;
}

int orc_sketch_sjlt(const double* A, int64_t n, int64_t d, int64_t ld, int64_t m, int s,
                    uint64_t seed, uint32_t t, double* SA) {
  int32_t* h = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * s));
  int8_t* sg = (int8_t*)malloc((size_t)(n * s));
  if (!h || !sg) { free(h); free(sg); return ORC_ERR_ARG; }
  int st = orc_sjlt_hash(n, m, s, seed, t, h, sg);
  if (st != ORC_OK) { free(h); free(sg); return st; }
  double scale = 1.0 / sqrt((double)s);
  memset(SA, 0, sizeof(double) * (size_t)(m * d));
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < s; ++k) {
      double w = scale * (double)sg[i * s + k];
      double* out = SA + (int64_t)h[i * s + k] * d;
      const double* a = A + i * ld;
      for (int64_t c = 0; c < d; ++c) out[c] += w * a[c];
    }
  free(h); free(sg);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Factorisation of H_S = (SA)^T (SA) = R^T R (Section 1, PCG paragraph;      */
/* Section 6: QR of SA or Cholesky of H_S).                                   */
/* ------------------------------------------------------------------------ */
void orc_gram(const double* M, int64_t m, int64_t d, double* G) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t a = 0; a < d; ++a)
    for (int64_t b = a; b < d; ++b) {
      double s = 0.0;
      for (int64_t r = 0; r < m; ++r) s += M[r * d + a] * M[r * d + b];
      G[a * d + b] = s;
      G[b * d + a] = s;
    }
}

/* upper R with R^T R = G, positive diagonal; returns k+1 if pivot k is not positive */
int orc_cholesky_upper(const double* G, int64_t d, double* R) {
  memset(R, 0, sizeof(double) * (size_t)(d * d));
  for (int64_t j = 0; j < d; ++j) {
    double s = G[j * d + j];
    for (int64_t k = 0; k < j; ++k) s -= R[k * d + j] * R[k * d + j];
    if (!(s > 0.0) || !isfinite(s)) return (int)(j + 1);
    double rjj = sqrt(s);
    R[j * d + j] = rjj;
    for (int64_t i = j + 1; i < d; ++i) {
      double v = G[j * d + i];
      for (int64_t k = 0; k < j; ++k) v -= R[k * d + j] * R[k * d + i];
      R[j * d + i] = v / rjj;
    }
  }
  return 0;
}

/* Householder QR of M (m x d, row-major, m >= d): R upper with positive diagonal.
   Returns k+1 if column k is (numerically) zero. */
int orc_qr_r(const double* M, int64_t m, int64_t d, double* R) {
  double* Q = (double*)malloc(sizeof(double) * (size_t)(m * d)); /* column-major work copy */
  double* v = (double*)malloc(sizeof(double) * (size_t)m);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t c = 0; c < d; ++c) Q[c * m + r] = M[r * d + c];
  memset(R, 0, sizeof(double) * (size_t)(d * d));
  int status = 0;
  for (int64_t k = 0; k < d; ++k) {
    double* col = Q + k * m;
    double norm2 = 0.0;
    for (int64_t r = k; r < m; ++r) norm2 += col[r] * col[r];
    double norm = sqrt(norm2);
    if (!(norm > 0.0)) { status = (int)(k + 1); break; }
    double alpha = col[k] > 0 ? -norm : norm;
    for (int64_t r = k; r < m; ++r) v[r] = col[r];
    v[k] -= alpha;
    double vnorm2 = 0.0;
    for (int64_t r = k; r < m; ++r) vnorm2 += v[r] * v[r];
    /* reflect the remaining columns: x <- x - 2 v (v^T x)/(v^T v) */
#pragma omp parallel for schedule(static)
    for (int64_t c = k; c < d; ++c) {
      double* x = Q + c * m;
      double dot = 0.0;
      for (int64_t r = k; r < m; ++r) dot += v[r] * x[r];
      double f = 2.0 * dot / vnorm2;
      for (int64_t r = k; r < m; ++r) x[r] -= f * v[r];
    }
    for (int64_t c = k; c < d; ++c) R[k * d + c] = Q[c * m + k];
  }
  /* positive diagonal: R <- diag(sign) R (Q absorbs the signs) */
  for (int64_t k = 0; k < d && status == 0; ++k)
    if (R[k * d + k] < 0)
      for (int64_t c = k; c < d; ++c) R[k * d + c] = -R[k * d + c];
  free(Q); free(v);
  return status;
}

/* Householder QR with column pivoting (Businger and Golub, 1965) of M (m x d, row-major,
   m >= d), one of the factorisations of H_S the paper allows (Section 1, PCG paragraph):
   M[:, perm] = Q R, R upper with positive diagonal.  At step k the column of largest
   remaining norm (rows k..m-1, recomputed from its entries; ties to the lower index) is
   moved to position k.  The numerical rank is the number of steps before the largest
   remaining norm falls to tol times the first pivot's norm; rows of R from the rank on
   are zero.  perm[k] = the column of M at position k. */
int orc_qr_pivoted(const double* M, int64_t m, int64_t d, double tol, double* R, int32_t* perm, int64_t* rank) {
  double* Q = (double*)malloc(sizeof(double) * (size_t)(m * d)); /* column-major work copy */
  double* v = (double*)malloc(sizeof(double) * (size_t)m);
  double* nrm = (double*)malloc(sizeof(double) * (size_t)d);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t c = 0; c < d; ++c) Q[c * m + r] = M[r * d + c];
  for (int64_t c = 0; c < d; ++c) perm[c] = (int32_t)c;
  memset(R, 0, sizeof(double) * (size_t)(d * d));
  double first = 0.0;
  int64_t k = 0;
  for (; k < d; ++k) {
    /* remaining column norms, then the pivot */
#pragma omp parallel for schedule(static)
    for (int64_t c = k; c < d; ++c) {
      double s2 = 0.0;
      for (int64_t r = k; r < m; ++r) s2 += Q[c * m + r] * Q[c * m + r];
      nrm[c] = sqrt(s2);
    }
    int64_t p = k;
    for (int64_t c = k + 1; c < d; ++c)
      if (nrm[c] > nrm[p]) p = c;
    if (k == 0) first = nrm[p];
    if (!(nrm[p] > tol * first) || !(nrm[p] > 0.0)) break;
    if (p != k) {
      for (int64_t r = 0; r < m; ++r) {
        double t = Q[k * m + r];
        Q[k * m + r] = Q[p * m + r];
        Q[p * m + r] = t;
      }
      int32_t tp = perm[k]; perm[k] = perm[p]; perm[p] = tp;
      for (int64_t r = 0; r < k; ++r) {
        double t = R[r * d + k];
        R[r * d + k] = R[r * d + p];
        R[r * d + p] = t;
      }
    }
    double* col = Q + k * m;
    double norm = nrm[p];
    double alpha = col[k] > 0 ? -norm : norm;
    for (int64_t r = k; r < m; ++r) v[r] = col[r];
    v[k] -= alpha;
    double vnorm2 = 0.0;
    for (int64_t r = k; r < m; ++r) vnorm2 += v[r] * v[r];
#pragma omp parallel for schedule(static)
    for (int64_t c = k; c < d; ++c) {
      double* x = Q + c * m;
      double dot = 0.0;
      for (int64_t r = k; r < m; ++r) dot += v[r] * x[r];
      double f = 2.0 * dot / vnorm2;
      for (int64_t r = k; r < m; ++r) x[r] -= f * v[r];
    }
    for (int64_t c = k; c < d; ++c) R[k * d + c] = Q[c * m + k];
    if (R[k * d + k] < 0)
      for (int64_t c = k; c < d; ++c) R[k * d + c] = -R[k * d + c];
  }
  *rank = k;
  free(Q); free(v); free(nrm);
  return 0;
}

/* W = R^{-1} for upper-triangular R, by back substitution on the columns of I */
void orc_tri_inv_upper(const double* R, int64_t d, double* W) {
  memset(W, 0, sizeof(double) * (size_t)(d * d));
  for (int64_t col = 0; col < d; ++col) {
    for (int64_t i = col; i >= 0; --i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int64_t k = i + 1; k <= col; ++k) s -= R[i * d + k] * W[k * d + col];
      W[i * d + col] = s / R[i * d + i];
    }
  }
}

/* solve (R^T R) z = r: forward solve R^T y = r, then back solve R z = y */
void orc_precond_solve(const double* R, int64_t d, const double* r, double* z) {
  double* y = (double*)malloc(sizeof(double) * (size_t)d);
  for (int64_t i = 0; i < d; ++i) {
    double s = r[i];
    for (int64_t k = 0; k < i; ++k) s -= R[k * d + i] * y[k];
    y[i] = s / R[i * d + i];
  }
  for (int64_t i = d - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t k = i + 1; k < d; ++k) s -= R[i * d + k] * z[k];
    z[i] = s / R[i * d + i];
  }
  free(y);
}

/* ------------------------------------------------------------------------ */
/* Products with H = A^T A.                                                  */
/* ------------------------------------------------------------------------ */

/* v = A^T (A p), q = ||A p||^2 = p^T H p */
void orc_hmatvec(const double* A, int64_t n, int64_t d, int64_t ld, const double* p, double* v, double* q) {
  int nt = orc_num_threads();
  double* part = (double*)calloc((size_t)nt * (size_t)(d + 1), sizeof(double));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* mine = part + (size_t)tid * (size_t)(d + 1);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const double* a = A + i * ld;
      double w = 0.0;
      for (int64_t c = 0; c < d; ++c) w += a[c] * p[c];
      for (int64_t c = 0; c < d; ++c) mine[c] += a[c] * w;
      mine[d] += w * w;
    }
  }
  for (int64_t c = 0; c <= d; ++c) {
    double s = 0.0;
    for (int k = 0; k < nt; ++k) s += part[(size_t)k * (size_t)(d + 1) + (size_t)c];
    if (c < d) v[c] = s; else *q = s;
  }
  free(part);
}

/* double-double arithmetic: Knuth's TwoSum and the FMA-based TwoProduct
   (Ogita, Rump, Oishi, "Accurate sum and dot product", SISC 2005) */
typedef struct { double hi, lo; } dd_t;

static dd_t two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb);
  dd_t r = {s, err};
  return r;
}

static dd_t dd_add(dd_t x, dd_t y) {
  dd_t s = two_sum(x.hi, y.hi);
  double lo = s.lo + x.lo + y.lo;
  return two_sum(s.hi, lo);
}

static dd_t dd_mul_d(dd_t x, double y) {
  double p = x.hi * y;
  double e = fma(x.hi, y, -p);
  e += x.lo * y;
  return two_sum(p, e);
}

/* r = b - A^T (A x) accumulated in double-double, rounded to FP64 at the end */
void orc_residual_dd(const double* A, int64_t n, int64_t d, int64_t ld, const double* b, const double* x,
                     double* r) {
  int nt = orc_num_threads();
  dd_t* part = (dd_t*)calloc((size_t)nt * (size_t)d, sizeof(dd_t));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    dd_t* mine = part + (size_t)tid * (size_t)d;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const double* a = A + i * ld;
      dd_t w = {0.0, 0.0};
      for (int64_t c = 0; c < d; ++c) {
        dd_t prod = {a[c] * x[c], fma(a[c], x[c], -(a[c] * x[c]))};
        w = dd_add(w, prod);
      }
      for (int64_t c = 0; c < d; ++c) mine[c] = dd_add(mine[c], dd_mul_d(w, a[c]));
    }
  }
  for (int64_t c = 0; c < d; ++c) {
    dd_t s = {b[c], 0.0};
    for (int k = 0; k < nt; ++k) {
      dd_t neg = {-part[(size_t)k * (size_t)d + (size_t)c].hi, -part[(size_t)k * (size_t)d + (size_t)c].lo};
      s = dd_add(s, neg);
    }
    r[c] = s.hi + s.lo;
  }
  free(part);
}

static double dot(const double* a, const double* b, int64_t d) {
  double s = 0.0;
  for (int64_t c = 0; c < d; ++c) s += a[c] * b[c];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Stopping rule (the paper fixes none).  On the event E_rho of Section 3,   */
/* lambda_1(C_S) <= (1+sqrt(rho))^2, and r^T H_S^{-1} r = Delta^T C_S^{-1}    */
/* Delta >= ||Delta||^2 / lambda_1, so ||x - x*||_H^2 <= (1+sqrt(rho))^2 *    */
/* r^T H_S^{-1} r.  <b, x> estimates ||x*||_H^2 = <b, x*>.  Stop when         */
/* (1+sqrt(rho))^2 r^T H_S^{-1} r <= tol^2 <b, x>.                           */
/* ------------------------------------------------------------------------ */
static int converged(double rhat_r, double rho_hat, double tol, double bx) {
  double lam1 = (1.0 + sqrt(rho_hat)) * (1.0 + sqrt(rho_hat));
  return lam1 * rhat_r <= tol * tol * bx;
}

/* optional diagnostics: delta_t = 1/2 ||x_t - x*||_H^2 */
static double half_h_err2(const double* A, int64_t n, int64_t d, int64_t ld, const double* x,
                          const double* xstar, double* scratch_e, double* scratch_v) {
  double q;
  for (int64_t c = 0; c < d; ++c) scratch_e[c] = x[c] - xstar[c];
  orc_hmatvec(A, n, d, ld, scratch_e, scratch_v, &q);
  return 0.5 * q;
}

/* ------------------------------------------------------------------------ */
/* PCG with a fixed preconditioner H_S = R^T R (Section 1, eq. (PCG)):       */
/* r0 = b - H x0; H_S r^0 = r0; p0 = r^0; alpha_t = r_t^T r^_t / p_t^T H p_t; */
/* x += alpha p; r -= alpha H p; H_S r^_{t+1} = r_{t+1};                      */
/* p_{t+1} = r^_{t+1} + (r_{t+1}^T r^_{t+1} / r_t^T r^_t) p_t.                */
/* hist (may be NULL) gets delta_t if xstar != NULL, else r_t^T r^_t,         */
/* for t = 0..iters.                                                         */
/* ------------------------------------------------------------------------ */
int orc_pcg(const double* A, int64_t n, int64_t d, int64_t ld, const double* b, const double* R,
            double* x, double tol, int maxit, double rho_hat, const double* xstar, int* iters_out,
            double* hist) {
  double* r = (double*)malloc(sizeof(double) * (size_t)d);
  double* rh = (double*)malloc(sizeof(double) * (size_t)d);
  double* p = (double*)malloc(sizeof(double) * (size_t)d);
  double* v = (double*)malloc(sizeof(double) * (size_t)d);
  double* e1 = (double*)malloc(sizeof(double) * (size_t)d);
  double* e2 = (double*)malloc(sizeof(double) * (size_t)d);
  double q;
  orc_hmatvec(A, n, d, ld, x, v, &q);
  for (int64_t c = 0; c < d; ++c) r[c] = b[c] - v[c];
  orc_precond_solve(R, d, r, rh);
  for (int64_t c = 0; c < d; ++c) p[c] = rh[c];
  double rr = dot(r, rh, d);
  if (hist) hist[0] = xstar ? half_h_err2(A, n, d, ld, x, xstar, e1, e2) : rr;
  int status = ORC_ERR_MAXIT;
  int t = 0;
  if (rr == 0.0 || converged(rr, rho_hat, tol, dot(b, x, d))) status = ORC_OK;
  while (status == ORC_ERR_MAXIT && t < maxit) {
    orc_hmatvec(A, n, d, ld, p, v, &q);
    if (!(q > 0.0) || !isfinite(q)) { status = ORC_ERR_BREAKDOWN; break; }
    double alpha = rr / q;
    for (int64_t c = 0; c < d; ++c) { x[c] += alpha * p[c]; r[c] -= alpha * v[c]; }
    orc_precond_solve(R, d, r, rh);
    double rr_new = dot(r, rh, d);
    double beta = rr_new / rr;
    for (int64_t c = 0; c < d; ++c) p[c] = rh[c] + beta * p[c];
    rr = rr_new;
    ++t;
    if (hist) hist[t] = xstar ? half_h_err2(A, n, d, ld, x, xstar, e1, e2) : rr;
    if (rr == 0.0 || converged(rr, rho_hat, tol, dot(b, x, d))) status = ORC_OK;
  }
  *iters_out = t;
  free(r); free(rh); free(p); free(v); free(e1); free(e2);
  return status;
}

/* ------------------------------------------------------------------------ */
/* IHS and Polyak-IHS (Section 1, eqs. eqnihs, eqnpolyakihs):                 */
/*   x_{t+1} = x_t - mu H_{S_t}^{-1} grad f(x_t) + beta (x_t - x_{t-1}),      */
/* grad f(x) = H x - b, x_{-1} = x_0 (beta = 0 gives IHS).  With a fixed      */
/* sketch R_fixed != NULL; otherwise every iteration t draws sketch instance  */
/* t of the given type (0 Gaussian, 1 SRHT, 2 SJLT) and factors it by Gram +   */
/* Cholesky (refreshed embeddings, Section 4).  Convergence is tested on       */
/* g_t^T H_{S_t}^{-1} g_t before the update, with the rule above.              */
/* ------------------------------------------------------------------------ */
int orc_ihs(const double* A, int64_t n, int64_t d, int64_t ld, const double* b, const double* R_fixed,
            int sketch_type, int64_t m, int s, uint64_t seed, double mu, double beta, double* x,
            double tol, int maxit, double rho_hat, const double* xstar, int* iters_out, double* hist) {
  double* g = (double*)malloc(sizeof(double) * (size_t)d);
  double* gh = (double*)malloc(sizeof(double) * (size_t)d);
  double* xprev = (double*)malloc(sizeof(double) * (size_t)d);
  double* e1 = (double*)malloc(sizeof(double) * (size_t)d);
  double* e2 = (double*)malloc(sizeof(double) * (size_t)d);
  double* SA = R_fixed ? NULL : (double*)malloc(sizeof(double) * (size_t)(m * d));
  double* G = R_fixed ? NULL : (double*)malloc(sizeof(double) * (size_t)(d * d));
  double* Rt = R_fixed ? NULL : (double*)malloc(sizeof(double) * (size_t)(d * d));
  memcpy(xprev, x, sizeof(double) * (size_t)d);
  int status = ORC_ERR_MAXIT;
  int t = 0;
  if (hist) hist[0] = xstar ? half_h_err2(A, n, d, ld, x, xstar, e1, e2) : 0.0;
  for (t = 0; t < maxit; ++t) {
    const double* R = R_fixed;
    if (!R_fixed) {
      int st = ORC_OK;
      if (sketch_type == 0) orc_sketch_gauss(A, n, d, ld, m, seed, (uint32_t)t, SA);
      else if (sketch_type == 1) st = orc_sketch_srht(A, n, d, ld, m, seed, (uint32_t)t, SA);
      else st = orc_sketch_sjlt(A, n, d, ld, m, s, seed, (uint32_t)t, SA);
      if (st != ORC_OK) { status = st; break; }
      orc_gram(SA, m, d, G);
      if (orc_cholesky_upper(G, d, Rt) != 0) { status = ORC_ERR_RANK; break; }
      R = Rt;
    }
    double q;
    orc_hmatvec(A, n, d, ld, x, g, &q);
    for (int64_t c = 0; c < d; ++c) g[c] -= b[c];
    orc_precond_solve(R, d, g, gh);
    double gg = dot(g, gh, d);
    if (!isfinite(gg)) { status = ORC_ERR_BREAKDOWN; break; }
    if (gg == 0.0 || converged(gg, rho_hat, tol, dot(b, x, d))) { status = ORC_OK; break; }
    for (int64_t c = 0; c < d; ++c) {
      double xn = x[c] - mu * gh[c] + beta * (x[c] - xprev[c]);
      xprev[c] = x[c];
      x[c] = xn;
    }
    if (hist) hist[t + 1] = xstar ? half_h_err2(A, n, d, ld, x, xstar, e1, e2) : gg;
  }
  *iters_out = t;
  free(g); free(gh); free(xprev); free(e1); free(e2); free(SA); free(G); free(Rt);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Flexible CG with refreshed embeddings (Section 1, eqs. eqnconjugatedirections- */
/* refreshed (GCC) and eqnflexiblecg (FCG); Section 4): at iteration t, with a     */
/* fresh sketch S_t (instance t) and r_t = b - H x_t,                             */
/*   v_t = H_{S_t}^{-1} r_t,                                                      */
/*   p_t = v_t - sum_{j = t-k_t}^{t-1} <v_t, H p_j> / <p_j, H p_j> p_j,           */
/*   x_{t+1} = x_t + <p_t, r_t> / <p_t, H p_t> p_t,  r_{t+1} = r_t - alpha H p_t,   */
/* k_t = min(t, kmax); kmax < 0 keeps every earlier direction (GCC), kmax = 1 is  */
/* IPCG.  The step <p_t, r_t>/<p_t, H p_t> is the paper's <p_t, b>/<p_t, H p_t>   */
/* for x_0 = 0 and conjugate directions, written for any x_0.  Convergence is     */
/* tested on r_t^T v_t before the update, as for IHS.                            */
/* ------------------------------------------------------------------------ */
int orc_fcg(const double* A, int64_t n, int64_t d, int64_t ld, const double* b, int sketch_type, int64_t m, int s,
            uint64_t seed, int kmax, double* x, double tol, int maxit, double rho_hat, const double* xstar,
            int* iters_out, double* hist) {
  double* r = (double*)malloc(sizeof(double) * (size_t)d);
  double* v = (double*)malloc(sizeof(double) * (size_t)d);
  double* p = (double*)malloc(sizeof(double) * (size_t)d);
  double* Hp = (double*)malloc(sizeof(double) * (size_t)d);
  double* P = (double*)malloc(sizeof(double) * (size_t)(d * (maxit + 1)));
  double* HP = (double*)malloc(sizeof(double) * (size_t)(d * (maxit + 1)));
  double* qs = (double*)malloc(sizeof(double) * (size_t)(maxit + 1));
  double* SA = (double*)malloc(sizeof(double) * (size_t)(m * d));
  double* G = (double*)malloc(sizeof(double) * (size_t)(d * d));
  double* R = (double*)malloc(sizeof(double) * (size_t)(d * d));
  double* e1 = (double*)malloc(sizeof(double) * (size_t)d);
  double* e2 = (double*)malloc(sizeof(double) * (size_t)d);
  double q;
  orc_hmatvec(A, n, d, ld, x, v, &q);
  for (int64_t c = 0; c < d; ++c) r[c] = b[c] - v[c];
  if (hist) hist[0] = xstar ? half_h_err2(A, n, d, ld, x, xstar, e1, e2) : 0.0;
  int status = ORC_ERR_MAXIT, t = 0;
  for (t = 0; t < maxit; ++t) {
    int st = ORC_OK;
    if (sketch_type == 0) orc_sketch_gauss(A, n, d, ld, m, seed, (uint32_t)t, SA);
    else if (sketch_type == 1) st = orc_sketch_srht(A, n, d, ld, m, seed, (uint32_t)t, SA);
    else st = orc_sketch_sjlt(A, n, d, ld, m, s, seed, (uint32_t)t, SA);
    if (st != ORC_OK) { status = st; break; }
    orc_gram(SA, m, d, G);
    if (orc_cholesky_upper(G, d, R) != 0) { status = ORC_ERR_RANK; break; }
    orc_precond_solve(R, d, r, v);
    double rv = dot(r, v, d);
    if (!isfinite(rv)) { status = ORC_ERR_BREAKDOWN; break; }
    if (rv == 0.0 || converged(rv, rho_hat, tol, dot(b, x, d))) { status = ORC_OK; break; }
    int kt = (kmax < 0 || kmax > t) ? t : kmax;
    for (int64_t c = 0; c < d; ++c) p[c] = v[c];
    for (int j = t - kt; j < t; ++j) {
      double coef = dot(v, HP + (int64_t)j * d, d) / qs[j];
      for (int64_t c = 0; c < d; ++c) p[c] -= coef * P[(int64_t)j * d + c];
    }
    orc_hmatvec(A, n, d, ld, p, Hp, &q);
    if (!(q > 0.0) || !isfinite(q)) { status = ORC_ERR_BREAKDOWN; break; }
    double alpha = dot(p, r, d) / q;
    for (int64_t c = 0; c < d; ++c) { x[c] += alpha * p[c]; r[c] -= alpha * Hp[c]; }
    memcpy(P + (int64_t)t * d, p, sizeof(double) * (size_t)d);
    memcpy(HP + (int64_t)t * d, Hp, sizeof(double) * (size_t)d);
    qs[t] = q;
    if (hist) hist[t + 1] = xstar ? half_h_err2(A, n, d, ld, x, xstar, e1, e2) : rv;
  }
  *iters_out = t;
  free(r); free(v); free(p); free(Hp); free(P); free(HP); free(qs); free(SA); free(G); free(R); free(e1); free(e2);
  return status;
}

/* ------------------------------------------------------------------------ */
/* x* by its definition, H x* = b: Householder QR of A (so H = R_A^T R_A),     */
/* then iterative refinement with the residual b - A^T A x in double-double   */
/* until the correction is below 1e-17 of x (at most 10 steps).               */
/* ------------------------------------------------------------------------ */
int orc_solve_direct(const double* A, int64_t n, int64_t d, int64_t ld, const double* b, double* x) {
  double* Ac = (double*)malloc(sizeof(double) * (size_t)(n * d));
  for (int64_t i = 0; i < n; ++i) memcpy(Ac + i * d, A + i * ld, sizeof(double) * (size_t)d);
  double* RA = (double*)malloc(sizeof(double) * (size_t)(d * d));
  int st = orc_qr_r(Ac, n, d, RA);
  free(Ac);
  if (st != 0) { free(RA); return ORC_ERR_RANK; }
  orc_precond_solve(RA, d, b, x);
  double* r = (double*)malloc(sizeof(double) * (size_t)d);
  double* c = (double*)malloc(sizeof(double) * (size_t)d);
  for (int it = 0; it < 10; ++it) {
    orc_residual_dd(A, n, d, ld, b, x, r);
    orc_precond_solve(RA, d, r, c);
    double cmax = 0.0, xmax = 0.0;
    for (int64_t k = 0; k < d; ++k) {
      x[k] += c[k];
      cmax = fmax(cmax, fabs(c[k]));
      xmax = fmax(xmax, fabs(x[k]));
    }
    if (cmax <= 1e-17 * xmax) break;
  }
  free(RA); free(r); free(c);
  return ORC_OK;
}

/* x* for large problems: iterative refinement whose inner solver is the
   oracle's own PCG (pinned separately) with preconditioner R, and whose
   residual is the double-double residual above. */
int orc_solve_refined(const double* A, int64_t n, int64_t d, int64_t ld, const double* b, const double* R,
                      double rho_hat, double* x, int outer) {
  double* r = (double*)malloc(sizeof(double) * (size_t)d);
  double* c = (double*)malloc(sizeof(double) * (size_t)d);
  memset(x, 0, sizeof(double) * (size_t)d);
  int status = ORC_OK;
  for (int it = 0; it < outer; ++it) {
    orc_residual_dd(A, n, d, ld, b, x, r);
    memset(c, 0, sizeof(double) * (size_t)d);
    int iters;
    int st = orc_pcg(A, n, d, ld, r, R, c, 1e-15, 4 * (int)d + 50, rho_hat, NULL, &iters, NULL);
    if (st == ORC_ERR_BREAKDOWN) { status = st; break; }
    double cmax = 0.0, xmax = 0.0;
    for (int64_t k = 0; k < d; ++k) {
      x[k] += c[k];
      cmax = fmax(cmax, fabs(c[k]));
      xmax = fmax(xmax, fabs(x[k]));
    }
    if (cmax <= 1e-17 * xmax) break;
  }
  free(r); free(c);
  return status;
}

/* gradient of L(x*) with respect to A, x* = H^{-1} b, lam = H^{-1} dL/dx*:
   dL/dA = -(A x*) lam^T - (A lam) x*^T (implicit differentiation of H x* = b, H = A^T A) */
void orc_grad_a(const double* A, int64_t n, int64_t d, int64_t ld, const double* x, const double* lam, double* gA) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* a = A + i * ld;
    double u = 0.0, w = 0.0;
    for (int64_t c = 0; c < d; ++c) { u += a[c] * x[c]; w += a[c] * lam[c]; }
    for (int64_t c = 0; c < d; ++c) gA[i * d + c] = -(u * lam[c] + w * x[c]);
  }
}

/* relative H-norm error ||x - x*||_H / ||x*||_H = ||A e|| / ||A x*||, e = x - x* */
double orc_rel_h_err(const double* A, int64_t n, int64_t d, int64_t ld, const double* x, const double* xstar) {
  double* e = (double*)malloc(sizeof(double) * (size_t)d);
  double* v = (double*)malloc(sizeof(double) * (size_t)d);
  double qe, qs;
  for (int64_t c = 0; c < d; ++c) e[c] = x[c] - xstar[c];
  orc_hmatvec(A, n, d, ld, e, v, &qe);
  orc_hmatvec(A, n, d, ld, xstar, v, &qs);
  free(e); free(v);
  return sqrt(qe) / sqrt(qs);
}
