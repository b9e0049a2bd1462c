/*
 * lsq.h -- C ABI of the GB300 (sm_103a) library for randomized-preconditioned
 * least squares, after Lacotte & Pilanci, "Faster Least Squares Optimization"
 * (arXiv 1911.02675).
 *
 * Problem (Section 1, eq. eqnconvexquadratic):
 *     x* = argmin_x  1/2 <x, H x> - <b, x>,   H = A^T A,  A in R^{n x d}, n >= d, b in R^d.
 * Method: a random embedding S (m x n) gives H_S = (SA)^T (SA) = R^T R; PCG with the
 * fixed preconditioner H_S (Section 1, eq. (PCG)), or IHS / Polyak-IHS (Section 1,
 * eqs. eqnihs and eqnpolyakihs) with a fixed or refreshed embedding (Sections 3, 4).
 *
 * Conventions for every entry point:
 *   - All pointers marked "device" are CUDA device pointers on the context's device;
 *     the library never frees or retains them past the call.
 *   - Matrices are row-major.  A has n rows of d entries, consecutive rows ld >= d
 *     elements apart.  SA is m x d with stride d.  R and W are d x d with stride d.
 *   - Work is issued on the context's stream.  lsq_sketch and lsq_factor return once
 *     the work is enqueued (their status covers argument checks and launch errors);
 *     lsq_solve waits for its own work to finish so that it can fill `info`.
 *   - Errors are reported as status codes; no entry point aborts the process.
 *     Scratch memory is owned by the context (grown on demand, freed by lsq_destroy).
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11) with key = (seed lo, seed hi),
 *     counter = (index lo, index hi or draw, sketch instance t, stream tag); see the
 *     individual sketches below.  The same seed and t give bit-identical embeddings.
 */
#ifndef LSQ_H
#define LSQ_H

#include <stdint.h>

#if defined(__GNUC__)
#define LSQ_API __attribute__((visibility("default")))
#else
#define LSQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSQ_OK = 0,
  LSQ_ERR_ARG = 1,        /* invalid argument (sizes, types, alignment, m < d, s > m, ...) */
  LSQ_ERR_RANK = 2,       /* H_S not positive definite: a Cholesky pivot <= 0 (SA rank deficient) */
  LSQ_ERR_BREAKDOWN = 3,  /* p^T H p <= 0 or a non-finite value inside the iteration */
  LSQ_ERR_MAXIT = 4,      /* tolerance not met within maxit iterations; x holds the last iterate */
  LSQ_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up (the context stays usable) */
  LSQ_ERR_CUDA = 6,       /* a CUDA runtime call failed */
  LSQ_ERR_ALLOC = 7       /* device scratch allocation failed */
} lsq_status;

typedef enum { LSQ_F64 = 0, LSQ_F32 = 1 } lsq_dtype;

typedef enum {
  LSQ_SKETCH_GAUSS = 0, /* Section 2: iid N(0, 1/m) entries */
  LSQ_SKETCH_SRHT = 1,  /* Section 2: S = R H E (sampling, Hadamard, signs), zero padding */
  LSQ_SKETCH_SJLT = 2   /* Section 2: s entries +-1/sqrt(s) per column of S */
} lsq_sketch_type;

typedef enum {
  LSQ_PCG = 0,        /* Section 1, eq. (PCG); fixed embedding */
  LSQ_IHS = 1,        /* Section 1, eq. eqnihs */
  LSQ_POLYAK_IHS = 2, /* Section 1, eq. eqnpolyakihs */
  LSQ_FCG = 3         /* Section 1, eqs. eqnconjugatedirectionsrefreshed / eqnflexiblecg:
                         conjugate directions against the last fcg_k directions, a fresh
                         embedding per iteration (GCC: fcg_k < 0, IPCG: fcg_k = 1) */
} lsq_method;

/* Arithmetic used for the passes over A inside lsq_solve.
 *   LSQ_PREC_F64:   native FP64 for every operation (the plain FP64 method).
 *   LSQ_PREC_MIXED: passes over A in FP32 arithmetic; the recursive residual is
 *                   replaced by b - H x evaluated in double-FP32 arithmetic (about 45
 *                   significant bits per element, TwoProduct/TwoSum accumulation) after
 *                   every 10^5 drop of its norm, every `refresh_every` iterations and
 *                   before convergence is declared; x, r and the preconditioner stay
 *                   FP64.  Reaches the same tolerance as LSQ_PREC_F64. */
typedef enum { LSQ_PREC_F64 = 0, LSQ_PREC_MIXED = 1 } lsq_precision;

/* A dense matrix in device memory (row-major, stride ld elements). */
typedef struct {
  const void* data; /* device; 16-byte aligned for the fast paths (any alignment of the element works) */
  int64_t n;        /* rows, 1 <= n < 2^31 */
  int64_t d;        /* columns, 1 <= d <= 1024 */
  int64_t ld;       /* row stride in elements, ld >= d */
  int32_t dtype;    /* lsq_dtype */
} lsq_matrix;

typedef struct lsq_ctx lsq_ctx;

/* Creates a context on the current CUDA device that issues its work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Returns LSQ_ERR_CUDA if no
 * device is usable.  No device memory is allocated until the first call that needs it. */
LSQ_API lsq_status lsq_create(lsq_ctx** ctx, void* cuda_stream);

/* Waits for the context's stream and frees its scratch.  NULL is accepted. */
LSQ_API lsq_status lsq_destroy(lsq_ctx* ctx);

/* Replaces the stream of the context (the previous stream is not synchronised). */
LSQ_API lsq_status lsq_set_stream(lsq_ctx* ctx, void* cuda_stream);

/* Deferred checks.  on = 1: lsq_sketch and lsq_factor / lsq_factor_ex stop waiting for their
 * own work.  The statuses they would have waited for (a timed-out wait inside a sketch
 * kernel, LSQ_ERR_RANK from the Cholesky) are kept on the device, the first error of each
 * kind, and reported with the usual codes by the next call on the context that waits for its
 * stream: lsq_solve (a deferred error is returned in preference to the solve's own status,
 * whose results are then meaningless) or lsq_sync.  Host code queued meanwhile (the next
 * call's set-up) overlaps the device work.  on = 0 (the default) restores waiting; statuses
 * already deferred stay pending until the next waiting call.  LSQ_ERR_ARG for a NULL ctx. */
LSQ_API lsq_status lsq_set_deferred_checks(lsq_ctx* ctx, int32_t on);

/* Waits for the context's stream and reports (then clears) the first deferred error, else
 * LSQ_OK.  LSQ_ERR_ARG for a NULL ctx. */
LSQ_API lsq_status lsq_sync(lsq_ctx* ctx);

/* Arithmetic of lsq_sketch.
 *   LSQ_SKETCH_F64: FP64 (the +-1 weights of SRHT/SJLT are exact; agrees with an FP64
 *                   evaluation of S A to rounding).
 *   LSQ_SKETCH_F32: A rounded to FP32 on load, FP32 arithmetic, FP64 output.  A sketch
 *                   only has to be a subspace embedding; the preconditioner it yields is
 *                   as good, and the solve still reaches its tolerance against FP64 x*.
 *   LSQ_SKETCH_BF16: Gaussian: S is generated in FP32 from the same Philox words
 *                   (each uniform keeps the top 24 of its 53 bits), S and A are rounded to
 *                   BF16 and multiplied on the tensor cores (tcgen05) with FP32
 *                   accumulation; FP64 output.  SJLT: also on the tensor cores, with the
 *                   +-1 entries of S exact in BF16: each element of A is narrowed to FP32
 *                   (FP64 A: mantissa truncation, as the mixed solve narrows it) and rounded
 *                   to BF16 (nearest, ties to even), the products are exact, the sums FP32 in
 *                   a fixed order (the sketch repeats bit for bit) and the 1/sqrt(s) scale
 *                   FP64.  Relative error of SA ~ 1e-3.
 *                   Not for the SRHT (LSQ_ERR_ARG). */
typedef enum { LSQ_SKETCH_F64 = 0, LSQ_SKETCH_F32 = 1, LSQ_SKETCH_BF16 = 2 } lsq_sketch_precision;

typedef struct {
  uint32_t t;        /* sketch instance (Philox counter word 2): 0 for a fixed embedding,
                        the iteration index for refreshed embeddings */
  int32_t s;         /* SJLT nonzeros per column of S, 1..32 (default 8); ignored otherwise */
  int32_t precision; /* lsq_sketch_precision (default LSQ_SKETCH_F64) */
  float* a32;        /* optional, FP64 A only: device, caller-owned n x ld32 FP32 buffer that
                        receives the FP32 narrowing of A (mantissa truncation, clamped
                        exponent), the values the FP32 passes of a mixed solve compute with;
                        hand it to lsq_solve through lsq_solve_opts.a32 so that the solve need
                        not make its own copy.  The FP32 SRHT writes it while it streams A;
                        other sketches add one pass.  NULL (zero-initialised opts) = none. */
  int64_t ld32;      /* row stride of a32 in elements: >= d and a multiple of 4; a32 16-byte
                        aligned (else LSQ_ERR_ARG) */
  int64_t row0;      /* A holds rows [row0, row0 + n) of a larger matrix of n_total rows (a row
                        slab, as on one of several GPUs): SA is then that slab's share
                        S[:, row0 : row0 + n] A of the whole matrix's sketch, with the same S
                        (Philox counters take the global row index; the SRHT's signs, sampled
                        rows and zero padding are the whole matrix's), so that the shares of
                        the slabs sum to the sketch of the whole matrix (Section 2's S A is a sum
                        over the rows of A).  SRHT: row0 a multiple of 2048.  Default 0. */
  int64_t n_total;   /* rows of the whole matrix; <= 0 (default): n.  row0 + n <= n_total < 2^31
                        (else LSQ_ERR_ARG). */
} lsq_sketch_opts;

/* ---------------------------------------------------------------------------------
 * lsq_sketch: SA = S A for one draw of the embedding S (Section 2).
 *   A     : the data matrix (device).
 *   type  : lsq_sketch_type.
 *   m     : sketch size, 1 <= m <= 65536; SRHT also m <= N = 2^ceil(log2 n) and
 *           (FP64) m <= 16384; SJLT s <= m.
 *   seed  : Philox key.
 *   opts  : may be NULL (t = 0, s = 8, FP64).
 *   SA    : device, m x d FP64 output (row-major), caller-owned.
 * Scaling makes E[S^T S] = I_n for every type:
 *   Gaussian  S[j,i] = z(j,i)/sqrt(m), z from Box-Muller on Philox(i, j/2, t, 1)
 *             (even j: cosine branch, odd j: sine branch; 53-bit uniforms (k+1/2) 2^-53
 *             from the word pairs (w0,w1) and (w2,w3));
 *   SRHT      S = (1/sqrt(m)) P H E on the zero-padded N rows; E_ii = -1 iff bit 0 of
 *             Philox(i, 0, t, 2).w0 is set; P keeps the m rows with the smallest 64-bit
 *             key (Philox(i, 0, t, 3).w0 << 32 | .w1, ties by index) in ascending order;
 *             H is the +-1 Sylvester Hadamard matrix in natural order;
 *   SJLT      column i of S holds s distinct rows drawn by Lemire's bounded-integer
 *             method from the successive words of Philox(i, r, t, 4), r = 0, 1, ...,
 *             duplicates skipped; the k-th drawn row has sign -1 iff bit k of
 *             Philox(i, 0, t, 5).w0 is set; entries +-1/sqrt(s).
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_sketch(lsq_ctx* ctx, const lsq_matrix* A, int32_t type, int64_t m, uint64_t seed,
                      const lsq_sketch_opts* opts, double* SA);

/* lsq_upload_sketch: lsq_sketch of a matrix that is still in host memory, with the
 * host-to-device copy overlapped by the transform.
 *   host_A  : host, n x d elements of A->dtype, row stride host_ld >= d elements; page-locked
 *             memory lets the copies run asynchronously (pageable memory is copied in turn).
 *   A       : device destination (data, n, d, ld, dtype as lsq_sketch); it receives the host
 *             matrix and is then the A of the sketch.
 *   other arguments, results and status as lsq_sketch (deferred checks apply).
 * SRHT with the staged transform (n > 1024 rows, so that the zero-padded length holds whole
 * 2048-row blocks; 16-byte aligned rows; FP32 arithmetic): the rows are copied per row-block group on an internal stream, which first
 * waits for the work already queued on the context stream, and each group's transform starts
 * on the context stream as soon as its rows have landed (the SRHT sums per-group partials, so
 * the result is that of lsq_sketch).  The tensor-core Gaussian sketch (LSQ_SKETCH_BF16) works
 * the same way on its row chunks (up to 1 GiB of BF16 A each): chunk k + 1 is copied while
 * chunk k is packed and multiplied.  Any other case copies the whole matrix on the context
 * stream, then sketches.  The context stream waits for every copy, also when the call returns
 * an error, so later calls see all of A.  LSQ_ERR_ARG for a NULL ctx, host_A or A, or
 * host_ld < d. */
LSQ_API lsq_status lsq_upload_sketch(lsq_ctx* ctx, const void* host_A, int64_t host_ld, const lsq_matrix* A,
                                     int32_t type, int64_t m, uint64_t seed, const lsq_sketch_opts* opts, double* SA);

/* ---------------------------------------------------------------------------------
 * lsq_factor: the preconditioner factor of H_S = (SA)^T (SA) (Section 1, PCG
 * paragraph; Section 6, which allows either a QR of SA or a Cholesky factor of H_S).
 *   SA : device, m x d FP64 (row-major), m >= d.
 *   R  : device, d x d FP64 output: upper triangular, positive diagonal, R^T R = H_S
 *        (Gram in FP64, then Cholesky); the strict lower triangle is written as 0.
 *   W  : device, d x d FP64 output: W = R^{-1} (upper triangular), which lsq_solve
 *        uses to apply H_S^{-1} r = W (W^T r) as two parallel triangular products.
 * Status LSQ_ERR_RANK (after a synchronisation) if a pivot is not positive. This call
 * waits for its own work so that it can report the rank check, unless deferred checks are
 * on (lsq_set_deferred_checks), when the rank failure is reported by the next waiting call.
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_factor(lsq_ctx* ctx, const double* SA, int64_t m, int64_t d, double* R, double* W);

/* lsq_factor_qr: the preconditioner factor by Householder QR with column pivoting of SA
 * (Businger-Golub; Section 1, PCG paragraph, names pivoted QR as a way to factor H_S):
 * SA[:, perm] = Q R, so H_S = P R^T R P^T and H_S^{-1} = W W^T with W = P R^{-1}.  It works on
 * SA itself, so the factor's error grows with cond(SA) rather than cond(SA)^2 (the Gram route),
 * and it reveals the numerical rank.
 *   SA   : device, m x d FP64 (row-major), d <= m <= 65536, d <= 1024.
 *   tol  : rank threshold in [0, 1): the factorisation stops when the largest remaining column
 *          norm is at most tol times the first pivot's (0: only exact zeros).
 *   R    : device, d x d FP64 out: upper triangular, positive non-increasing diagonal, rows from
 *          the rank on zero.
 *   W    : device, d x d FP64 out (full rank only): W = P R^{-1}, row perm[i] of W is row i of
 *          R^{-1}; pass it to lsq_solve with lsq_solve_opts.w_dense = 1.
 *   perm : device, d int32 out: column perm[k] of SA is the k-th pivot.
 *   rank_out : host, may be NULL: the numerical rank.
 * Waits for its work.  LSQ_ERR_RANK if the rank is below d (R and perm are still written),
 * LSQ_ERR_TIMEOUT if a bounded wait gave up, LSQ_ERR_ARG for bad sizes or tol.  FP64 throughout. */
LSQ_API lsq_status lsq_factor_qr(lsq_ctx* ctx, const double* SA, int64_t m, int64_t d, double tol, double* R,
                                 double* W, int32_t* perm, int64_t* rank_out);

/* lsq_factor_ex: lsq_factor with the arithmetic of the Gram matrix chosen.
 *   gram_precision : LSQ_PREC_F64 (= lsq_factor) or LSQ_PREC_MIXED, which forms
 *                    H_S = (SA)^T (SA) in double-FP32 on the FP32 pipe: each entry of SA is
 *                    split into a 21-bit head and the FP32 rounding of the rest (about 45
 *                    significant bits), products are exact (TwoProduct by FMA) and sums are
 *                    (head, tail) pairs (TwoSum), a relative error near 1e-13 per entry,
 *                    far below what an FP32 sketch (LSQ_SKETCH_F32) already carries.  The
 *                    Cholesky factor and the inverse stay FP64.
 * Other arguments, results and status as lsq_factor; LSQ_ERR_ARG for another precision. */
LSQ_API lsq_status lsq_factor_ex(lsq_ctx* ctx, const double* SA, int64_t m, int64_t d, double* R, double* W,
                                 int32_t gram_precision);

/* Options of lsq_solve; lsq_solve_opts_default fills the defaults noted below. */
typedef struct {
  double rho;          /* deviation parameter rho in (0,1) of the event E_rho (Section 3);
                          default (<= 0): d/m for the fixed embedding, where m comes from
                          `m` below (required for IHS/Polyak defaults and the stopping rule) */
  double mu;           /* step size; default (NaN): IHS fixed (1-rho)^2/(1+rho), Polyak fixed
                          (1-rho)^2 (theorem theoremihsfixed); refreshed theta1/theta2
                          (theorem theoremexacterrorrefreshed, Gaussian moments of Section 2;
                          SRHT: Haar trace approximations rescaled to E[S^T S] = I) */
  double beta;         /* momentum; default (NaN): rho for fixed Polyak-IHS, 0.1 refreshed */
  int32_t refresh;     /* IHS / Polyak only: 1 = a fresh embedding every iteration */
  int32_t sketch_type; /* refreshed embeddings: lsq_sketch_type */
  int64_t m;           /* sketch size of the embedding behind W (fixed) or refreshed */
  uint64_t seed;       /* refreshed embeddings: Philox key (instance t = iteration index) */
  int32_t s;           /* refreshed SJLT: nonzeros per column (default 8) */
  int32_t precision;   /* lsq_precision (default LSQ_PREC_F64) */
  int32_t refresh_every; /* MIXED only: most iterations between exact residual replacements
                            (default 40; a replacement also follows every 10^5 drop of the
                            residual norm and every recursive convergence) */
  int32_t grid_blocks; /* 0 = automatic; else the number of resident CTAs of the solve kernel */
  int32_t x0_zero;     /* 1: x0 is zero, so the initial residual b - H x0 = b needs no pass over A */
  int32_t fcg_k;       /* LSQ_FCG: directions kept for orthogonalisation; < 0 (default) keeps
                          all of them (GCC), 1 gives IPCG, k gives FCG(k) */
  const float* a32;    /* optional: the FP32 narrowing of A (lsq_sketch_opts.a32), row stride
                          ld32; MIXED solves of FP64 A stream it instead of making a copy.  The
                          caller guarantees it holds the narrowing of this A.  NULL = none. */
  int64_t ld32;
  int32_t a32_copy;    /* MIXED PCG / IHS with FP64 A and maxit >= 3: 1 (default) makes an FP32
                          copy of A once per call (n x ceil32(d) x 4 bytes of device memory,
                          kept by the context for later calls) that the FP32 passes read
                          instead of A, halving their bytes; it holds the values those passes
                          compute with, so results are bit-identical with 0 (every pass
                          narrows A itself).  Where the memory cannot be had the solve runs as
                          with 0. */
  int32_t w_dense;     /* fixed-embedding PCG / IHS / Polyak: 1 = W is a general d x d matrix with
                          H_S^{-1} = W W^T (the pivoted-QR factor of lsq_factor_qr, W = P R^{-1}),
                          so the two products run over whole rows; 0 (default) = W upper
                          triangular (lsq_factor), whose zero halves are skipped */
} lsq_solve_opts;

/* Results of lsq_solve. */
typedef struct {
  int32_t iters;        /* iterations taken (passes of the loop; PCG: updates of x) */
  int32_t status;       /* same as the return value */
  int32_t passes;       /* passes over A, including the initial residual and replacements */
  int32_t exact_passes; /* of which passes in full precision (MIXED: the residual replacements) */
  double est_err;       /* final stopping quantity sqrt((1+sqrt(rho))^2 r^T H_S^-1 r / <b,x>) */
  double ms_total;      /* device time of the whole call (ms), CUDA events */
  double ms_sketch;     /* refreshed only: time in sketch + factor (ms) */
  int32_t a32_copy;     /* FP32 passes over an FP32 copy of A: 1 made by this call
                           (opts->a32_copy), 2 the caller's (opts->a32); 0 none */
  int32_t reserved;
} lsq_solve_info;

LSQ_API void lsq_solve_opts_default(lsq_solve_opts* opts);

/* ---------------------------------------------------------------------------------
 * lsq_solve: iterates from x0 to an approximation of x*.
 *   A      : the data matrix (device).
 *   b      : device, d FP64.
 *   method : lsq_method.
 *   W      : device, d x d FP64, W = R^{-1} from lsq_factor (fixed embedding); NULL
 *            with opts->refresh = 1 draws a new embedding every iteration (IHS, Polyak,
 *            FCG; the sketches of LSQ_FCG are FP32 under LSQ_PREC_MIXED, FP64 otherwise).
 *            LSQ_FCG takes every H p_t from a full-precision pass (FP64, or double-FP32
 *            under LSQ_PREC_MIXED) since its orthogonalisation uses the stored H p_j.
 *   x      : device, d FP64; in: x0, out: the last iterate.
 *   tol    : stop when (1+sqrt(rho))^2 r^T H_S^{-1} r <= tol^2 <b, x>, which bounds the
 *            relative H-norm error ||x - x*||_H / ||x*||_H by tol on the event E_rho
 *            (Section 3) since r^T H_S^{-1} r = Delta^T C_S^{-1} Delta; tol = 0 runs maxit.
 *   maxit  : iteration limit (>= 0).
 *   opts   : may be NULL (defaults); info: may be NULL.
 * Returns LSQ_OK, LSQ_ERR_MAXIT (x = last iterate), LSQ_ERR_BREAKDOWN, LSQ_ERR_RANK
 * (refreshed factor), LSQ_ERR_TIMEOUT, LSQ_ERR_ARG or LSQ_ERR_CUDA.
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_solve(lsq_ctx* ctx, const lsq_matrix* A, const double* b, int32_t method,
                     const double* W, double* x, double tol, int32_t maxit,
                     const lsq_solve_opts* opts, lsq_solve_info* info);

/* One fused pass over A: v = A^T (A p) and q = ||A p||^2 = p^T H p (the iteration cost
 * of Section 6), FP64 arithmetic.  p, v: device, d FP64; q: device, 1 FP64. */
LSQ_API lsq_status lsq_hmatvec(lsq_ctx* ctx, const lsq_matrix* A, const double* p, double* v, double* q);

/* ---------------------------------------------------------------------------------
 * lsq_grad_a: the gradient with respect to A of a loss L(x*), x* = H^{-1} b, given x*
 * and lambda = H^{-1} dL/dx* (a second lsq_solve with the forward's W):
 *     dL/dA = -(A x*) lambda^T - (A lambda) x*^T          (dL/db = lambda).
 * Derived from the problem statement of Section 1 (implicit differentiation of H x* = b).
 *   A      : the data matrix (device, FP64 or FP32).
 *   x, lam : device, d FP64.
 *   gA     : device, n x d output with row stride ldg >= d, same dtype as A, caller-owned.
 * One pass over A (u = A x*, w = A lambda per row in FP64) and one write of gA.
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_grad_a(lsq_ctx* ctx, const lsq_matrix* A, const double* x, const double* lam, void* gA,
                              int64_t ldg);

/* ---------------------------------------------------------------------------------
 * lsq_hmatvec_noalloc: the same fused pass as lsq_hmatvec (v = A^T (A p), q = ||A p||^2,
 * FP64 arithmetic) for callers that cannot allocate device memory -- code whose device
 * memory all belongs to its own pool allocator, or latency-bound loops that cannot take
 * the synchronisation an allocation may cause.  The paper has no counterpart: this is a
 * deployment variant of the pass, not a step of the method.
 *   A, p, v, q : as lsq_hmatvec (device; p, v: d FP64; q: 1 FP64), caller-owned.
 *   cuda_stream: the cudaStream_t to issue on (NULL = legacy default stream).
 * Needs no context and calls no allocator.  Its only scratch is a fixed array of
 * 160 x 1025 doubles (1.25 MiB) inside the library, present on every GPU that loads it
 * until the process exits; the number of CTAs is chosen so that the partial sums fit,
 * and d > 1024 (or any size that would not fit) is rejected with LSQ_ERR_ARG.
 * The first call on each device looks up the array's device address (with that device
 * current); make that first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (other streams, other host threads) race and give
 * wrong results, so serialise them.  Nothing in the array needs clearing between calls.
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_hmatvec_noalloc(const lsq_matrix* A, const double* p, double* v, double* q,
                                       void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * lsq_advise_sketch_size: host-only advisor of Section 6 (optimized sketch size).
 *   Gaussian (theorem theoremoptimalcomplexitygaussian):
 *       m* = d exp(W0((n/d^2) log(1/eps))),  cost ratio = 1 / log(n/d^2);
 *   SRHT (theorem theoremoptimalcomplexitysrht), for n > d^2:
 *       (i)  sqrt(log 1/eps) < log(n/d^2): m* = e^{sqrt(log 1/eps)} d log d,
 *            cost ratio = (log d + sqrt(log 1/eps)) / (log d + log 1/eps);
 *       (ii) otherwise: m* = (n/d) max(log d, log(1/eps)/log(n/d^2)),
 *            cost ratio = (log d + log(1/eps)/log(n/d^2)) / (log d + log 1/eps).
 * The cost ratios are the paper's flop models with constants dropped, against the
 * classical m = O(d) (Gaussian) or O(d log d) (SRHT).  predicted_iters is
 * ceil(log(4/eps) / log(m_star / m_delta)) with m_delta = d (Gaussian) or d log d (SRHT).
 * LSQ_ERR_ARG for n <= d^2, eps outside (0,1), or an SJLT (no result in the paper).
 * --------------------------------------------------------------------------------- */
typedef struct {
  double m_star;          /* optimized sketch size (real; round as needed) */
  double cost_ratio;      /* model cost at m* over the classical cost */
  double predicted_iters; /* PCG iterations predicted at m_star (-1 if m_star <= m_delta) */
  int32_t regime;         /* 0 Gaussian; 1, 2: SRHT cases (i), (ii) */
} lsq_advice;

LSQ_API lsq_status lsq_advise_sketch_size(int64_t n, int64_t d, double eps, int32_t sketch_type, lsq_advice* out);

/* ---------------------------------------------------------------------------------
 * Batched solves: many independent problems of uneven n, d and numbers of right-hand
 * sides, each solved by PCG with its own fixed embedding (Section 1, eq. (PCG), applied
 * per right-hand side; the iterations of all problems share one persistent launch).
 * --------------------------------------------------------------------------------- */
#define LSQ_MAX_RHS 16

typedef struct {
  lsq_matrix A;      /* n x d (device), d <= 512 */
  const double* B;   /* device, k right-hand sides of length d: entry c of b_j at B[j * d + c] */
  double* X;         /* device, same layout: in x0 (ignored when x0_zero), out the iterates */
  int32_t k;         /* right-hand sides, 1 .. LSQ_MAX_RHS */
  int32_t iters;     /* out: iterations until the last right-hand side of the problem stopped */
  int32_t status;    /* out: LSQ_OK, LSQ_ERR_MAXIT, LSQ_ERR_BREAKDOWN or LSQ_ERR_RANK */
  int32_t reserved;
} lsq_problem;

typedef struct {
  int32_t sketch_type;      /* default LSQ_SKETCH_SJLT */
  int32_t s;                /* SJLT nonzeros per column (default 8; at most m of a problem) */
  double m_factor;          /* sketch size m = ceil(m_factor * d) (default 4; m >= d enforced) */
  uint64_t seed;            /* problem p draws sketch instance t = p of this seed */
  int32_t sketch_precision; /* lsq_sketch_precision (default LSQ_SKETCH_F32) */
  int32_t precision;        /* lsq_precision (default LSQ_PREC_MIXED) */
  double rho;               /* stopping-rule deviation parameter; default (<= 0): d/m per problem */
  int32_t x0_zero;          /* 1 (default): every x0 is zero and X is overwritten */
  int32_t refresh_every;    /* MIXED: most iterations between exact residual replacements (40);
                               a replacement also follows a 10^5 drop of the residual norm and
                               every convergence of the recursive residual */
  int32_t chunk_rows;       /* rows of A per work unit of the pass (0: about 2^20 elements of A) */
  int32_t grid_blocks;      /* CTAs of the pass kernel (0: as many as are resident) */
  int32_t profile_phases;   /* 1: run the iterations without the CUDA graph and time each kernel
                               into lsq_batch_info.ms_phase (slower; for tuning) */
  int32_t autotune;         /* 1 (default): on the first batch of a shape (the n, d and k of every
                               problem) on a device, time one pass of the first iteration at each
                               candidate work-unit size (2^19, 2^20, 2^21 elements of A) and pass
                               grid (all resident CTAs, one per SM) that chunk_rows / grid_blocks
                               leave open, and keep the fastest for the process */
} lsq_batch_opts;

typedef struct {
  int32_t iters_max;     /* iterations of the slowest right-hand side */
  int32_t status;        /* LSQ_OK if every right-hand side converged, else the first error */
  int32_t passes;        /* passes of the persistent launch over the active problems */
  int32_t exact_passes;  /* of which exact (FP64 or double-FP32) residual passes */
  double ms_total;       /* device time of the call (ms) */
  double ms_sketch;      /* sketches of all problems */
  double ms_factor;      /* factorisations of all problems */
  double ms_solve;       /* the persistent PCG launch */
  double ms_phase[8];    /* with opts.profile_phases: time in the pass, update, W^T r, W t and
                            direction kernels of the iterations ([5..7] unused); else zero */
  int64_t pass_chunk_elems; /* the pass's work unit (elements of A per chunk) the iterations used */
  int32_t pass_grid;        /* CTAs of the pass kernel the iterations used */
  int32_t tuned;            /* 1 if this call ran the autotuner (first batch of its shape) */
} lsq_batch_info;

LSQ_API void lsq_batch_opts_default(lsq_batch_opts* opts);

/* lsq_solve_batched: for every problem p (host array `probs` of nprob entries, device data),
 * draws its sketch (instance t = p), factors it (Cholesky of the Gram matrix, W = R^{-1}),
 * then runs PCG on all right-hand sides of all problems in lockstep iterations: one launch of a
 * CUDA graph whose conditional WHILE node repeats the iteration's kernels until no problem is
 * active or maxit iterations have run (decided on the device); per iteration, one pass over A_p
 * per active problem yields A_p^T (A_p P) for all of its search directions at once, then the
 * vector updates and W W^T per right-hand side.
 * A right-hand side stops by rule (1+sqrt(rho))^2 r^T H_S^{-1} r <= tol^2 <b, x> (as in
 * lsq_solve); a problem stops when all of its right-hand sides have. Under LSQ_PREC_MIXED the
 * passes run in FP32-level arithmetic with exact (double-FP32) residual replacement as in
 * lsq_solve; when every A_p is FP32 with contiguous rows (ld = d) and a 16-byte aligned first
 * element, those passes run on the tensor cores as three TF32 products per element (a TF32 head
 * and the FP32 remainder of both operands, the remainders' product dropped: below 2^-22 of the
 * product), with FP32 sums; otherwise in FP32 on the SIMT pipes.
 * Returns LSQ_OK, LSQ_ERR_MAXIT, LSQ_ERR_BREAKDOWN, LSQ_ERR_RANK (see probs[p].status),
 * LSQ_ERR_TIMEOUT, LSQ_ERR_ARG or LSQ_ERR_CUDA. Synchronises before returning. */
LSQ_API lsq_status lsq_solve_batched(lsq_ctx* ctx, int32_t nprob, lsq_problem* probs, double tol, int32_t maxit,
                                     const lsq_batch_opts* opts, lsq_batch_info* info);

/* ---------------------------------------------------------------------------------
 * lsq_pcg_tail: the part of one PCG iteration (Section 1, eq. (PCG)) that follows the pass over
 * A, as a call of its own, for solves whose rows of A are split across GPUs.  H p is a sum over
 * the rows of A, so with A in row slabs A_k (one per GPU, lsq_sketch's row0 / n_total give the
 * matching sketch shares) each GPU computes v_k = A_k^T (A_k p) and q_k = ||A_k p||^2 with
 * lsq_hmatvec, the d + 1 numbers are summed across the GPUs (one all-reduce per iteration), and
 * every GPU calls lsq_pcg_tail on the same sums, so all of them keep the same iterate.
 *   d      : 1..1024.
 *   W      : device, d x d FP64, W = R^{-1} from lsq_factor of the (summed) sketch.
 *   b      : device, d FP64.
 *   vq     : device, d + 1 FP64: phase 0: H x0 in vq[0..d) (zeros for x0 = 0; vq[d] unused);
 *            phase 1: H p in vq[0..d) and p^T H p in vq[d], p the state's current direction.
 *   phase  : 0 starts (r = b - H x0, z = W W^T r, p = z), 1 takes one step
 *            (alpha = r^T z / p^T H p, x += alpha p, r -= alpha H p, z = W W^T r,
 *            beta = r^T z / previous r^T z, p = z + beta p).
 *   tol, rho : the stopping rule of lsq_solve, (1 + sqrt(rho))^2 r^T z <= tol^2 <b, x>.
 *   state  : device, 4 d + 8 FP64, caller-owned: x (holding x0 before phase 0), r, z, p, then
 *            r^T z, <b, x>, alpha, beta, flag (0 running, 1 converged, 2 failed), status, iterations.
 *            Once the flag is nonzero, phase 1 leaves the state unchanged.
 *   flag_out : NULL, or host int that receives the flag (the call then waits for its work).
 * Status LSQ_ERR_BREAKDOWN (with flag_out) when p^T H p <= 0 or a value is not finite;
 * LSQ_ERR_ARG for bad sizes, phase, tol or rho outside (0, 1).  FP64 throughout.
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_pcg_tail(lsq_ctx* ctx, int64_t d, const double* W, const double* b, const double* vq,
                                int32_t phase, double tol, double rho, double* state, int32_t* flag_out);

/* ---------------------------------------------------------------------------------
 * lsq_selftest_wait: a check of the library's failure detection, with no counterpart in the
 * paper.  Every cooperative kernel synchronises its CTAs with bounded grid barriers: a CTA
 * that waits longer than the limit gives up, records LSQ_ERR_TIMEOUT and returns, so a kernel
 * never spins forever and the context stays usable.  This call runs one cooperative launch
 * (one CTA per SM) of such a barrier -- kind 0: the arrival-count barrier of the solve
 * kernels, kind 1: the generation barrier of the factor kernels -- that waits for `missing`
 * arrivals more than the grid has (0 <= missing <= 1024).  missing = 0 returns LSQ_OK;
 * missing > 0 can never complete and returns LSQ_ERR_TIMEOUT once each waiter has given up
 * after wait_ns nanoseconds of %globaltimer (<= 0: the library's own 4 s limit; at most 4 s).
 * Waits for its own work.  LSQ_ERR_ARG for a NULL ctx or a bad kind, missing or wait_ns.
 * --------------------------------------------------------------------------------- */
LSQ_API lsq_status lsq_selftest_wait(lsq_ctx* ctx, int32_t kind, int32_t missing, int64_t wait_ns);

/* Human-readable name of a status code (static storage). */
LSQ_API const char* lsq_status_str(int32_t status);

/* Number of CUDA kernels this library has launched in the calling process so far
 * (host-side counter; lets a caller count the kernels inside a timed region). */
LSQ_API uint64_t lsq_launch_count(void);

/* Library version string (static storage). */
LSQ_API const char* lsq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LSQ_H */
