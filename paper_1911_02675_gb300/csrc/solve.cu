// solve.cu -- the iteration loop: PCG (Section 1, eq. (PCG)), IHS and Polyak-IHS
// (Section 1, eqs. eqnihs / eqnpolyakihs) with a fixed or refreshed embedding.
//
// One persistent cooperative kernel runs the whole loop.  Each iteration is
//   A pass   : v = A^T (A p) and q = ||A p||^2 in one read of every row of A
//              (CTA-private partials, no atomics)                         -- barrier
//   columns  : fixed-order reduction of the partials, x and r updates       -- barrier
//   W^T r    : z = W^T r, one warp per output                                -- barrier
//   W z      : r^ = W z and r^T r^ partials                                  -- barrier
//   tail     : every CTA forms rho, beta, p (kept whole in shared memory) and
//              the stopping decision from the same numbers in the same order.
// H_S^{-1} r = R^{-1} R^{-T} r is applied as W (W^T r) with W = R^{-1}, two parallel
// triangular products instead of two sequential triangular solves.
#include <algorithm>
#include <math.h>

#include "apass.cuh"
#include "common.cuh"

using namespace lsq_apass;

namespace {

struct SolveArgs {
  const void* A;
  int dtype;
  int64_t n;
  int d;
  int dp;  // d rounded up to 32 * EPL
  int64_t ld;
  int64_t rows_per_cta;
  const double* b;
  const double* W;   // d x d upper, stride d
  const double* WT;  // W^T (lower), stride d
  int w_dense;       // 1: W is a general d x d matrix (H_S^{-1} = W W^T), the products run over whole rows
  double* x;         // user x (in: x0, out)
  double* xprev;     // IHS/Polyak: x_{t-1} carried between single-step launches
  int method;
  double mu, beta;
  double tol2;       // tol^2 / (1 + sqrt(rho))^2
  double lam1;       // (1 + sqrt(rho))^2
  int maxit;
  int x0_zero;       // PCG: skip the initial pass when x0 = 0
  int first_step;    // IHS single-step launches: 1 when x_{-1} = x_0
  int force_exact;   // mixed IHS single-step launches: the gradient is already small, pass in FP64
  int refresh_every; // mixed PCG: longest run of FP32 passes between exact residual replacements
  double replace2;   // mixed PCG: replace when rho has dropped by this factor since the last one
  double exact2;     // mixed IHS: passes in FP64 once gamma <= exact2 * <b, x>
  double* part;      // [(dp + 1)][P] pass partials
  double* red;       // [4][P] scalar partials
  double* r;         // dp each
  double* z;
  double* rh;
  double* g;
  unsigned* bar;
  int* err;
  double* out;       // [0] iters, [1] status, [2] passes, [3] est_err, [4] exact passes
  const float* a32;  // COPY kernels: FP32 copy of A (row stride ld32) that the FP32 passes read
  int64_t ld32;
  int ring;          // FP32 rows, 256 < d <= 1024: the FP32 passes stage rows by bulk copies
};

// out[i] = sum_k M[i*d + k] vec_s[k] for k in [k_lo(i), k_hi(i)), one warp per output
__device__ __forceinline__ double warp_row_dot(const double* __restrict__ row, const double* vec_s, int k_lo, int k_hi) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = k_lo + lane; k < k_hi; k += 32) s = fma(__ldg(row + k), vec_s[k], s);
  return warp_sum(s);
}

struct SolveSmem {
  double* vec;   // dp: p (PCG) or x (IHS)
  double* vec2;  // dp: x_{t-1} (IHS) / r or z staging
  double* wred;  // LSQ_WARPS * dp
  double* qred;  // LSQ_WARPS
  double* scal;  // 8
};

// The FP32 copy of an FP64 A that the FP32 passes of a mixed solve stream (half the bytes of
// A): a warp per row, the narrowing of the passes themselves (narrow_f32), so a pass over the
// copy computes with exactly the values a pass over A would.
template <int EPL>
__global__ void __launch_bounds__(LSQ_THREADS) narrow_copy_kernel(const double* __restrict__ A, int64_t n, int d,
                                                                  int64_t ld, float* __restrict__ a32, int64_t ld32) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * LSQ_WARPS;
  for (int64_t i = (int64_t)blockIdx.x * LSQ_WARPS + (threadIdx.x >> 5); i < n; i += nw) {
    const double* a = A + i * ld;
    double v[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) v[k] = lane + 32 * k < d ? __ldcs(a + lane + 32 * k) : 0.0;
    float* o = a32 + i * ld32;
#pragma unroll
    for (int k = 0; k < EPL; ++k)
      if (lane + 32 * k < d) o[lane + 32 * k] = narrow_f32(v[k]);
  }
}

// MIXED = false: every pass in FP64 arithmetic.  MIXED = true: PCG's passes over A run in
// FP32 arithmetic and the recursive residual is replaced by an exact b - H x (FP64 pass) when
// it has dropped by `replace2` since the last replacement, after `refresh_every` iterations,
// and whenever it passes the stopping test (so convergence is always declared on an exact
// residual); IHS / Polyak-IHS compute the gradient in FP32 until it is small relative to
// <b, x> and in FP64 after that (their update has no recursive residual to correct).
template <typename TA, int EPL, bool MIXED, bool COPY = false>
__global__ void __launch_bounds__(LSQ_THREADS, (EPL <= 16 ? 2 : 1)) solve_kernel(SolveArgs a) {
  extern __shared__ __align__(16) double smem[];
  const int dp = a.dp, d = a.d;
  SolveSmem S;
  S.vec = smem;
  S.vec2 = S.vec + dp;
  S.wred = S.vec2 + dp;
  double* stage = S.wred + LSQ_WARPS * dp;  // dp: r or z staging for the triangular products
  S.qred = stage + dp;
  S.scal = S.qred + LSQ_WARPS;
  // FP32 rows at the widest d (256 < d <= 1024): the bulk-copy ring of the FP32 passes (after the
  // scalars, on a 128-byte boundary) and its mbarriers
  constexpr bool RING = MIXED && EPL >= 16 && (COPY || sizeof(TA) == 4);
  __shared__ __align__(8) uint64_t ring_bars[RING ? LSQ_WARPS * RING_NS : 1];
  float* ring = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(S.scal + 8) + 127) & ~static_cast<uintptr_t>(127));
  uint32_t ring_phase = 0;
  if constexpr (RING) {
    if (a.ring && threadIdx.x == 0) ring_init(ring_bars);
    __syncthreads();
  }
  // the staged exact pass (MIXED, FP64 A): x in wred[0, dp), one row slot per warp in
  // wred[dp, 8 dp) + stage
  double* slots = S.wred + dp;

  const int P = gridDim.x, cta = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = P * LSQ_WARPS;
  // the grid's warps take the columns of the vectors and the rows of W in turn, CTA-major
  // (column i on CTA i mod P), so their FP64 work and loads run on every SM
  const int cw = cta + P * warp;
  const int64_t r0 = (int64_t)cta * a.rows_per_cta;
  const int64_t r1 = min(a.n, r0 + a.rows_per_cta);
  const TA* A = reinterpret_cast<const TA*>(a.A);
  // grid barriers: a count that only grows (bar[2..3], zeroed before the launch)
  unsigned long long bar_target = 0;
  unsigned long long* bar_count = reinterpret_cast<unsigned long long*>(a.bar + 2);
  auto gsync = [&]() -> int { return grid_sync_count(bar_count, bar_target, P, a.err); };
  double* red_rho = a.red;
  double* red_bx = a.red + P;
  int passes = 0, exact_passes = 0;
  const bool pcg = a.method == LSQ_PCG;

  // ---- H_S^{-1} applied to the vector `src` (global, dp), result into `dst` (global);
  //      also returns (through red_rho) the CTA partial of src^T dst.
  auto precond = [&](const double* src, double* dst) -> int {
    for (int c = threadIdx.x; c < dp; c += blockDim.x) stage[c] = c < d ? src[c] : 0.0;
    __syncthreads();
    for (int i = cw; i < d; i += nw) {
      const double zi = warp_row_dot(a.WT + (int64_t)i * d, stage, 0, a.w_dense ? d : i + 1);
      if (lane == 0) a.z[i] = zi;
    }
    if (gsync()) return 1;
    for (int c = threadIdx.x; c < dp; c += blockDim.x) stage[c] = c < d ? a.z[c] : 0.0;
    __syncthreads();
    double part_rho = 0.0;
    for (int j = cw; j < d; j += nw) {
      const double v = warp_row_dot(a.W + (int64_t)j * d, stage, a.w_dense ? 0 : j, d);
      if (lane == 0) {
        dst[j] = v;
        part_rho += v * src[j];
      }
    }
    if (lane == 0) S.qred[warp] = part_rho;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < LSQ_WARPS; ++w) s += S.qred[w];
      red_rho[cta] = s;
    }
    return gsync();
  };

  // every CTA: the same fixed-order sums of the per-CTA scalars
  auto total = [&](const double* red) -> double {
    if (warp == 0) {
      const double s = warp_sum_strip(red, P);
      if (lane == 0) S.scal[7] = s;
    }
    __syncthreads();
    const double s = S.scal[7];
    __syncthreads();
    return s;
  };

  // the same sums for two strips at once (warps 0 and 1)
  auto total2 = [&](const double* red0, const double* red1, double& s0, double& s1) {
    if (warp < 2) {
      const double s = warp_sum_strip(warp == 0 ? red0 : red1, P);
      if (lane == 0) S.scal[6 + warp] = s;
    }
    __syncthreads();
    s0 = S.scal[6];
    s1 = S.scal[7];
    __syncthreads();
  };

  // partial of <b, x> over the columns this CTA owns, x read from `xsrc`
  auto bx_partial = [&](const double* xsrc) {
    double s = 0.0;
    for (int c = cw; c < d; c += nw)
      if (lane == 0) s += a.b[c] * xsrc[c];
    if (lane == 0) S.qred[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < LSQ_WARPS; ++w) t += S.qred[w];
      red_bx[cta] = t;
    }
    __syncthreads();
  };

  // a pass whose v is accurate to (nearly) FP64: native FP64, or double-FP32 in MIXED mode
  auto exact_pass = [&](const double* vec) {
    if constexpr (MIXED && sizeof(TA) == 8)
      fused_pass_df_staged<EPL>(reinterpret_cast<const double*>(A), a.ld, d, dp, r0, r1, vec, S.wred, S.qred, a.part,
                                P, cta, slots);
    else if (MIXED) fused_pass_df<TA, EPL>(A, a.ld, d, dp, r0, r1, vec, S.wred, S.qred, a.part, P, cta);
    else fused_pass<TA, EPL, (EPL <= 4)>(A, a.ld, d, dp, r0, r1, vec, S.wred, S.qred, a.part, P, cta);
  };

  // an FP32 pass: over the FP32 copy of A (COPY), else narrowing the rows of A as they arrive;
  // both compute with the same FP32 values
  auto f32_pass = [&](const double* vec) {
    if constexpr (RING) {
      if (a.ring) {
        if constexpr (COPY)
          fused_pass_f32_ring<EPL>(a.a32, a.ld32, d, dp, r0, r1, vec, S.wred, S.qred, a.part, P, cta, ring, dp,
                                   ring_bars, ring_phase, a.err);
        else
          fused_pass_f32_ring<EPL>(reinterpret_cast<const float*>(A), a.ld, d, dp, r0, r1, vec, S.wred, S.qred,
                                   a.part, P, cta, ring, dp, ring_bars, ring_phase, a.err);
        return;
      }
    }
    if constexpr (COPY) fused_pass_f32<float, EPL>(a.a32, a.ld32, d, dp, r0, r1, vec, S.wred, S.qred, a.part, P, cta);
    else fused_pass_f32<TA, EPL>(A, a.ld, d, dp, r0, r1, vec, S.wred, S.qred, a.part, P, cta);
  };

  int status = LSQ_ERR_MAXIT;
  int it = 0;
  double est = 0.0;

  if (pcg) {
    // r0 = b - H x0
    if (!a.x0_zero) {
      for (int c = threadIdx.x; c < dp; c += blockDim.x) S.vec[c] = c < d ? a.x[c] : 0.0;
      __syncthreads();
      exact_pass(S.vec);
      ++passes;
      ++exact_passes;
      if (gsync()) return;
    }
    for (int c = cw; c < d; c += nw) {
      const double v = a.x0_zero ? 0.0 : warp_sum_strip(a.part + (int64_t)c * P, P);
      if (lane == 0) a.r[c] = a.b[c] - v;
    }
    bx_partial(a.x);
    if (gsync()) return;
    if (precond(a.r, a.rh)) return;
    double rho, bx;
    total2(red_rho, red_bx, rho, bx);
    for (int c = threadIdx.x; c < dp; c += blockDim.x) S.vec[c] = c < d ? a.rh[c] : 0.0;
    __syncthreads();
    est = (bx > 0.0) ? sqrt(a.lam1 * rho / bx) : 0.0;
    if (rho == 0.0 || rho <= a.tol2 * bx) status = LSQ_OK;
    double rho_last = rho;  // rho at the last exact residual
    int it_last = 0;
    while (status == LSQ_ERR_MAXIT && it < a.maxit) {
      if (MIXED) {
        f32_pass(S.vec);
      } else {
        fused_pass<TA, EPL, (!MIXED && EPL <= 4)>(A, a.ld, d, dp, r0, r1, S.vec, S.wred, S.qred, a.part, P, cta);
        ++exact_passes;
      }
      ++passes;
      if (gsync()) return;
      // q (warp 0) and the first column of every warp are summed in one round of loads, with
      // the same per-strip order as warp_sum_strip; b, x and r of that column come with them
      double sq = 0.0, sv = 0.0, b0 = 0.0, x0 = 0.0, rr0 = 0.0;
      {
        const double* pq = a.part + (int64_t)dp * P;
        const double* pv = a.part + (int64_t)cw * P;
        const bool hasv = cw < d;
        if (hasv && lane == 0) {
          b0 = a.b[cw];
          x0 = a.x[cw];
          rr0 = a.r[cw];
        }
        for (int j = lane; j < P; j += 32) {
          if (warp == 0) sq += pq[j];
          if (hasv) sv += pv[j];
        }
        sq = warp_sum(sq);
        sv = warp_sum(sv);
      }
      if (warp == 0 && lane == 0) S.scal[0] = sq;
      __syncthreads();
      const double q = S.scal[0];
      if (!(q > 0.0) || !isfinite(q) || !isfinite(rho)) {
        status = LSQ_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rho / q;
      // x += alpha p, r -= alpha H p, and this CTA's partial of <b, x> (bx_partial's order)
      double bxp = 0.0;
      if (cw < d && lane == 0) {
        const double xn = x0 + alpha * S.vec[cw];
        a.x[cw] = xn;
        a.r[cw] = rr0 - alpha * sv;
        bxp += b0 * xn;
      }
      for (int c = cw + nw; c < d; c += nw) {  // more columns than warps in the grid
        const double v = warp_sum_strip(a.part + (int64_t)c * P, P);
        if (lane == 0) {
          const double xn = a.x[c] + alpha * S.vec[c];
          a.x[c] = xn;
          a.r[c] -= alpha * v;
          bxp += a.b[c] * xn;
        }
      }
      if (lane == 0) S.qred[warp] = bxp;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LSQ_WARPS; ++w) t += S.qred[w];
        red_bx[cta] = t;
      }
      if (gsync()) return;
      if (precond(a.r, a.rh)) return;
      double rho_new;
      total2(red_rho, red_bx, rho_new, bx);
      bool conv = rho_new == 0.0 || rho_new <= a.tol2 * bx;
      // a drop-triggered replacement within 10^2 (in norm) of the tolerance is left to the one
      // that confirms convergence a few iterations later -- unless the drop since the last
      // exact residual passes FP32's resolution (10^7 in norm), where the recursive residual
      // is rounding noise
      const bool near = rho_new <= 1e4 * a.tol2 * bx && rho_new >= 1e-14 * rho_last;
      bool replaced = false;
      if (MIXED && (conv || (!near && rho_new <= a.replace2 * rho_last) || it + 1 - it_last >= a.refresh_every)) {
        // replace the recursive residual by b - H x evaluated in FP64
        for (int c = threadIdx.x; c < dp; c += blockDim.x) S.vec2[c] = c < d ? a.x[c] : 0.0;
        __syncthreads();
        exact_pass(S.vec2);
        ++passes;
        ++exact_passes;
        if (gsync()) return;
        for (int c = cw; c < d; c += nw) {
          const double v = warp_sum_strip(a.part + (int64_t)c * P, P);
          if (lane == 0) a.r[c] = a.b[c] - v;
        }
        if (gsync()) return;
        if (precond(a.r, a.rh)) return;
        rho_new = total(red_rho);
        conv = rho_new == 0.0 || rho_new <= a.tol2 * bx;
        rho_last = rho_new;
        it_last = it + 1;
        replaced = true;
      }
      // after an exact residual more than twice (in norm) the recursive one of the previous
      // iteration, the old direction is not trusted: restart from the preconditioned residual
      const double beta = (replaced && rho_new > 4.0 * rho) ? 0.0 : rho_new / rho;
      for (int c = threadIdx.x; c < dp; c += blockDim.x) S.vec[c] = c < d ? a.rh[c] + beta * S.vec[c] : 0.0;
      __syncthreads();
      rho = rho_new;
      ++it;
      est = (bx > 0.0) ? sqrt(a.lam1 * rho / bx) : 0.0;
      if (!isfinite(rho)) status = LSQ_ERR_BREAKDOWN;
      else if (conv) status = LSQ_OK;
    }
  } else {
    // IHS / Polyak-IHS: x and x_{t-1} whole in every CTA
    for (int c = threadIdx.x; c < dp; c += blockDim.x) {
      const double xc = c < d ? a.x[c] : 0.0;
      S.vec[c] = xc;
      S.vec2[c] = a.first_step ? xc : (c < d ? a.xprev[c] : 0.0);
    }
    __syncthreads();
    bool exact = !MIXED || a.force_exact;
    while (it < a.maxit) {
      if (exact) {
        exact_pass(S.vec);
        ++exact_passes;
      } else {
        f32_pass(S.vec);
      }
      ++passes;
      if (gsync()) return;
      for (int c = cw; c < d; c += nw) {
        const double v = warp_sum_strip(a.part + (int64_t)c * P, P);
        if (lane == 0) a.g[c] = v - a.b[c];
      }
      bx_partial(S.vec);
      if (gsync()) return;
      if (precond(a.g, a.rh)) return;
      const double gam = total(red_rho);
      const double bx = total(red_bx);
      est = (bx > 0.0) ? sqrt(a.lam1 * gam / bx) : 0.0;
      if (!isfinite(gam)) { status = LSQ_ERR_BREAKDOWN; break; }
      if (gam == 0.0 || gam <= a.tol2 * bx) {
        if (exact) { status = LSQ_OK; break; }
        exact = true;  // confirm on an FP64 gradient before stopping
        continue;
      }
      if (!exact && gam <= a.exact2 * bx) exact = true;
      for (int c = threadIdx.x; c < dp; c += blockDim.x) {
        const double xc = S.vec[c];
        const double xn = c < d ? xc - a.mu * a.rh[c] + a.beta * (xc - S.vec2[c]) : 0.0;
        S.vec2[c] = xc;
        S.vec[c] = xn;
      }
      __syncthreads();
      ++it;
    }
    if (cta == 0) {
      for (int c = threadIdx.x; c < d; c += blockDim.x) {
        a.x[c] = S.vec[c];
        a.xprev[c] = S.vec2[c];
      }
    }
  }
  if (cta == 0 && threadIdx.x == 0) {
    a.out[0] = (double)it;
    a.out[1] = (double)status;
    a.out[2] = (double)passes;
    a.out[3] = est;
    a.out[4] = (double)exact_passes;
  }
}

__global__ void transpose_kernel(const double* __restrict__ W, int d, double* __restrict__ WT) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = by + k, c = bx + threadIdx.x;
    tile[k][threadIdx.x] = (r < d && c < d) ? W[(int64_t)r * d + c] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = bx + k, c = by + threadIdx.x;
    if (r < d && c < d) WT[(int64_t)r * d + c] = tile[threadIdx.x][k];
  }
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
typedef void (*solve_fn)(SolveArgs);

template <typename TA, bool MIXED, bool COPY = false>
static void* pick_solve(int epl) {
  switch (epl) {
    case 1: return (void*)solve_kernel<TA, 1, MIXED, COPY>;
    case 2: return (void*)solve_kernel<TA, 2, MIXED, COPY>;
    case 4: return (void*)solve_kernel<TA, 4, MIXED, COPY>;
    case 8: return (void*)solve_kernel<TA, 8, MIXED, COPY>;
    case 16: return (void*)solve_kernel<TA, 16, MIXED, COPY>;
    default: return (void*)solve_kernel<TA, 32, MIXED, COPY>;
  }
}

static void* pick_narrow(int epl) {
  switch (epl) {
    case 1: return (void*)narrow_copy_kernel<1>;
    case 2: return (void*)narrow_copy_kernel<2>;
    case 4: return (void*)narrow_copy_kernel<4>;
    case 8: return (void*)narrow_copy_kernel<8>;
    case 16: return (void*)narrow_copy_kernel<16>;
    default: return (void*)narrow_copy_kernel<32>;
  }
}

static lsq_status check_matrix(const lsq_matrix* A) {
  if (!A || !A->data) return LSQ_ERR_ARG;
  if (A->n < 1 || A->n >= (1ll << 31) || A->d < 1 || A->d > LSQ_MAX_D || A->ld < A->d) return LSQ_ERR_ARG;
  if (A->dtype != LSQ_F64 && A->dtype != LSQ_F32) return LSQ_ERR_ARG;
  const size_t es = A->dtype == LSQ_F64 ? 8 : 4;
  if (((uintptr_t)A->data) % es) return LSQ_ERR_ARG;
  return LSQ_OK;
}

// vec, vec2, wred, stage, qred, scal
static size_t solve_smem_bytes(int dp) { return (size_t)(dp * 2 + LSQ_WARPS * dp + dp + LSQ_WARPS + 8) * 8; }

static double theta_ratio(int type, double m, double d, double N) {
  // mu = theta1 / theta2 for refreshed embeddings
  if (type == LSQ_SKETCH_SRHT) {
    const double t1 = (N - d) / (m - d) * (m / N);
    const double t2 = (N - d) / ((m - d) * (m - d) * (m - d)) * (d * d + m * N - 2 * d * m) * (m / N) * (m / N);
    return t1 / t2;
  }
  const double t1 = m / (m - d - 1);
  const double t2 = m * m * (m - 1) / ((m - d) * (m - d - 1) * (m - d - 3));
  return t1 / t2;
}

}  // namespace

extern "C" void lsq_solve_opts_default(lsq_solve_opts* o) {
  if (!o) return;
  o->rho = 0.0;
  o->mu = NAN;
  o->beta = NAN;
  o->refresh = 0;
  o->sketch_type = LSQ_SKETCH_GAUSS;
  o->m = 0;
  o->seed = 0;
  o->s = 8;
  o->precision = LSQ_PREC_F64;
  o->refresh_every = 40;
  o->grid_blocks = 0;
  o->x0_zero = 0;
  o->fcg_k = -1;
  o->a32 = nullptr;
  o->ld32 = 0;
  o->a32_copy = 1;
  o->w_dense = 0;
}

lsq_status lsq_narrow_copy(lsq_ctx* ctx, const lsq_matrix* A, float* a32, int64_t ld32) {
  const int d = (int)A->d, epl = epl_for(d);
  void* nk = pick_narrow(epl);
  const void* Ad = A->data;
  int64_t n = A->n, ld = A->ld, l32 = ld32;
  int di = d;
  void* nargs[] = {(void*)&Ad, &n, &di, &ld, (void*)&a32, &l32};
  const int nblk = (int)std::min<int64_t>((A->n + LSQ_WARPS - 1) / LSQ_WARPS, 8 * (int64_t)ctx->sm_count);
  LSQ_CUDA_TRY(cudaLaunchKernel(nk, dim3(nblk), dim3(LSQ_THREADS), nargs, 0, ctx->stream));
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

extern "C" lsq_status lsq_hmatvec(lsq_ctx* ctx, const lsq_matrix* A, const double* p, double* v, double* q) {
  if (!ctx || !p || !v || !q) return LSQ_ERR_ARG;
  lsq_status st = check_matrix(A);
  if (st != LSQ_OK) return st;
  const int d = (int)A->d, epl = epl_for(d), dp = 32 * epl;
  void* kern = A->dtype == LSQ_F64 ? pick_hmv<double>(epl) : pick_hmv<float>(epl);
  const size_t smem = hmatvec_smem_bytes(dp);
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LSQ_THREADS, smem));
  int P = std::max(1, per_sm) * ctx->sm_count;
  P = (int)std::min<int64_t>(P, (A->n + 31) / 32);
  P = std::max(P, 1);
  const int64_t rows_per_cta = (A->n + P - 1) / P;
  P = (int)((A->n + rows_per_cta - 1) / rows_per_cta);
  st = lsq_ensure_scratch(ctx, lsq_align256((size_t)(dp + 1) * P * 8));
  if (st != LSQ_OK) return st;
  double* part = reinterpret_cast<double*>(ctx->scratch);
  const void* Ad = A->data;
  int64_t n = A->n, ld = A->ld;
  int di = d, dpi = dp;
  void* args[] = {(void*)&Ad, &n, &di, &dpi, &ld, (void*)&rows_per_cta, (void*)&p, &part};
  LSQ_CUDA_TRY(cudaLaunchKernel(kern, dim3(P), dim3(LSQ_THREADS), args, smem, ctx->stream));
  lsq_count_launch();
  reduce_part_kernel<<<std::max(1, (d + 1 + 7) / 8), 256, 0, ctx->stream>>>(part, P, d, dp, v, q);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

extern "C" lsq_status lsq_solve(lsq_ctx* ctx, const lsq_matrix* A, const double* b, int32_t method, const double* W,
                                double* x, double tol, int32_t maxit, const lsq_solve_opts* opts_in,
                                lsq_solve_info* info) {
  if (!ctx || !b || !x) return LSQ_ERR_ARG;
  lsq_status st = check_matrix(A);
  if (st != LSQ_OK) return st;
  if (method != LSQ_PCG && method != LSQ_IHS && method != LSQ_POLYAK_IHS && method != LSQ_FCG) return LSQ_ERR_ARG;
  if (!(tol >= 0.0) || maxit < 0) return LSQ_ERR_ARG;
  lsq_solve_opts o;
  lsq_solve_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (o.precision != LSQ_PREC_F64 && o.precision != LSQ_PREC_MIXED) return LSQ_ERR_ARG;
  const bool mixed = o.precision == LSQ_PREC_MIXED;
  const int d = (int)A->d;
  const bool refresh = (method != LSQ_PCG) && o.refresh;
  if (!refresh && !W) return LSQ_ERR_ARG;
  if (refresh && (o.m < d || o.m > 65536)) return LSQ_ERR_ARG;
  double rho = o.rho;
  if (!(rho > 0.0)) {
    if (o.m <= 0) return LSQ_ERR_ARG;
    rho = (double)d / (double)o.m;
  }
  if (!(rho < 1.0)) return LSQ_ERR_ARG;
  const double lam1 = (1.0 + sqrt(rho)) * (1.0 + sqrt(rho));
  if (method == LSQ_FCG) {
    const lsq_status fst = lsq_fcg_solve(ctx, A, b, refresh ? nullptr : W, x, tol, maxit, o, lam1, info);
    if (ctx->pending) {  // a deferred sketch or factor error outranks the solve's status
      if (lsq_pending_enqueue(ctx) != LSQ_OK) return LSQ_ERR_CUDA;
      LSQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      const lsq_status deferred = lsq_pending_take(ctx);
      if (deferred != LSQ_OK) return deferred;
    }
    return fst;
  }
  double mu = o.mu, beta = o.beta;
  if (method == LSQ_PCG) {
    mu = 0.0;
    beta = 0.0;
  } else if (!refresh) {
    if (isnan(mu)) mu = method == LSQ_IHS ? (1 - rho) * (1 - rho) / (1 + rho) : (1 - rho) * (1 - rho);
    if (isnan(beta)) beta = method == LSQ_IHS ? 0.0 : rho;
  } else {
    if (isnan(mu)) {
      int64_t N = 1;
      while (N < A->n) N <<= 1;
      if (o.sketch_type != LSQ_SKETCH_SRHT && o.m < d + 4) return LSQ_ERR_ARG;
      mu = theta_ratio(o.sketch_type, (double)o.m, (double)d, (double)N);
    }
    if (isnan(beta)) beta = method == LSQ_IHS ? 0.0 : 0.1;
  }
  if (method == LSQ_IHS) beta = 0.0;

  const int epl = epl_for(d), dp = 32 * epl;
  // MIXED with FP64 A: the FP32 passes stream an FP32 copy of A (half the bytes), made once per
  // call; without the memory for it every pass narrows A itself (the same values)
  float* a32 = nullptr;
  int64_t ld32 = (d + 31) & ~31;
  const bool user_a32 = o.a32 != nullptr && mixed && A->dtype == LSQ_F64;
  if (user_a32) {
    if (o.ld32 < d || o.ld32 % 4 != 0 || ((uintptr_t)o.a32 % 16) != 0) return LSQ_ERR_ARG;
    a32 = const_cast<float*>(o.a32);
    ld32 = o.ld32;
  } else if (mixed && A->dtype == LSQ_F64 && o.a32_copy && maxit >= 3) {
    if (lsq_ensure_a32(ctx, (size_t)A->n * (size_t)ld32 * 4) == LSQ_OK) a32 = reinterpret_cast<float*>(ctx->a32);
  }
  void* kern = A->dtype == LSQ_F64
                   ? (mixed ? (a32 ? pick_solve<double, true, true>(epl) : pick_solve<double, true>(epl))
                            : pick_solve<double, false>(epl))
                   : (mixed ? pick_solve<float, true>(epl) : pick_solve<float, false>(epl));
  // the FP32 passes of the widest rows stage them by bulk copies (16-byte aligned rows whose
  // length is a multiple of 16 bytes)
  const bool f32_rows = mixed && (a32 != nullptr || A->dtype == LSQ_F32);
  const float* rows32 = a32 ? a32 : reinterpret_cast<const float*>(A->data);
  const int64_t ld_rows = a32 ? ld32 : A->ld;
  const bool ring = f32_rows && epl >= 16 && d % 4 == 0 && ((uintptr_t)rows32 % 16) == 0 && (ld_rows * 4) % 16 == 0;
  const size_t smem = solve_smem_bytes(dp) + (ring ? 128 + (size_t)LSQ_WARPS * lsq_apass::RING_NS * dp * 4 : 0);
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LSQ_THREADS, smem));
  if (per_sm < 1) return LSQ_ERR_CUDA;
  int P = per_sm * ctx->sm_count;
  if (o.grid_blocks > 0) P = std::min(P, o.grid_blocks);
  P = (int)std::min<int64_t>(P, std::max<int64_t>(1, (A->n + 31) / 32));
  const int64_t rows_per_cta = (A->n + P - 1) / P;
  P = (int)((A->n + rows_per_cta - 1) / rows_per_cta);

  // scratch: part, red, r, z, rh, g, xprev, WT, bar, out, + (refresh) SA, R, W
  const size_t mat = (size_t)d * d;
  size_t need = lsq_align256((size_t)(dp + 1) * P * 8) + lsq_align256((size_t)4 * P * 8) + 5 * lsq_align256((size_t)dp * 8) +
                lsq_align256(mat * 8) + lsq_align256(64) + lsq_align256(64);
  size_t refresh_extra = 0;
  if (refresh) refresh_extra = lsq_align256((size_t)o.m * d * 8) + 3 * lsq_align256(mat * 8);
  st = lsq_ensure_state(ctx, need + refresh_extra);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->state), 0};
  SolveArgs a;
  a.w_dense = 0;
  a.part = cv.take<double>((size_t)(dp + 1) * P);
  a.red = cv.take<double>((size_t)4 * P);
  a.r = cv.take<double>(dp);
  a.z = cv.take<double>(dp);
  a.rh = cv.take<double>(dp);
  a.g = cv.take<double>(dp);
  a.xprev = cv.take<double>(dp);
  double* WT = cv.take<double>(mat);
  a.bar = cv.take<unsigned>(16);
  a.err = reinterpret_cast<int*>(a.bar + 8);
  a.out = cv.take<double>(8);
  double* SA = refresh ? cv.take<double>((size_t)o.m * d) : nullptr;
  double* Rr = refresh ? cv.take<double>(mat) : nullptr;
  double* Wr = refresh ? cv.take<double>(mat) : nullptr;

  a.A = A->data;
  a.dtype = A->dtype;
  a.n = A->n;
  a.d = d;
  a.dp = dp;
  a.ld = A->ld;
  a.rows_per_cta = rows_per_cta;
  a.b = b;
  a.x = x;
  a.method = method;
  a.mu = mu;
  a.beta = beta;
  a.lam1 = lam1;
  a.tol2 = tol * tol / lam1;
  a.maxit = maxit;
  a.x0_zero = o.x0_zero ? 1 : 0;
  a.first_step = 1;
  a.force_exact = 0;
  a.refresh_every = o.refresh_every > 0 ? o.refresh_every : 40;
  a.a32 = a32;
  a.ld32 = ld32;
  a.ring = ring ? 1 : 0;
  // replace after a 10^5 drop of the residual norm: the FP32 passes' drift after it (about 1e-6
  // of that level) stays near 1e-11 of the initial residual, and convergence is confirmed on an
  // exact residual in any case
  a.replace2 = 1e-10;
  a.exact2 = 1e-8;    // IHS: FP64 gradients once the relative gradient is below 10^-4
  cudaStream_t s = ctx->stream;
  LSQ_CUDA_TRY(cudaEventRecord(ctx->ev0, s));
  if (a32 && !user_a32) {
    st = lsq_narrow_copy(ctx, A, a32, ld32);
    if (st != LSQ_OK) return st;
  }

  double ms_sketch = 0.0;
  int iters = 0, passes = 0, exact_passes = 0, status = LSQ_ERR_MAXIT;
  double est = 0.0;
  if (!refresh) {
    a.W = W;
    a.WT = WT;
    a.w_dense = o.w_dense ? 1 : 0;
    transpose_kernel<<<dim3((d + 31) / 32, (d + 31) / 32), dim3(32, 8), 0, s>>>(W, d, WT);
    LSQ_LAUNCH_CHECK();
    LSQ_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, s));
    void* args[] = {&a};
    LSQ_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(P), dim3(LSQ_THREADS), args, smem, s));
    lsq_count_launch();
    LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status, a.out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 12, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaEventRecord(ctx->ev1, s));
    if (lsq_pending_enqueue(ctx) != LSQ_OK) return LSQ_ERR_CUDA;
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    const double* o4 = reinterpret_cast<const double*>(ctx->host_status);
    const int errc = ctx->host_status[12];
    iters = (int)o4[0];
    status = errc ? errc : (int)o4[1];
    passes = (int)o4[2];
    est = o4[3];
    exact_passes = (int)o4[4];
  } else {
    a.W = Wr;
    a.WT = WT;
    a.maxit = 1;
    cudaEvent_t e_a, e_b;
    LSQ_CUDA_TRY(cudaEventCreate(&e_a));
    LSQ_CUDA_TRY(cudaEventCreate(&e_b));
    lsq_sketch_opts so = {};
    so.s = o.s > 0 ? o.s : 8;
    so.precision = LSQ_SKETCH_F64;
    so.a32 = nullptr;
    so.ld32 = 0;
    for (int t = 0; t <= maxit; ++t) {
      if (t == maxit) {
        status = LSQ_ERR_MAXIT;
        break;
      }
      so.t = (uint32_t)t;
      cudaEventRecord(e_a, s);
      st = lsq_sketch(ctx, A, o.sketch_type, o.m, o.seed, &so, SA);
      if (st == LSQ_OK) st = lsq_factor(ctx, SA, o.m, d, Rr, Wr);
      cudaEventRecord(e_b, s);
      if (st != LSQ_OK) {
        status = st;
        break;
      }
      transpose_kernel<<<dim3((d + 31) / 32, (d + 31) / 32), dim3(32, 8), 0, s>>>(Wr, d, WT);
      LSQ_LAUNCH_CHECK();
      a.first_step = t == 0;
      a.force_exact = (t > 0 && est * est <= a.exact2 * a.lam1) ? 1 : 0;
      LSQ_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, s));
      void* args[] = {&a};
      LSQ_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(P), dim3(LSQ_THREADS), args, smem, s));
      lsq_count_launch();
      LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status, a.out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
      LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 12, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
      LSQ_CUDA_TRY(cudaStreamSynchronize(s));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e_a, e_b);
      ms_sketch += ms;
      const double* o4 = reinterpret_cast<const double*>(ctx->host_status);
      const int errc = ctx->host_status[12];
      passes += (int)o4[2];
      exact_passes += (int)o4[4];
      est = o4[3];
      const int stt = errc ? errc : (int)o4[1];
      iters = t + (int)o4[0];
      if (stt == LSQ_ERR_MAXIT) continue;  // the one step was taken
      status = stt;
      break;
    }
    cudaEventRecord(ctx->ev1, s);
    if (lsq_pending_enqueue(ctx) != LSQ_OK) return LSQ_ERR_CUDA;
    cudaStreamSynchronize(s);
    cudaEventDestroy(e_a);
    cudaEventDestroy(e_b);
  }
  float ms_total = 0.f;
  cudaEventElapsedTime(&ms_total, ctx->ev0, ctx->ev1);
  (void)cudaGetLastError();
  if (info) {
    info->iters = iters;
    info->status = status;
    info->passes = passes;
    info->exact_passes = exact_passes;
    info->est_err = est;
    info->ms_total = ms_total;
    info->ms_sketch = ms_sketch;
    info->a32_copy = a32 ? (user_a32 ? 2 : 1) : 0;
    info->reserved = 0;
  }
  // a deferred sketch or factor error (lsq_set_deferred_checks) outranks the solve's status
  const lsq_status deferred = lsq_pending_take(ctx);
  if (deferred != LSQ_OK) return deferred;
  return (lsq_status)status;
}
