// batch.cu -- many independent least-squares problems of uneven n, d and numbers of
// right-hand sides k, each solved by PCG (Section 1, eq. (PCG)) per right-hand side with
// the problem's own fixed embedding; the iterations of every problem run in one persistent
// cooperative launch.
//
// Per iteration (all problems in lockstep, converged right-hand sides masked out):
//   pass      one read of every active A_p, in chunks of rows scheduled over the CTAs, gives
//             V = A_p^T (A_p P_p) and q_j = ||A_p p_j||^2 for all k_p directions at once: a tile
//             of 32 rows is staged in shared memory, Y = A_tile P (rows x k) and then
//             V += A_tile^T Y (register tiles), FP32 under LSQ_PREC_MIXED, FP64 otherwise;
//   update    alpha_j = r_j^T z_j / q_j, x_j += alpha_j p_j, r_j -= alpha_j v_j;
//   precond   t = W^T r, then z = W t (W = R^{-1}), one warp per 32 rows of W;
//   direction beta_j = r_j^T z_j / (previous), p_j = z_j + beta_j p_j, stopping rule.
// Under LSQ_PREC_MIXED a right-hand side whose recursive residual should be replaced (as in
// lsq_solve: convergence, a 10^4 drop since the last exact residual, or refresh_every
// iterations) makes its problem take an exact pass in double-FP32 arithmetic, r = b - A^T A x,
// before the direction update. Phases are separated by bounded grid barriers.
// Work units and per-unit partial sums are reduced in a fixed order (deterministic results).
#include <algorithm>
#include <math.h>
#include <vector>

#include "apass.cuh"
#include "common.cuh"

using lsq_apass::df_add;
using lsq_apass::df_fma;
using lsq_apass::narrow_f32;
using lsq_apass::split_df;

namespace {

constexpr int BT = 256;      // threads per CTA
constexpr int BW = BT / 32;  // warps per CTA
constexpr int KPMAX = 16;

// per right-hand side status bits
constexpr int F_ACTIVE = 1;

struct BProb {
  const void* A;
  int64_t n, ld;
  int d, dp, k, kp, nblk, chunk0, nchunk;
  const double* B;
  double* X;
  const double* W;
  const double* WT;
  double* R;    // [kp][dp]
  double* T;    // [kp][dp] W^T r
  double* Z;    // [kp][dp]
  double* P;    // [kp][dp]
  float* Pf;    // [dp][kp] FP32 copy of P (zero for stopped / padding right-hand sides)
  float* Xh;    // [dp][kp] head of x (exact passes)
  float* Xl;    // [dp][kp] tail of x
  double* slot; // [nblk][2][kp] per-block partial sums: 0 <b, x>, 1 r^T z
  double* rz;   // [2][kp] r^T z of the current residual (by iteration parity: read cur, write next)
  double* rz_rep;  // [kp] r^T z at the last exact residual
  int* flags;      // [2][kp] (by iteration parity)
  int* its;        // [kp] iterations taken
  int* st;         // [kp] status
  int* it_last;    // [kp] iteration of the last exact residual
  int* pstate;     // [2 * par] right-hand sides left and [2 * par + 1] the iteration this count is
                   // for, by iteration parity par; [4] needs an exact pass this iteration
  double lam1, tol2;
};

struct BatchArgs {
  BProb* probs;
  const int4* chunks;     // (problem, row0, row1, 0)
  const int64_t* part_off;  // chunk -> offset of its partials (kp * dp + kp doubles)
  const int* sched;       // chunk indices, CTA by CTA
  const int* sched_off;   // [P + 1]
  const int2* blocks;     // (problem, block of 32 columns / rows)
  int nblocks;
  double* part;
  unsigned* bar;
  int* err;
  int* cnt;               // [3] problems still active, rotating by iteration
  int* anyx;              // [3] some problem needs an exact pass, rotating
  int maxit, mixed, x0_zero, refresh_every;
  double replace2;
  int* out;               // [0] iterations, [1] passes, [2] exact passes
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// a problem is active in iteration `it` if the count written for that iteration is positive
__device__ __forceinline__ bool prob_active(const BProb& pr, int it) {
  const int par = it & 1;
  return pr.pstate[2 * par + 1] == it && pr.pstate[2 * par] > 0;
}

__device__ __forceinline__ void set_left(const BProb& pr, int it, int left) {
  const int par = it & 1;
  pr.pstate[2 * par] = left;
  pr.pstate[2 * par + 1] = it;
}

// ------------------------------------------------------------------------------------
// The pass over one chunk of rows in FP32 (TT = float) or FP64 (TT = double):
// part[j * dp + c] = sum_rows a_c (a . p_j),  part[kp * dp + j] = sum_rows (a . p_j)^2.
// Shared memory: As[TR][dp + 1] (tile), Ps[dp][KP] (directions), Yp[BW][KP][TR], Ys[TR][KP].
// ------------------------------------------------------------------------------------
template <typename TA, typename TT, int TR, int KP>
__device__ void pass_chunk(const BProb& pr, int64_t r0, int64_t r1, double* __restrict__ out, uint8_t* smem) {
  const int dp = pr.dp, d = pr.d, kp = pr.kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lda = dp + 1;
  TT* As = reinterpret_cast<TT*>(smem);
  TT* Ps = As + TR * lda;
  TT* Yp = Ps + dp * KP;
  TT* Ys = Yp + BW * KP * TR;
  const TA* A = reinterpret_cast<const TA*>(pr.A);
  // directions (padding columns j >= kp are zero)
  for (int e = tid; e < dp * KP; e += BT) {
    const int c = e / KP, j = e - c * KP;
    TT v = 0;
    if (j < kp) {
      if constexpr (sizeof(TT) == 4) v = pr.Pf[c * kp + j];
      else v = pr.P[j * dp + c];
    }
    Ps[e] = v;
  }
  // stage-2 ownership: NC groups of 32 columns; warp -> (group, row phase)
  const int NC = dp >> 5;
  const int cpw = NC > BW ? NC / BW : 1;       // column groups per warp (<= 2)
  const int rsplit = NC >= BW ? 1 : BW / NC;   // warps sharing a column group
  const int g0 = NC >= BW ? warp : warp % NC;
  const int rphase = NC >= BW ? 0 : warp / NC;
  TT acc[2][KP];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < KP; ++j) acc[h][j] = 0;
  TT qacc[2] = {0, 0};
  // register prefetch of the next tile: TR * dp / BT elements per thread (<= 64)
  constexpr int PFN = TR * 512 / BT;
  TA pf[PFN];
  const int per = TR * dp;
  auto load_tile = [&](int64_t t0) {
#pragma unroll
    for (int u = 0; u < PFN; ++u) {
      const int e = tid + u * BT;
      TA v = 0;
      if (e < per) {
        const int r = e / dp, c = e - r * dp;
        const int64_t row = t0 + r;
        if (row < r1 && c < d) v = __ldg(A + row * pr.ld + c);
      }
      pf[u] = v;
    }
  };
  load_tile(r0);
  for (int64_t t0 = r0; t0 < r1; t0 += TR) {
    __syncthreads();  // the previous tile is no longer read
#pragma unroll
    for (int u = 0; u < PFN; ++u) {
      const int e = tid + u * BT;
      if (e < per) {
        const int r = e / dp, c = e - r * dp;
        if constexpr (sizeof(TT) == 4) As[r * lda + c] = narrow_f32(pf[u]);
        else As[r * lda + c] = (TT)pf[u];
      }
    }
    __syncthreads();
    if (t0 + TR < r1) load_tile(t0 + TR);
    // stage 1: Y[r][j] = sum_c As[r][c] Ps[c][j]; warp w takes a slice of the columns, lane = row
    if (lane < TR) {
      TT y[KP];
#pragma unroll
      for (int j = 0; j < KP; ++j) y[j] = 0;
      const int cs = dp / BW, c0 = warp * cs;
      for (int c = c0; c < c0 + cs; ++c) {
        const TT a = As[lane * lda + c];
        const TT* pc = Ps + c * KP;
#pragma unroll
        for (int j = 0; j < KP; ++j) y[j] = fma(a, pc[j], y[j]);
      }
#pragma unroll
      for (int j = 0; j < KP; ++j) Yp[(warp * KP + j) * TR + lane] = y[j];
    }
    __syncthreads();
    for (int e = tid; e < TR * KP; e += BT) {
      const int j = e / TR, r = e - j * TR;
      TT s = 0;
#pragma unroll
      for (int w = 0; w < BW; ++w) s += Yp[(w * KP + j) * TR + r];
      Ys[r * KP + j] = s;
      qacc[e / BT] = fma(s, s, qacc[e / BT]);
    }
    __syncthreads();
    // stage 2: acc[h][j] += As[r][c] Ys[r][j] for the warp's column groups and row phase
    for (int r = rphase; r < TR; r += rsplit) {
      const TT* yr = Ys + r * KP;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h < cpw) {
          const TT a = As[r * lda + ((g0 + h * BW) << 5) + lane];
#pragma unroll
          for (int j = 0; j < KP; ++j) acc[h][j] = fma(a, yr[j], acc[h][j]);
        }
      }
    }
  }
  __syncthreads();
  // combine the row phases (reuse the tile area), then write the chunk's partials in FP64
  double* red = reinterpret_cast<double*>(smem);
  if (rsplit > 1) {
    for (int j = 0; j < KP; ++j) red[(rphase * KP + j) * (NC * 32) + (g0 << 5) + lane] = (double)acc[0][j];
    __syncthreads();
    for (int e = tid; e < kp * dp; e += BT) {
      const int j = e / dp, c = e - j * dp;
      double s = 0.0;
      for (int ph = 0; ph < rsplit; ++ph) s += red[(ph * KP + j) * (NC * 32) + c];
      out[e] = s;
    }
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (h < cpw)
        for (int j = 0; j < kp; ++j) out[j * dp + ((g0 + h * BW) << 5) + lane] = (double)acc[h][j];
  }
  // q_j: thread e of the reduction handled j = e / TR (TR = 32: warp w -> j = w, w + 8)
  __syncthreads();
  if (TR == 32) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = warp + h * BW;
      const double qs = warp_sum_d((double)qacc[h]);
      if (lane == 0 && j < kp && j < KP) out[kp * dp + j] = qs;
    }
  } else {
    // TR = 16: e = j * 16 + r, thread e -> j = e / 16 (threads 0..255 cover KP * 16 = 256 entries)
    double* qr = red;
    qr[tid] = (double)qacc[0];
    __syncthreads();
    if (tid < kp) {
      double s = 0.0;
      for (int r = 0; r < 16; ++r) s += qr[tid * 16 + r];
      out[kp * dp + tid] = s;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// Exact pass in double-FP32: part[j * dp + c] = sum_rows a_c (a . x_j) for every column of
// X (heads and tails of x, and of A when it is FP64); 16-row tiles.
// ------------------------------------------------------------------------------------
template <typename TA, int KP>
__device__ void pass_chunk_df(const BProb& pr, int64_t r0, int64_t r1, double* __restrict__ out, uint8_t* smem) {
  constexpr int TR = 16;
  const int dp = pr.dp, d = pr.d, kp = pr.kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lda = dp + 1;
  constexpr bool HASLO = sizeof(TA) == 8;
  float* Ah = reinterpret_cast<float*>(smem);
  float* Al = Ah + TR * lda;
  float* Xh = Al + (HASLO ? TR * lda : 0);
  float* Xl = Xh + dp * KP;
  float* Yph = Xl + dp * KP;
  float* Ypl = Yph + BW * KP * TR;
  float* Ysh = Ypl + BW * KP * TR;
  float* Ysl = Ysh + TR * KP;
  const TA* A = reinterpret_cast<const TA*>(pr.A);
  for (int e = tid; e < dp * KP; e += BT) {
    const int c = e / KP, j = e - c * KP;
    Xh[e] = j < kp ? pr.Xh[c * kp + j] : 0.f;
    Xl[e] = j < kp ? pr.Xl[c * kp + j] : 0.f;
  }
  const int NC = dp >> 5;
  const int cpw = NC > BW ? NC / BW : 1;
  const int rsplit = NC >= BW ? 1 : BW / NC;
  const int g0 = NC >= BW ? warp : warp % NC;
  const int rphase = NC >= BW ? 0 : warp / NC;
  float ah_[2][KP], al_[2][KP];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < KP; ++j) ah_[h][j] = al_[h][j] = 0.f;
  const int per = TR * dp;
  for (int64_t t0 = r0; t0 < r1; t0 += TR) {
    __syncthreads();
    for (int e = tid; e < per; e += BT) {
      const int r = e / dp, c = e - r * dp;
      const int64_t row = t0 + r;
      float hh = 0.f, ll = 0.f;
      if (row < r1 && c < d) split_df(__ldg(A + row * pr.ld + c), hh, ll);
      Ah[r * lda + c] = hh;
      if (HASLO) Al[r * lda + c] = ll;
    }
    __syncthreads();
    // stage 1 (lanes 0..15 = rows; two half-warps take adjacent column slices)
    {
      const int r = lane & 15, half = lane >> 4;
      float yh[KP], yl[KP];
#pragma unroll
      for (int j = 0; j < KP; ++j) yh[j] = yl[j] = 0.f;
      const int cs = dp / (2 * BW), c0 = (2 * warp + half) * cs;
      for (int c = c0; c < c0 + cs; ++c) {
        const float a = Ah[r * lda + c];
        const float al = HASLO ? Al[r * lda + c] : 0.f;
#pragma unroll
        for (int j = 0; j < KP; ++j) df_fma(a, al, Xh[c * KP + j], Xl[c * KP + j], yh[j], yl[j]);
      }
      // combine the two halves in double-FP32, then one entry per (warp, j, row)
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        const float oh = __shfl_xor_sync(0xffffffffu, yh[j], 16);
        const float ol = __shfl_xor_sync(0xffffffffu, yl[j], 16);
        df_add(yh[j], yl[j], oh, ol);
        if (half == 0) {
          Yph[(warp * KP + j) * TR + r] = yh[j];
          Ypl[(warp * KP + j) * TR + r] = yl[j];
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < TR * KP; e += BT) {
      const int j = e / TR, r = e - j * TR;
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int w = 0; w < BW; ++w) df_add(sh, sl, Yph[(w * KP + j) * TR + r], Ypl[(w * KP + j) * TR + r]);
      // renormalise so that the head carries the sum
      float h2, e2;
      lsq_apass::two_sum(sh, sl, h2, e2);
      Ysh[r * KP + j] = h2;
      Ysl[r * KP + j] = e2;
    }
    __syncthreads();
    for (int r = rphase; r < TR; r += rsplit) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h < cpw) {
          const int c = ((g0 + h * BW) << 5) + lane;
          const float a = Ah[r * lda + c];
          const float al = HASLO ? Al[r * lda + c] : 0.f;
#pragma unroll
          for (int j = 0; j < KP; ++j) df_fma(a, al, Ysh[r * KP + j], Ysl[r * KP + j], ah_[h][j], al_[h][j]);
        }
      }
    }
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem);
  if (rsplit > 1) {
    for (int j = 0; j < KP; ++j)
      red[(rphase * KP + j) * (NC * 32) + (g0 << 5) + lane] = (double)ah_[0][j] + (double)al_[0][j];
    __syncthreads();
    for (int e = tid; e < kp * dp; e += BT) {
      const int j = e / dp, c = e - j * dp;
      double s = 0.0;
      for (int ph = 0; ph < rsplit; ++ph) s += red[(ph * KP + j) * (NC * 32) + c];
      out[e] = s;
    }
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (h < cpw)
        for (int j = 0; j < kp; ++j)
          out[j * dp + ((g0 + h * BW) << 5) + lane] = (double)ah_[h][j] + (double)al_[h][j];
  }
  if (tid < kp) out[kp * dp + tid] = 0.0;
  __syncthreads();
}

// one pass over the chunks of this CTA; exact = double-FP32 (MIXED) pass over X for problems
// that asked for one, else the pass over the search directions
template <typename TA, bool MIXED>
__device__ void pass_phase(const BatchArgs& a, bool exact, int it, uint8_t* smem) {
  using TT = typename std::conditional<MIXED, float, double>::type;
  constexpr int TRP = (MIXED && sizeof(TA) == 4) ? 32 : 16;
  for (int u = a.sched_off[blockIdx.x]; u < a.sched_off[blockIdx.x + 1]; ++u) {
    const int ch = a.sched[u];
    const int4 cd = a.chunks[ch];
    const BProb& pr = a.probs[cd.x];
    if (!prob_active(pr, it)) continue;
    if (exact && pr.pstate[4] == 0) continue;
    double* out = a.part + a.part_off[ch];
    if (exact) {
      if (MIXED) {
        switch (pr.kp) {
          case 4: pass_chunk_df<TA, 4>(pr, cd.y, cd.z, out, smem); break;
          case 8: pass_chunk_df<TA, 8>(pr, cd.y, cd.z, out, smem); break;
          default: pass_chunk_df<TA, 16>(pr, cd.y, cd.z, out, smem); break;
        }
      } else {
        // FP64 mode: the exact pass is the FP64 pass over X (stored as P's FP64 layout by the caller)
        switch (pr.kp) {
          case 4: pass_chunk<TA, double, 16, 4>(pr, cd.y, cd.z, out, smem); break;
          case 8: pass_chunk<TA, double, 16, 8>(pr, cd.y, cd.z, out, smem); break;
          default: pass_chunk<TA, double, 16, 16>(pr, cd.y, cd.z, out, smem); break;
        }
      }
    } else {
      switch (pr.kp) {
        case 4: pass_chunk<TA, TT, TRP, 4>(pr, cd.y, cd.z, out, smem); break;
        case 8: pass_chunk<TA, TT, TRP, 8>(pr, cd.y, cd.z, out, smem); break;
        default: pass_chunk<TA, TT, TRP, 16>(pr, cd.y, cd.z, out, smem); break;
      }
    }
  }
}

// sum of the chunk partials of problem pr at offset `off` within each chunk's block (fixed order)
__device__ __forceinline__ double chunk_sum(const BatchArgs& a, const BProb& pr, int off) {
  double s = 0.0;
  for (int ch = pr.chunk0; ch < pr.chunk0 + pr.nchunk; ++ch) s += a.part[a.part_off[ch] + off];
  return s;
}

__device__ __forceinline__ double chunk_sum_warp(const BatchArgs& a, const BProb& pr, int off) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int ch = pr.chunk0 + lane; ch < pr.chunk0 + pr.nchunk; ch += 32) s += a.part[a.part_off[ch] + off];
  return warp_sum_d(s);
}

// t = W^T r (phase 1) or z = W t and the block's partial r^T z (phase 2), rows of one block
__device__ void precond_block(const BatchArgs& a, const BProb& pr, int blk, int phase, int cur) {
  const int lane = threadIdx.x & 31;
  const int d = pr.d, dp = pr.dp;
  double rzp[KPMAX];
#pragma unroll
  for (int j = 0; j < KPMAX; ++j) rzp[j] = 0.0;
  const int i0 = blk * 32, i1 = min(d, i0 + 32);
  for (int i = i0; i < i1; ++i) {
    double s[KPMAX];
#pragma unroll
    for (int j = 0; j < KPMAX; ++j) s[j] = 0.0;
    if (phase == 1) {
      const double* row = pr.WT + (int64_t)i * d;
      for (int c = lane; c <= i; c += 32) {
        const double w = __ldg(row + c);
#pragma unroll
        for (int j = 0; j < KPMAX; ++j)
          if (j < pr.k && (pr.flags[cur * pr.kp + j] & F_ACTIVE)) s[j] = fma(w, pr.R[j * dp + c], s[j]);
      }
    } else {
      const double* row = pr.W + (int64_t)i * d;
      for (int c = i + lane; c < d; c += 32) {
        const double w = __ldg(row + c);
#pragma unroll
        for (int j = 0; j < KPMAX; ++j)
          if (j < pr.k && (pr.flags[cur * pr.kp + j] & F_ACTIVE)) s[j] = fma(w, pr.T[j * dp + c], s[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < KPMAX; ++j) {
      if (j < pr.k && (pr.flags[cur * pr.kp + j] & F_ACTIVE)) {
        const double v = warp_sum_d(s[j]);
        if (phase == 1) {
          if (lane == 0) pr.T[j * dp + i] = v;
        } else {
          if (lane == 0) pr.Z[j * dp + i] = v;
          rzp[j] = fma(pr.R[j * dp + i], v, rzp[j]);
        }
      }
    }
  }
  if (phase == 2 && lane == 0) {
    for (int j = 0; j < pr.k; ++j)
      if (pr.flags[cur * pr.kp + j] & F_ACTIVE) pr.slot[(blk * 2 + 1) * pr.kp + j] = rzp[j];
  }
}

// split x into FP32 head and tail ([dp][kp] layout) for the columns of one block
__device__ void split_x_block(const BProb& pr, int blk) {
  const int lane = threadIdx.x & 31;
  const int c = blk * 32 + lane;
  for (int j = 0; j < pr.kp; ++j) {
    float h = 0.f, l = 0.f;
    if (c < pr.d && j < pr.k) {
      const double x = pr.X[j * pr.d + c];
      h = (float)x;
      l = (float)(x - (double)h);
    }
    if (c < pr.dp) {
      pr.Xh[c * pr.kp + j] = h;
      pr.Xl[c * pr.kp + j] = l;
    }
  }
}

// the stopping rule, the replacement rule and the direction update for one block of columns.
// Every block of a problem takes the same decisions (same sums in the same order); state shared
// by the blocks is read from parity `cur` and written to parity `nxt` by the block-0 warp.
__device__ void direction_block(const BatchArgs& a, const BProb& pr, int blk, int it, bool after_exact,
                                int* any_exact, int* active_cnt) {
  const int lane = threadIdx.x & 31;
  const int c = blk * 32 + lane;
  const int dp = pr.dp, kp = pr.kp;
  const int cur = it & 1, nxt = cur ^ 1;
  bool need = false;
  bool conv[KPMAX], act[KPMAX], fin[KPMAX];
  double rzn[KPMAX];
#pragma unroll
  for (int j = 0; j < KPMAX; ++j) {
    conv[j] = act[j] = fin[j] = false;
    rzn[j] = 0.0;
    if (j < pr.k && (pr.flags[cur * kp + j] & F_ACTIVE)) {
      act[j] = true;
      double rz = 0.0, bx = 0.0;
      for (int b = 0; b < pr.nblk; ++b) {
        rz += pr.slot[(b * 2 + 1) * kp + j];
        bx += pr.slot[(b * 2 + 0) * kp + j];
      }
      rzn[j] = rz;
      fin[j] = isfinite(rz);
      conv[j] = fin[j] && (rz == 0.0 || rz <= pr.tol2 * bx);
      if (a.mixed && !after_exact && fin[j] &&
          (conv[j] || rz <= a.replace2 * pr.rz_rep[j] || it + 1 - pr.it_last[j] >= a.refresh_every))
        need = true;
    }
  }
  if (need) {
    // the whole problem takes an exact residual before its directions are updated
    split_x_block(pr, blk);
    if (blk == 0 && lane == 0) {
      pr.pstate[4] = 1;
      atomicOr(any_exact, 1);
      atomicAdd(active_cnt, 1);
    }
    return;
  }
  int left = 0;
#pragma unroll
  for (int j = 0; j < KPMAX; ++j) {
    if (j >= kp) continue;
    const bool w0 = blk == 0 && lane == 0;
    if (!act[j]) {
      if (w0) {
        pr.flags[nxt * kp + j] = 0;
        pr.rz[nxt * kp + j] = pr.rz[cur * kp + j];
      }
      continue;
    }
    const bool stop = !fin[j] || conv[j] || it + 1 >= a.maxit;
    if (stop) {
      if (c < dp) pr.Pf[c * kp + j] = 0.f;
      if (w0) {
        pr.st[j] = !fin[j] ? LSQ_ERR_BREAKDOWN : (conv[j] ? LSQ_OK : LSQ_ERR_MAXIT);
        pr.flags[nxt * kp + j] = 0;
        pr.its[j] = it + 1;
        pr.rz[nxt * kp + j] = rzn[j];
      }
      continue;
    }
    ++left;
    const double beta = rzn[j] / pr.rz[cur * kp + j];
    if (c < pr.d) {
      const double p = pr.Z[j * dp + c] + beta * pr.P[j * dp + c];
      pr.P[j * dp + c] = p;
      pr.Pf[c * kp + j] = (float)p;
    }
    if (w0) {
      pr.flags[nxt * kp + j] = F_ACTIVE;
      pr.rz[nxt * kp + j] = rzn[j];
      pr.its[j] = it + 1;
      if (after_exact) {
        pr.rz_rep[j] = rzn[j];
        pr.it_last[j] = it + 1;
      }
    }
  }
  if (blk == 0 && lane == 0) {
    set_left(pr, it + 1, left);
    if (!after_exact) pr.pstate[4] = 0;
    if (left && !after_exact) atomicAdd(active_cnt, 1);
  }
}

template <typename TA, bool MIXED>
__global__ void __launch_bounds__(BT, 1) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int P = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * BW + (threadIdx.x >> 5), nw = P * BW;
  int passes = 0, exact_passes = 0;
#define BAR()                                        \
  do {                                               \
    if (grid_barrier(a.bar, P, a.err)) return;       \
  } while (0)

  // ---- initial residual r = b - A^T A x0 (or b), z = W W^T r, p = z
  for (int w = gw; w < a.nblocks; w += nw) {
    const int2 bk = a.blocks[w];
    const BProb& pr = a.probs[bk.x];
    const int c = bk.y * 32 + lane;
    for (int j = 0; j < pr.kp; ++j) {
      if (c < pr.dp) {
        const bool in = c < pr.d && j < pr.k;
        if (in && a.x0_zero) pr.X[j * pr.d + c] = 0.0;
        pr.R[j * pr.dp + c] = in ? pr.B[j * pr.d + c] : 0.0;
        pr.P[j * pr.dp + c] = (in && !MIXED) ? pr.X[j * pr.d + c] : 0.0;  // FP64 exact pass reads P
        pr.Pf[c * pr.kp + j] = 0.f;
        pr.Z[j * pr.dp + c] = 0.0;
        pr.T[j * pr.dp + c] = 0.0;
      }
    }
    if (!a.x0_zero && MIXED) split_x_block(pr, bk.y);
    if (bk.y == 0 && lane == 0) {
      set_left(pr, 0, 1);
      pr.pstate[2] = 0;
      pr.pstate[3] = -1;
      pr.pstate[4] = a.x0_zero ? 0 : 1;
      for (int j = 0; j < pr.kp; ++j) {
        pr.flags[j] = j < pr.k ? F_ACTIVE : 0;  // parity 0: iteration 0 reads it
        pr.flags[pr.kp + j] = 0;
        pr.its[j] = 0;
        pr.st[j] = LSQ_ERR_MAXIT;
        pr.it_last[j] = 0;
      }
    }
  }
  BAR();
  if (!a.x0_zero) {
    pass_phase<TA, MIXED>(a, true, 0, smem);
    ++passes;
    ++exact_passes;
    BAR();
    for (int w = gw; w < a.nblocks; w += nw) {
      const int2 bk = a.blocks[w];
      const BProb& pr = a.probs[bk.x];
      const int c = bk.y * 32 + lane;
      for (int j = 0; j < pr.k; ++j) {
        const double v = c < pr.d ? chunk_sum(a, pr, j * pr.dp + c) : 0.0;
        if (c < pr.d) pr.R[j * pr.dp + c] = pr.B[j * pr.d + c] - v;
      }
    }
    BAR();
  }
  // <b, x0> per block
  for (int w = gw; w < a.nblocks; w += nw) {
    const int2 bk = a.blocks[w];
    const BProb& pr = a.probs[bk.x];
    const int c = bk.y * 32 + lane;
    for (int j = 0; j < pr.k; ++j) {
      const double bx = warp_sum_d(c < pr.d ? pr.B[j * pr.d + c] * pr.X[j * pr.d + c] : 0.0);
      if (lane == 0) pr.slot[(bk.y * 2 + 0) * pr.kp + j] = bx;
    }
    if (!MIXED) {
      for (int j = 0; j < pr.k; ++j)
        if (c < pr.d) pr.P[j * pr.dp + c] = 0.0;
    }
  }
  BAR();
  for (int w = gw; w < a.nblocks; w += nw) precond_block(a, a.probs[a.blocks[w].x], a.blocks[w].y, 1, 0);
  BAR();
  for (int w = gw; w < a.nblocks; w += nw) precond_block(a, a.probs[a.blocks[w].x], a.blocks[w].y, 2, 0);
  BAR();
  // p = z, rz, stopping rule at x0
  {
    int* cnt = a.cnt + 0;
    for (int w = gw; w < a.nblocks; w += nw) {
      const int2 bk = a.blocks[w];
      const BProb& pr = a.probs[bk.x];
      const int c = bk.y * 32 + lane;
      int left = 0;
      for (int j = 0; j < pr.k; ++j) {
        double rz = 0.0, bx = 0.0;
        for (int b = 0; b < pr.nblk; ++b) {
          rz += pr.slot[(b * 2 + 1) * pr.kp + j];
          bx += pr.slot[(b * 2 + 0) * pr.kp + j];
        }
        const bool conv = rz == 0.0 || rz <= pr.tol2 * bx;
        const bool stop = conv || !isfinite(rz) || a.maxit == 0;
        if (c < pr.d) {
          const double z = pr.Z[j * pr.dp + c];
          pr.P[j * pr.dp + c] = stop ? 0.0 : z;
          pr.Pf[c * pr.kp + j] = stop ? 0.f : (float)z;
        }
        if (!stop) ++left;
        if (bk.y == 0 && lane == 0) {
          pr.rz[j] = rz;
          pr.rz_rep[j] = rz;
          if (stop) {
            pr.flags[j] = 0;  // parity 0 (no other block reads it in this phase)
            pr.st[j] = conv ? LSQ_OK : (isfinite(rz) ? LSQ_ERR_MAXIT : LSQ_ERR_BREAKDOWN);
          }
        }
      }
      if (bk.y == 0 && lane == 0) {
        set_left(pr, 0, left);
        pr.pstate[4] = 0;
        if (left) atomicAdd(cnt, 1);
      }
    }
  }
  BAR();
  int it = 0;
  while (it < a.maxit) {
    const int slot = it % 3, cur = it & 1;
    if (*(volatile int*)(a.cnt + slot) == 0) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.cnt[(it + 1) % 3] = 0;
      a.anyx[(it + 1) % 3] = 0;
    }
    // ---- pass over the search directions
    pass_phase<TA, MIXED>(a, false, it, smem);
    ++passes;
    if (!MIXED) ++exact_passes;
    BAR();
    // ---- x += alpha p, r -= alpha v, <b, x>
    for (int w = gw; w < a.nblocks; w += nw) {
      const int2 bk = a.blocks[w];
      const BProb& pr = a.probs[bk.x];
      if (!prob_active(pr, it)) continue;
      const int c = bk.y * 32 + lane;
      for (int j = 0; j < pr.k; ++j) {
        if (!(pr.flags[cur * pr.kp + j] & F_ACTIVE)) continue;
        const double q = chunk_sum_warp(a, pr, pr.kp * pr.dp + j);
        const double rz = pr.rz[cur * pr.kp + j];
        if (!(q > 0.0) || !isfinite(q)) {
          // breakdown: stop this right-hand side (the direction phase sees rz = NaN)
          if (lane == 0) pr.slot[(bk.y * 2 + 1) * pr.kp + j] = NAN;
          continue;
        }
        const double alpha = rz / q;
        double bxp = 0.0;
        if (c < pr.d) {
          const double v = chunk_sum(a, pr, j * pr.dp + c);
          const double x = pr.X[j * pr.d + c] + alpha * pr.P[j * pr.dp + c];
          pr.X[j * pr.d + c] = x;
          pr.R[j * pr.dp + c] -= alpha * v;
          bxp = pr.B[j * pr.d + c] * x;
        }
        bxp = warp_sum_d(bxp);
        if (lane == 0) pr.slot[(bk.y * 2 + 0) * pr.kp + j] = bxp;
      }
    }
    BAR();
    for (int w = gw; w < a.nblocks; w += nw) {
      const BProb& pr = a.probs[a.blocks[w].x];
      if (prob_active(pr, it)) precond_block(a, pr, a.blocks[w].y, 1, cur);
    }
    BAR();
    for (int w = gw; w < a.nblocks; w += nw) {
      const BProb& pr = a.probs[a.blocks[w].x];
      if (!prob_active(pr, it)) continue;
      // a breakdown marked in the update phase survives in the block's r^T z slot
      const int2 bk = a.blocks[w];
      unsigned nanmask = 0;
#pragma unroll
      for (int j = 0; j < KPMAX; ++j)
        if (j < pr.k && isnan(pr.slot[(bk.y * 2 + 1) * pr.kp + j])) nanmask |= 1u << j;
      precond_block(a, pr, bk.y, 2, cur);
      if (lane == 0)
        for (int j = 0; j < pr.k; ++j)
          if (nanmask & (1u << j)) pr.slot[(bk.y * 2 + 1) * pr.kp + j] = NAN;
    }
    BAR();
    int* cnt_next = a.cnt + (it + 1) % 3;
    int* anyx = a.anyx + (it + 1) % 3;
    for (int w = gw; w < a.nblocks; w += nw) {
      const BProb& pr = a.probs[a.blocks[w].x];
      if (prob_active(pr, it)) direction_block(a, pr, a.blocks[w].y, it, false, anyx, cnt_next);
    }
    BAR();
    if (MIXED && *(volatile int*)anyx) {
      // ---- exact residual for the problems that asked for one
      pass_phase<TA, MIXED>(a, true, it, smem);
      ++passes;
      ++exact_passes;
      BAR();
      for (int w = gw; w < a.nblocks; w += nw) {
        const int2 bk = a.blocks[w];
        const BProb& pr = a.probs[bk.x];
        if (!prob_active(pr, it) || !pr.pstate[4]) continue;
        const int c = bk.y * 32 + lane;
        for (int j = 0; j < pr.k; ++j) {
          if (!(pr.flags[cur * pr.kp + j] & F_ACTIVE)) continue;
          if (c < pr.d) pr.R[j * pr.dp + c] = pr.B[j * pr.d + c] - chunk_sum(a, pr, j * pr.dp + c);
        }
      }
      BAR();
      for (int w = gw; w < a.nblocks; w += nw) {
        const BProb& pr = a.probs[a.blocks[w].x];
        if (prob_active(pr, it) && pr.pstate[4]) precond_block(a, pr, a.blocks[w].y, 1, cur);
      }
      BAR();
      for (int w = gw; w < a.nblocks; w += nw) {
        const BProb& pr = a.probs[a.blocks[w].x];
        if (prob_active(pr, it) && pr.pstate[4]) precond_block(a, pr, a.blocks[w].y, 2, cur);
      }
      BAR();
      // the problem-wide counter of this iteration already counted these problems once
      for (int w = gw; w < a.nblocks; w += nw) {
        const BProb& pr = a.probs[a.blocks[w].x];
        if (prob_active(pr, it) && pr.pstate[4]) direction_block(a, pr, a.blocks[w].y, it, true, anyx, a.cnt + 3);
      }
      BAR();
    }
    ++it;
  }
#undef BAR
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = it;
    a.out[1] = passes;
    a.out[2] = exact_passes;
  }
}

__global__ void transpose_batch_kernel(const double* __restrict__ W, int d, double* __restrict__ WT) {
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

template <typename TA>
size_t pass_smem(bool mixed, int dp, int kp) {
  const int KP = kp <= 4 ? 4 : (kp <= 8 ? 8 : 16);
  size_t f32 = 0, df = 0, f64 = 0;
  if (mixed) {
    const int TR = sizeof(TA) == 4 ? 32 : 16;
    f32 = (size_t)(TR * (dp + 1) + dp * KP + BW * KP * TR + TR * KP) * 4;
    const int TRd = 16;
    df = (size_t)(TRd * (dp + 1) * (sizeof(TA) == 8 ? 2 : 1) + 2 * dp * KP + 2 * BW * KP * TRd + 2 * TRd * KP) * 4;
  } else {
    f64 = (size_t)(16 * (dp + 1) + dp * KP + BW * KP * 16 + 16 * KP) * 8;
  }
  // the row-phase reduction reuses the area: rsplit * KP * dp = 256 * KP doubles for dp < 256
  const size_t red = (size_t)(dp >= 256 ? 0 : 256) * KP * 8;
  return std::max(std::max(f32, df), std::max(f64, red));
}

int kp_of(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : 16); }
int dp_of(int d) {
  int e = 1;
  while (32 * e < d) e <<= 1;
  return 32 * e;
}

}  // namespace

extern "C" void lsq_batch_opts_default(lsq_batch_opts* o) {
  if (!o) return;
  o->sketch_type = LSQ_SKETCH_SJLT;
  o->s = 8;
  o->m_factor = 4.0;
  o->seed = 0;
  o->sketch_precision = LSQ_SKETCH_F32;
  o->precision = LSQ_PREC_MIXED;
  o->rho = 0.0;
  o->x0_zero = 1;
  o->refresh_every = 12;
  o->chunk_rows = 0;
  o->grid_blocks = 0;
}

extern "C" lsq_status lsq_solve_batched(lsq_ctx* ctx, int32_t nprob, lsq_problem* probs, double tol, int32_t maxit,
                                        const lsq_batch_opts* opts_in, lsq_batch_info* info) {
  if (!ctx || nprob < 1 || !probs || !(tol >= 0.0) || maxit < 0) return LSQ_ERR_ARG;
  lsq_batch_opts o;
  lsq_batch_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (o.precision != LSQ_PREC_F64 && o.precision != LSQ_PREC_MIXED) return LSQ_ERR_ARG;
  if (!(o.m_factor >= 1.0)) return LSQ_ERR_ARG;
  const bool mixed = o.precision == LSQ_PREC_MIXED;
  int dtype = -1;
  int max_d = 1, max_kp = 4;
  int64_t max_md = 1;
  for (int p = 0; p < nprob; ++p) {
    const lsq_problem& q = probs[p];
    if (!q.A.data || !q.B || !q.X) return LSQ_ERR_ARG;
    if (q.A.n < 1 || q.A.n >= (1ll << 31) || q.A.d < 1 || q.A.d > 512 || q.A.ld < q.A.d) return LSQ_ERR_ARG;
    if (q.A.dtype != LSQ_F64 && q.A.dtype != LSQ_F32) return LSQ_ERR_ARG;
    if (dtype >= 0 && q.A.dtype != dtype) return LSQ_ERR_ARG;  // one storage type per batch
    dtype = q.A.dtype;
    if (q.k < 1 || q.k > LSQ_MAX_RHS) return LSQ_ERR_ARG;
    const int64_t m = std::max<int64_t>(q.A.d, (int64_t)ceil(o.m_factor * (double)q.A.d));
    max_d = std::max<int>(max_d, (int)q.A.d);
    max_kp = std::max(max_kp, kp_of(q.k));
    max_md = std::max<int64_t>(max_md, m * q.A.d);
  }
  const int max_dp = dp_of(max_d);
  const int chunk_rows = o.chunk_rows > 0 ? ((o.chunk_rows + 31) / 32) * 32 : 2048;

  // ---- layout of the state arena
  std::vector<int4> chunks;
  std::vector<int64_t> part_off;
  std::vector<int2> blocks;
  std::vector<int> chunk0(nprob), nchunk(nprob);
  int64_t part_total = 0;
  size_t need = 0;
  auto add = [&](size_t bytes) {
    const size_t at = need;
    need += lsq_align256(bytes);
    return at;
  };
  struct Off {
    size_t W, WT, R, T, Z, P, Pf, Xh, Xl, slot, rz, rz_rep, flags, its, st, it_last, pstate;
  };
  std::vector<Off> off(nprob);
  for (int p = 0; p < nprob; ++p) {
    const int d = (int)probs[p].A.d, dp = dp_of(d), kp = kp_of(probs[p].k), nblk = (d + 31) / 32;
    Off& f = off[p];
    f.W = add((size_t)d * d * 8);
    f.WT = add((size_t)d * d * 8);
    f.R = add((size_t)kp * dp * 8);
    f.T = add((size_t)kp * dp * 8);
    f.Z = add((size_t)kp * dp * 8);
    f.P = add((size_t)kp * dp * 8);
    f.Pf = add((size_t)kp * dp * 4);
    f.Xh = add((size_t)kp * dp * 4);
    f.Xl = add((size_t)kp * dp * 4);
    f.slot = add((size_t)nblk * 2 * kp * 8);
    f.rz = add((size_t)2 * kp * 8);
    f.rz_rep = add((size_t)kp * 8);
    f.flags = add((size_t)2 * kp * 4);
    f.its = add((size_t)kp * 4);
    f.st = add((size_t)kp * 4);
    f.it_last = add((size_t)kp * 4);
    f.pstate = add(32);
    chunk0[p] = (int)chunks.size();
    for (int64_t r0 = 0; r0 < probs[p].A.n; r0 += chunk_rows) {
      chunks.push_back(make_int4(p, (int)r0, (int)std::min<int64_t>(probs[p].A.n, r0 + chunk_rows), 0));
      part_off.push_back(part_total);
      part_total += (int64_t)kp * dp + kp;
    }
    nchunk[p] = (int)chunks.size() - chunk0[p];
    for (int b = 0; b < nblk; ++b) blocks.push_back(make_int2(p, b));
  }
  const int nch = (int)chunks.size();

  // ---- persistent launch shape
  void* kern = dtype == LSQ_F64 ? (mixed ? (void*)batch_kernel<double, true> : (void*)batch_kernel<double, false>)
                                : (mixed ? (void*)batch_kernel<float, true> : (void*)batch_kernel<float, false>);
  const size_t smem = dtype == LSQ_F64 ? pass_smem<double>(mixed, max_dp, max_kp) : pass_smem<float>(mixed, max_dp, max_kp);
  if (smem > 227 * 1024) return LSQ_ERR_ARG;
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem));
  if (per_sm < 1) return LSQ_ERR_CUDA;
  int G = per_sm * ctx->sm_count;
  if (o.grid_blocks > 0) G = std::min(G, o.grid_blocks);
  G = std::max(1, std::min(G, std::max(nch, (int)blocks.size() / BW + 1)));

  // ---- static schedule of the chunks: longest first onto the least-loaded CTA
  std::vector<int> order(nch);
  std::vector<double> cost(nch);
  for (int c = 0; c < nch; ++c) {
    order[c] = c;
    const lsq_problem& q = probs[chunks[c].x];
    const double rows = chunks[c].z - chunks[c].y;
    const double kp = kp_of(q.k);
    cost[c] = rows * (double)dp_of((int)q.A.d) * std::max(1.0, kp / (mixed ? 6.0 : 1.0));
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> load(G, 0.0);
  std::vector<std::vector<int>> lists(G);
  for (int c : order) {
    int best = 0;
    for (int g = 1; g < G; ++g)
      if (load[g] < load[best]) best = g;
    load[best] += cost[c];
    lists[best].push_back(c);
  }
  std::vector<int> sched, sched_off(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    std::sort(lists[g].begin(), lists[g].end());
    sched_off[g] = (int)sched.size();
    for (int c : lists[g]) sched.push_back(c);
  }
  sched_off[G] = (int)sched.size();

  const size_t o_probs = add(sizeof(BProb) * nprob);
  const size_t o_chunks = add(sizeof(int4) * nch);
  const size_t o_poff = add(sizeof(int64_t) * nch);
  const size_t o_sched = add(sizeof(int) * std::max<size_t>(1, sched.size()));
  const size_t o_soff = add(sizeof(int) * (G + 1));
  const size_t o_blocks = add(sizeof(int2) * blocks.size());
  const size_t o_part = add((size_t)part_total * 8);
  const size_t o_bar = add(256);
  const size_t o_SA = add((size_t)max_md * 8);
  const size_t o_R = add((size_t)max_d * max_d * 8);
  lsq_status st = lsq_ensure_state(ctx, need);
  if (st != LSQ_OK) return st;
  char* base = reinterpret_cast<char*>(ctx->state);
  cudaStream_t s = ctx->stream;
  LSQ_CUDA_TRY(cudaEventRecord(ctx->ev0, s));

  // ---- sketch and factor every problem (instance t = p of the seed)
  cudaEvent_t e1, e2;
  LSQ_CUDA_TRY(cudaEventCreate(&e1));
  LSQ_CUDA_TRY(cudaEventCreate(&e2));
  float ms_sketch = 0.f, ms_factor = 0.f;
  std::vector<int> prob_status(nprob, LSQ_OK);
  lsq_status first_err = LSQ_OK;
  double* SA = reinterpret_cast<double*>(base + o_SA);
  double* Rtmp = reinterpret_cast<double*>(base + o_R);
  for (int p = 0; p < nprob; ++p) {
    const int d = (int)probs[p].A.d;
    const int64_t m = std::max<int64_t>(d, (int64_t)ceil(o.m_factor * (double)d));
    lsq_sketch_opts so;
    so.t = (uint32_t)p;
    so.s = (int)std::min<int64_t>(o.s > 0 ? o.s : 8, m);  // an SJLT column has at most m nonzeros
    so.precision = o.sketch_precision;
    cudaEventRecord(e1, s);
    st = lsq_sketch(ctx, &probs[p].A, o.sketch_type, m, o.seed, &so, SA);
    if (st != LSQ_OK) return st;
    cudaEventRecord(e2, s);
    double* W = reinterpret_cast<double*>(base + off[p].W);
    st = lsq_factor(ctx, SA, m, d, Rtmp, W);  // synchronises (rank check)
    float t1 = 0.f, t2 = 0.f;
    cudaEventElapsedTime(&t1, e1, e2);
    ms_sketch += t1;
    cudaEventRecord(e1, s);
    if (st == LSQ_ERR_RANK) {
      prob_status[p] = LSQ_ERR_RANK;
      if (first_err == LSQ_OK) first_err = st;
      LSQ_CUDA_TRY(cudaMemsetAsync(W, 0, (size_t)d * d * 8, s));
    } else if (st != LSQ_OK) {
      return st;
    }
    transpose_batch_kernel<<<dim3((d + 31) / 32, (d + 31) / 32), dim3(32, 8), 0, s>>>(
        W, d, reinterpret_cast<double*>(base + off[p].WT));
    LSQ_LAUNCH_CHECK();
    cudaEventRecord(e2, s);
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&t2, e1, e2);
    (void)t2;
  }
  {
    float tt = 0.f;
    cudaEventRecord(e1, s);
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&tt, ctx->ev0, e1);
    ms_factor = tt - ms_sketch;
  }

  // ---- device tables
  std::vector<BProb> hp(nprob);
  for (int p = 0; p < nprob; ++p) {
    const lsq_problem& q = probs[p];
    const Off& f = off[p];
    BProb& b = hp[p];
    b.A = q.A.data;
    b.n = q.A.n;
    b.ld = q.A.ld;
    b.d = (int)q.A.d;
    b.dp = dp_of(b.d);
    b.k = q.k;
    b.kp = kp_of(q.k);
    b.nblk = (b.d + 31) / 32;
    b.chunk0 = chunk0[p];
    b.nchunk = nchunk[p];
    b.B = q.B;
    b.X = q.X;
    b.W = reinterpret_cast<const double*>(base + f.W);
    b.WT = reinterpret_cast<const double*>(base + f.WT);
    b.R = reinterpret_cast<double*>(base + f.R);
    b.T = reinterpret_cast<double*>(base + f.T);
    b.Z = reinterpret_cast<double*>(base + f.Z);
    b.P = reinterpret_cast<double*>(base + f.P);
    b.Pf = reinterpret_cast<float*>(base + f.Pf);
    b.Xh = reinterpret_cast<float*>(base + f.Xh);
    b.Xl = reinterpret_cast<float*>(base + f.Xl);
    b.slot = reinterpret_cast<double*>(base + f.slot);
    b.rz = reinterpret_cast<double*>(base + f.rz);
    b.rz_rep = reinterpret_cast<double*>(base + f.rz_rep);
    b.flags = reinterpret_cast<int*>(base + f.flags);
    b.its = reinterpret_cast<int*>(base + f.its);
    b.st = reinterpret_cast<int*>(base + f.st);
    b.it_last = reinterpret_cast<int*>(base + f.it_last);
    b.pstate = reinterpret_cast<int*>(base + f.pstate);
    const int64_t m = std::max<int64_t>(b.d, (int64_t)ceil(o.m_factor * (double)b.d));
    double rho = o.rho > 0.0 ? o.rho : (double)b.d / (double)m;
    if (!(rho < 1.0)) rho = 0.999;
    b.lam1 = (1.0 + sqrt(rho)) * (1.0 + sqrt(rho));
    b.tol2 = tol * tol / b.lam1;
  }
  LSQ_CUDA_TRY(cudaMemcpy(base + o_probs, hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemcpy(base + o_chunks, chunks.data(), sizeof(int4) * nch, cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemcpy(base + o_poff, part_off.data(), sizeof(int64_t) * nch, cudaMemcpyHostToDevice));
  if (!sched.empty())
    LSQ_CUDA_TRY(cudaMemcpy(base + o_sched, sched.data(), sizeof(int) * sched.size(), cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemcpy(base + o_soff, sched_off.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemcpy(base + o_blocks, blocks.data(), sizeof(int2) * blocks.size(), cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemsetAsync(base + o_bar, 0, 256, s));

  BatchArgs a;
  a.probs = reinterpret_cast<BProb*>(base + o_probs);
  a.chunks = reinterpret_cast<const int4*>(base + o_chunks);
  a.part_off = reinterpret_cast<const int64_t*>(base + o_poff);
  a.sched = reinterpret_cast<const int*>(base + o_sched);
  a.sched_off = reinterpret_cast<const int*>(base + o_soff);
  a.blocks = reinterpret_cast<const int2*>(base + o_blocks);
  a.nblocks = (int)blocks.size();
  a.part = reinterpret_cast<double*>(base + o_part);
  a.bar = reinterpret_cast<unsigned*>(base + o_bar);
  a.err = reinterpret_cast<int*>(base + o_bar + 64);
  a.cnt = reinterpret_cast<int*>(base + o_bar + 96);    // [4]: 3 rotating + 1 sink
  a.anyx = reinterpret_cast<int*>(base + o_bar + 128);  // [3]
  a.out = reinterpret_cast<int*>(base + o_bar + 160);   // [3]
  a.maxit = maxit;
  a.mixed = mixed ? 1 : 0;
  a.x0_zero = o.x0_zero ? 1 : 0;
  a.refresh_every = o.refresh_every > 0 ? o.refresh_every : 12;
  a.replace2 = 1e-8;
  cudaEvent_t e3;
  LSQ_CUDA_TRY(cudaEventCreate(&e3));
  cudaEventRecord(e1, s);
  void* args[] = {&a};
  LSQ_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(G), dim3(BT), args, smem, s));
  lsq_count_launch();
  cudaEventRecord(e3, s);
  cudaEventRecord(ctx->ev1, s);
  LSQ_CUDA_TRY(cudaStreamSynchronize(s));
  float ms_solve = 0.f, ms_total = 0.f;
  cudaEventElapsedTime(&ms_solve, e1, e3);
  cudaEventElapsedTime(&ms_total, ctx->ev0, ctx->ev1);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  cudaEventDestroy(e3);
  int hdr[48];
  LSQ_CUDA_TRY(cudaMemcpy(hdr, base + o_bar, sizeof(hdr), cudaMemcpyDeviceToHost));
  const int errc = hdr[16];
  // per-problem results
  int iters_max = 0;
  lsq_status overall = errc ? (lsq_status)errc : first_err;
  for (int p = 0; p < nprob; ++p) {
    const int kp = kp_of(probs[p].k);
    std::vector<int> its(kp), sts(kp);
    LSQ_CUDA_TRY(cudaMemcpy(its.data(), base + off[p].its, kp * 4, cudaMemcpyDeviceToHost));
    LSQ_CUDA_TRY(cudaMemcpy(sts.data(), base + off[p].st, kp * 4, cudaMemcpyDeviceToHost));
    int it_p = 0, st_p = prob_status[p];
    for (int j = 0; j < probs[p].k; ++j) {
      it_p = std::max(it_p, its[j]);
      if (st_p == LSQ_OK && sts[j] != LSQ_OK) st_p = sts[j];
    }
    if (errc) st_p = errc;
    probs[p].iters = it_p;
    probs[p].status = st_p;
    iters_max = std::max(iters_max, it_p);
    if (overall == LSQ_OK && st_p != LSQ_OK) overall = (lsq_status)st_p;
  }
  if (info) {
    info->iters_max = iters_max;
    info->status = overall;
    info->passes = hdr[41];
    info->exact_passes = hdr[42];
    info->ms_total = ms_total;
    info->ms_sketch = ms_sketch;
    info->ms_factor = ms_factor;
    info->ms_solve = ms_solve;
  }
  return overall;
}
