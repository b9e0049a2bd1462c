// batch.cu -- many independent least-squares problems of uneven n, d and numbers of
// right-hand sides k, each solved by PCG (Section 1, eq. (PCG)) per right-hand side with
// the problem's own fixed embedding; all problems advance in lockstep iterations.
//
// One iteration is a CUDA graph of six kernels (replayed; the iteration index lives in device
// memory):
//   pass      one read of every active A_p gives V = A_p^T (A_p P_p) and q_j = ||A_p p_j||^2 for
//             all k_p directions at once; chunks of rows are taken from a queue (costliest
//             first) by 512-thread CTAs; a tile of rows is staged in shared memory,
//             Y = A_tile P (rows x k) and then V += A_tile^T Y (register tiles), FP32 under
//             LSQ_PREC_MIXED, FP64 otherwise;
//   update    alpha_j = r_j^T z_j / q_j, x_j += alpha_j p_j, r_j -= alpha_j v_j (a warp per 32
//             columns);
//   precond   t = W^T r, then z = W t (W = R^{-1}), a CTA per 32 rows of W whose warps split the
//             columns, so a problem's FP64 work spreads over many SMs;
//   direction beta_j, p_j = z_j + beta_j p_j, the stopping rule; then a one-thread tick.
// Under LSQ_PREC_MIXED a right-hand side whose recursive residual should be replaced (a 10^5
// drop of its norm since the last exact residual, refresh_every iterations, or convergence)
// makes its problem spend its next iteration on an exact residual r = b - A^T A x from a pass
// in double-FP32 arithmetic, before its directions are updated.  Partial sums are reduced in a
// fixed order (deterministic results).
#include <algorithm>
#include <map>
#include <math.h>
#include <mutex>
#include <vector>

#include "apass.cuh"
#include "common.cuh"

using lsq_apass::df_add;
using lsq_apass::df_fma;
using lsq_apass::narrow_f32;
using lsq_apass::split_df;

namespace {

constexpr int BT = 256;      // threads per CTA of the block kernels
constexpr int BW = BT / 32;  // warps per CTA
constexpr int KPMAX = 16;

// per right-hand side status bits
constexpr int F_ACTIVE = 1;

struct BProb {
  const void* A;
  int64_t n, ld;
  int d, dp, k, kp, nblk, chunk0, nchunk, vec;  // vec: rows of A allow 16-byte loads
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
  int* pstate;     // by iteration parity par: [2 * par] right-hand sides left, [2 * par + 1] the
                   // iteration this count is for, [4 + par] this iteration is an exact residual step
  double lam1, tol2;
};

struct BatchArgs {
  BProb* probs;
  int nprob;
  const int4* chunks;       // (problem, row0, row1, 0)
  const int64_t* part_off;  // chunk -> offset of its partials (kp * dp + kp doubles)
  const int* order;         // chunks by decreasing cost (the queue)
  int nchunks;
  const int2* blocks;       // (problem, block of 32 columns / rows)
  int nblocks;
  double* part;
  int* iter;                // the current iteration
  int* qhead;               // [3] queue heads, rotating by iteration
  int* cnt;                 // [4] problems active in the next iteration, rotating; [3] unused
  int* anyx;                // [3] some problem takes an exact residual step, rotating
  int* stats;               // [0] iterations run, [1] iterations with an exact residual step
  int* err;                 // first error of a kernel
  int smem_bytes;           // dynamic shared memory of the pass kernel
  int maxit, mixed, x0_zero, refresh_every;
  double replace2;
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

__device__ __forceinline__ bool exact_step(const BProb& pr, int it) { return pr.pstate[4 + (it & 1)] != 0; }

__device__ __forceinline__ void set_left(const BProb& pr, int it, int left) {
  const int par = it & 1;
  pr.pstate[2 * par] = left;
  pr.pstate[2 * par + 1] = it;
}

// ------------------------------------------------------------------------------------
// The pass over one chunk of rows in FP32 (TT = float) or FP64 (TT = double):
// part[j * dp + c] = sum_rows a_c (a . p_j),  part[kp * dp + j] = sum_rows (a . p_j)^2.
// A tile holds TE elements: tr = TE / dp rows (dp a power of two >= 32), so narrow problems
// take tall tiles.  Stage 1, Y = A_tile P: each of the 256 lanes owns one row and a slice of
// the columns (S = 256 / tr slices; for tr > 256 a lane owns tr / 256 whole rows); stage 2,
// V += A_tile^T Y: a warp owns 32 columns (or 64) and every KP accumulator of them, warps
// sharing columns split the rows.  Shared memory: As[tr][dp] (XOR-swizzled), Ps[dp][KP],
// Yp[S][KP][tr] (S > 1), Ys[tr][KP].
// ------------------------------------------------------------------------------------
template <typename TA, typename TT, int TE, int KP, int PT>
__device__ __forceinline__ void pass_chunk(const BProb& pr, int64_t r0, int64_t r1, double* __restrict__ out,
                                           uint8_t* smem) {
  constexpr int BT = PT, BW = PT / 32;
  constexpr int CPWMAX = 16 / BW > 1 ? 16 / BW : 1;  // column groups per warp at dp = 512
  const int dp = pr.dp, d = pr.d, kp = pr.kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lgdp = 31 - __clz(dp);
  const int tr = TE >> lgdp;                 // rows per tile
  const int S = tr >= BT ? 1 : BT / tr;      // column slices of stage 1
  const int RPL = tr > BT ? tr / BT : 1;     // rows per lane of stage 1 (<= 2)
  TT* As = reinterpret_cast<TT*>(smem);
  TT* Ps = As + TE;
  TT* Yp = Ps + dp * KP;
  TT* Ys = Yp + (S > 1 ? S * KP * tr : 0);
  const TA* A = reinterpret_cast<const TA*>(pr.A);
  // directions: zero past the problem's columns and right-hand sides, whose stored entries are
  // never written (the tile's A is zero there, but a stale non-finite value times zero is not)
  for (int e = tid; e < dp * KP; e += BT) {
    const int c = e / KP, j = e - c * KP;
    TT v = 0;
    if (j < pr.k && c < d) {
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
  TT acc[CPWMAX][KP];
#pragma unroll
  for (int h = 0; h < CPWMAX; ++h)
#pragma unroll
    for (int j = 0; j < KP; ++j) acc[h][j] = 0;
  // sums of squares for q: S == 1, qacc[j] of the rows the thread owns; S > 1, qacc[h] of its
  // entries h of the slice reduction (tr KP / BT <= KP / 2 of them)
  TT qacc[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) qacc[j] = 0;
  constexpr int QH = KP / 2 > 1 ? KP / 2 : 1;
  const int lgtr = 31 - __clz(TE) - lgdp;
  // stage-1 ownership: global lane g -> row g % tr (+ BT i) and slice g / tr
  const int g = tid;
  const int s_row = tr >= BT ? g : g % tr;
  const int s_slice = tr >= BT ? 0 : g / tr;
  const int cs = dp / S;
  // Tile element (r, c) sits at As[r * dp + (c ^ 4 (r & 7))]: aligned groups of 4 columns move
  // together, so a 16-byte read of 4 columns by 8 consecutive rows (a quarter warp) and a read
  // of 32 consecutive columns of one row both hit distinct banks.  Loads are
  // 16-byte vectors (V elements) when A allows; the next tile waits in registers.
  constexpr int V = sizeof(TA) == 4 ? 4 : 2;
  using VT = typename std::conditional<sizeof(TA) == 4, float4, double2>::type;
  constexpr int NU = TE / (V * BT);
  const int lgu = lgdp - (V == 4 ? 2 : 1);  // log2 of the vectors per row
  const int units = tr << lgu;
  const bool vec_ok = pr.vec != 0;
  TA pf[NU * V];
#define LSQ_LOAD_TILE(t0_)                                                                   \
  _Pragma("unroll") for (int i = 0; i < NU; ++i) {                                           \
    const int u = tid + i * BT;                                                              \
    const int r = u >> lgu, c = (u & ((1 << lgu) - 1)) * V;                                  \
    const int64_t row = (t0_) + r;                                                           \
    const bool in_ = u < units && row < r1;                                                  \
    const TA* src = A + (in_ ? row * pr.ld + c : 0);                                         \
    if (in_ && vec_ok && c + V <= d) {                                                       \
      const VT x = __ldg(reinterpret_cast<const VT*>(src));                                  \
      pf[i * V + 0] = x.x;                                                                   \
      pf[i * V + 1] = x.y;                                                                   \
      if constexpr (V == 4) {                                                                \
        pf[i * V + 2] = reinterpret_cast<const float4&>(x).z;                                \
        pf[i * V + 3] = reinterpret_cast<const float4&>(x).w;                                \
      }                                                                                      \
    } else {                                                                                 \
      _Pragma("unroll") for (int q = 0; q < V; ++q) pf[i * V + q] =                          \
          (in_ && c + q < d) ? __ldg(src + q) : (TA)0;                                       \
    }                                                                                        \
  }
  LSQ_LOAD_TILE(r0)
  for (int64_t t0 = r0; t0 < r1; t0 += tr) {
    __syncthreads();  // the previous tile is no longer read
#pragma unroll
    for (int i = 0; i < NU; ++i) {
      const int u = tid + i * BT;
      if (u < units) {
        const int r = u >> lgu, c = (u & ((1 << lgu) - 1)) * V;
        const int sw = (r & 7) << 2;
        if constexpr (sizeof(TT) == 4 && V == 4) {
          // the swizzle moves whole aligned groups of 4 columns: one 16-byte store
          *reinterpret_cast<float4*>(As + r * dp + (c ^ sw)) =
              make_float4(narrow_f32(pf[i * V + 0]), narrow_f32(pf[i * V + 1]), narrow_f32(pf[i * V + 2]),
                          narrow_f32(pf[i * V + 3]));
        } else {
#pragma unroll
          for (int q = 0; q < V; ++q) {
            if constexpr (sizeof(TT) == 4) As[r * dp + ((c + q) ^ sw)] = narrow_f32(pf[i * V + q]);
            else As[r * dp + ((c + q) ^ sw)] = (TT)pf[i * V + q];
          }
        }
      }
    }
    __syncthreads();
    if (t0 + tr < r1) {
      LSQ_LOAD_TILE(t0 + tr)
    }
    // stage 1
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (i < RPL) {
        const int r = s_row + i * BT;
        TT y[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) y[j] = 0;
        const int c0 = s_slice * cs;
        const TT* arow = As + r * dp;
        const int sw = (r & 7) << 2;
        if constexpr (sizeof(TT) == 4 && TE == 16384) {
          // cs = TE / BT = 32 columns: 8 groups of 4, each one 16-byte load of the row
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const int c = c0 + 4 * g;
            const float4 a4 = *reinterpret_cast<const float4*>(arow + (c ^ sw));
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const TT* pc = Ps + (c + q) * KP;
#pragma unroll
              for (int j = 0; j < KP; ++j) y[j] = fma(av[q], pc[j], y[j]);
            }
          }
        } else {
          for (int c = c0; c < c0 + cs; ++c) {
            const TT a = arow[c ^ sw];
            const TT* pc = Ps + c * KP;
#pragma unroll
            for (int j = 0; j < KP; ++j) y[j] = fma(a, pc[j], y[j]);
          }
        }
        if (S == 1) {
#pragma unroll
          for (int j = 0; j < KP; ++j) {
            Ys[r * KP + j] = y[j];
            qacc[j] = fma(y[j], y[j], qacc[j]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < KP; ++j) Yp[(s_slice * KP + j) * tr + r] = y[j];
        }
      }
    }
    __syncthreads();
    if (S > 1) {
      // every thread: entries e = tid + BT h -> (j = e / tr, r = e % tr), summed over the slices;
      // with tr | BT a thread sees j = tid / tr + h BT / tr and row tid % tr
#pragma unroll
      for (int h = 0; h < QH; ++h) {
        const int e = tid + h * BT;
        if (e < tr * KP) {
          const int j = e >> lgtr, r = e & (tr - 1);
          TT sum = 0;
          for (int q = 0; q < S; ++q) sum += Yp[(q * KP + j) * tr + r];
          Ys[r * KP + j] = sum;
          qacc[h] = fma(sum, sum, qacc[h]);
        }
      }
      __syncthreads();
    }
    // stage 2: acc[h][j] += As[r][c] Ys[r][j] for the warp's column groups and row phase
    for (int r = rphase; r < tr; r += rsplit) {
      const TT* yr = Ys + r * KP;
      const int sw = (r & 7) << 2;
#pragma unroll
      for (int h = 0; h < CPWMAX; ++h) {
        if (h < cpw) {
          const TT a = As[r * dp + ((((g0 + h * BW) << 5) + lane) ^ sw)];
#pragma unroll
          for (int j = 0; j < KP; ++j) acc[h][j] = fma(a, yr[j], acc[h][j]);
        }
      }
    }
  }
#undef LSQ_LOAD_TILE
  __syncthreads();
  // combine the row phases (reuse the tile area), then write the chunk's partials in FP64
  double* red = reinterpret_cast<double*>(smem);
  if (rsplit > 1) {
#pragma unroll
    for (int j = 0; j < KP; ++j) red[(rphase * KP + j) * (NC * 32) + (g0 << 5) + lane] = (double)acc[0][j];
    __syncthreads();
    for (int e = tid; e < kp * dp; e += BT) {
      const int j = e / dp, c = e - j * dp;
      double sum = 0.0;
      for (int ph = 0; ph < rsplit; ++ph) sum += red[(ph * KP + j) * (NC * 32) + c];
      out[e] = sum;
    }
  } else {
#pragma unroll
    for (int h = 0; h < CPWMAX; ++h)
      if (h < cpw)
#pragma unroll
        for (int j = 0; j < KP; ++j)
          if (j < kp) out[j * dp + ((g0 + h * BW) << 5) + lane] = (double)acc[h][j];
  }
  __syncthreads();
  if (S == 1) {
    // q_j = sum of the per-thread sums of squares: warp sums, then the warps in order
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const double w = warp_sum_d((double)qacc[j]);
      if (lane == 0) red[warp * KP + j] = w;
    }
    __syncthreads();
    if (tid < kp) {
      double sum = 0.0;
      for (int w = 0; w < BW; ++w) sum += red[w * KP + tid];
      out[kp * dp + tid] = sum;
    }
  } else {
    // q_j from the threads that summed rows of j: h = j / (BT / tr), threads (j % (BT / tr)) tr + r
#pragma unroll
    for (int h = 0; h < QH; ++h) red[h * BT + tid] = (double)qacc[h];
    __syncthreads();
    if (tid < kp) {
      const int per_h = BT / tr;
      const int h = tid / per_h, t0 = (tid % per_h) * tr;
      double sum = 0.0;
      for (int r = 0; r < tr; ++r) sum += red[h * BT + t0 + r];
      out[kp * dp + tid] = sum;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// Exact pass in double-FP32: part[j * dp + c] = sum_rows a_c (a . x_j) for every column of
// X (heads and tails of x, and of A when it is FP64).  The structure of pass_chunk (tiles of
// TE elements, tall for narrow problems; stage 1 with a lane per row and S column slices;
// stage 2 with a warp per 32 columns) with every product and sum in double-FP32: products by
// FMA-exact TwoProduct plus the cross terms, sums by TwoSum (Dekker 1971; Knuth).
// ------------------------------------------------------------------------------------
template <typename TA, int KP, int PT>
__device__ __forceinline__ void pass_chunk_df(const BProb& pr, int64_t r0, int64_t r1, double* __restrict__ out,
                                              uint8_t* smem) {
  constexpr int BT = PT, BW = PT / 32;
  constexpr int CPWMAX = 16 / BW > 1 ? 16 / BW : 1;
  constexpr int TE = 8192;
  constexpr bool HASLO = sizeof(TA) == 8;
  const int dp = pr.dp, d = pr.d, kp = pr.kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lgdp = 31 - __clz(dp);
  const int tr = TE >> lgdp;
  const int S = tr >= BT ? 1 : BT / tr;
  const int RPL = tr > BT ? tr / BT : 1;
  float* Ah = reinterpret_cast<float*>(smem);
  float* Al = Ah + TE;
  float* Xh = Al + (HASLO ? TE : 0);
  float* Xl = Xh + dp * KP;
  float* Yph = Xl + dp * KP;
  float* Ypl = Yph + (S > 1 ? S * KP * tr : 0);
  float* Ysh = Ypl + (S > 1 ? S * KP * tr : 0);
  float* Ysl = Ysh + tr * KP;
  const TA* A = reinterpret_cast<const TA*>(pr.A);
  for (int e = tid; e < dp * KP; e += BT) {
    const int c = e / KP, j = e - c * KP;
    // (zero past the problem's columns and right-hand sides, as for the directions)
    Xh[e] = (j < pr.k && c < d) ? pr.Xh[c * kp + j] : 0.f;
    Xl[e] = (j < pr.k && c < d) ? pr.Xl[c * kp + j] : 0.f;
  }
  const int NC = dp >> 5;
  const int cpw = NC > BW ? NC / BW : 1;
  const int rsplit = NC >= BW ? 1 : BW / NC;
  const int g0 = NC >= BW ? warp : warp % NC;
  const int rphase = NC >= BW ? 0 : warp / NC;
  float ah_[CPWMAX][KP], al_[CPWMAX][KP];
#pragma unroll
  for (int h = 0; h < CPWMAX; ++h)
#pragma unroll
    for (int j = 0; j < KP; ++j) ah_[h][j] = al_[h][j] = 0.f;
  const int s_row = tr >= BT ? tid : tid % tr;
  const int s_slice = tr >= BT ? 0 : tid / tr;
  const int cs = dp / S;
  const int per = tr * dp;
  for (int64_t t0 = r0; t0 < r1; t0 += tr) {
    __syncthreads();
    for (int e = tid; e < per; e += BT) {
      const int r = e >> lgdp, c = e & (dp - 1);
      const int64_t row = t0 + r;
      float hh = 0.f, ll = 0.f;
      if (row < r1 && c < d) split_df(__ldg(A + row * pr.ld + c), hh, ll);
      const int sc = r * dp + (c ^ (r & 31));
      Ah[sc] = hh;
      if (HASLO) Al[sc] = ll;
    }
    __syncthreads();
    // stage 1
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (i < RPL) {
        const int r = s_row + i * BT;
        float yh[KP], yl[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) yh[j] = yl[j] = 0.f;
        const int c0 = s_slice * cs;
        const int sw = r & 31;
        for (int c = c0; c < c0 + cs; ++c) {
          const int sc = r * dp + (c ^ sw);
          const float av = Ah[sc];
          const float al = HASLO ? Al[sc] : 0.f;
#pragma unroll
          for (int j = 0; j < KP; ++j) df_fma(av, al, Xh[c * KP + j], Xl[c * KP + j], yh[j], yl[j]);
        }
        if (S == 1) {
#pragma unroll
          for (int j = 0; j < KP; ++j) {
            float h2, e2;
            lsq_apass::two_sum(yh[j], yl[j], h2, e2);
            Ysh[r * KP + j] = h2;
            Ysl[r * KP + j] = e2;
          }
        } else {
#pragma unroll
          for (int j = 0; j < KP; ++j) {
            Yph[(s_slice * KP + j) * tr + r] = yh[j];
            Ypl[(s_slice * KP + j) * tr + r] = yl[j];
          }
        }
      }
    }
    __syncthreads();
    if (S > 1) {
      for (int e = tid; e < tr * KP; e += BT) {
        const int j = e / tr, r = e - j * tr;
        float sh = 0.f, sl = 0.f;
        for (int q = 0; q < S; ++q) df_add(sh, sl, Yph[(q * KP + j) * tr + r], Ypl[(q * KP + j) * tr + r]);
        float h2, e2;
        lsq_apass::two_sum(sh, sl, h2, e2);
        Ysh[r * KP + j] = h2;
        Ysl[r * KP + j] = e2;
      }
      __syncthreads();
    }
    // stage 2
    for (int r = rphase; r < tr; r += rsplit) {
      const int sw = r & 31;
#pragma unroll
      for (int h = 0; h < CPWMAX; ++h) {
        if (h < cpw) {
          const int c = ((g0 + h * BW) << 5) + lane;
          const int sc = r * dp + (c ^ sw);
          const float av = Ah[sc];
          const float al = HASLO ? Al[sc] : 0.f;
#pragma unroll
          for (int j = 0; j < KP; ++j) df_fma(av, al, Ysh[r * KP + j], Ysl[r * KP + j], ah_[h][j], al_[h][j]);
        }
      }
    }
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem);
  if (rsplit > 1) {
#pragma unroll
    for (int j = 0; j < KP; ++j)
      red[(rphase * KP + j) * (NC * 32) + (g0 << 5) + lane] = (double)ah_[0][j] + (double)al_[0][j];
    __syncthreads();
    for (int e = tid; e < kp * dp; e += BT) {
      const int j = e / dp, c = e - j * dp;
      double sum = 0.0;
      for (int ph = 0; ph < rsplit; ++ph) sum += red[(ph * KP + j) * (NC * 32) + c];
      out[e] = sum;
    }
  } else {
#pragma unroll
    for (int h = 0; h < CPWMAX; ++h)
      if (h < cpw)
#pragma unroll
        for (int j = 0; j < KP; ++j)
          if (j < kp) out[j * dp + ((g0 + h * BW) << 5) + lane] = (double)ah_[h][j] + (double)al_[h][j];
  }
  if (tid < kp) out[kp * dp + tid] = 0.0;
  __syncthreads();
}

constexpr int PT = 512;  // threads of a pass CTA (the other kernels use BT)

// shared memory of the passes for one problem shape (the launch takes the maximum); mirrors
// the layouts of pass_chunk and pass_chunk_df with PT threads
__host__ __device__ inline size_t pass_smem_shape(bool mixed, bool a_f64, int dp, int KP) {
  auto tile = [&](size_t es, int TE) {
    const int tr = TE / dp;
    const int S = tr >= PT ? 1 : PT / tr;
    return (size_t)(TE + dp * KP + (S > 1 ? S * KP * tr : 0) + tr * KP) * es;
  };
  size_t f = 0;
  if (mixed) {
    f = tile(4, a_f64 ? 8192 : 16384);
    const int TEd = 8192, trd = TEd / dp, Sd = trd >= PT ? 1 : PT / trd;
    const size_t df =
        (size_t)(TEd * (a_f64 ? 2 : 1) + 2 * dp * KP + (Sd > 1 ? 2 * Sd * KP * trd : 0) + 2 * trd * KP) * 4;
    f = f > df ? f : df;
  } else {
    f = tile(8, 8192);
  }
  // the end-of-chunk reductions reuse the area: PT * KP doubles (row phases), W * KP (q)
  const size_t red = (size_t)PT * KP * 8;
  return f > red ? f : red;
}


// one chunk of the pass: for a problem in an exact residual step the double-FP32 (MIXED) or
// FP64 pass over X, else the pass over the search directions
template <typename TA, bool MIXED>
__device__ void pass_one(const BatchArgs& a, int ch, bool force_exact, int it, uint8_t* smem) {
  using TT = typename std::conditional<MIXED, float, double>::type;
  // elements of a tile: 64 KB of FP32; 8192 when the tile or the prefetch is FP64
  constexpr int TEP = (MIXED && sizeof(TA) == 4) ? 16384 : 8192;
  const int4 cd = a.chunks[ch];
  const BProb& pr = a.probs[cd.x];
  if (!prob_active(pr, it)) return;
  if (pass_smem_shape(MIXED, sizeof(TA) == 8, pr.dp, pr.kp) > (size_t)a.smem_bytes) {
    // the launch's shared memory does not hold this shape (cannot happen with the host's sizing)
    if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)LSQ_ERR_ARG);
    return;
  }
  const bool exact = force_exact || exact_step(pr, it);
  double* out = a.part + a.part_off[ch];
  if (exact) {
    if constexpr (MIXED) {
      switch (pr.kp) {
        case 4: pass_chunk_df<TA, 4, PT>(pr, cd.y, cd.z, out, smem); break;
        case 8: pass_chunk_df<TA, 8, PT>(pr, cd.y, cd.z, out, smem); break;
        case 12: pass_chunk_df<TA, 12, PT>(pr, cd.y, cd.z, out, smem); break;
        default: pass_chunk_df<TA, 16, PT>(pr, cd.y, cd.z, out, smem); break;
      }
    } else {
      // FP64 mode: the exact pass is the FP64 pass over X (held in P's layout by the caller)
      switch (pr.kp) {
        case 4: pass_chunk<TA, double, 8192, 4, PT>(pr, cd.y, cd.z, out, smem); break;
        case 8: pass_chunk<TA, double, 8192, 8, PT>(pr, cd.y, cd.z, out, smem); break;
        case 12: pass_chunk<TA, double, 8192, 12, PT>(pr, cd.y, cd.z, out, smem); break;
        default: pass_chunk<TA, double, 8192, 16, PT>(pr, cd.y, cd.z, out, smem); break;
      }
    }
  } else {
    switch (pr.kp) {
      case 4: pass_chunk<TA, TT, TEP, 4, PT>(pr, cd.y, cd.z, out, smem); break;
      case 8: pass_chunk<TA, TT, TEP, 8, PT>(pr, cd.y, cd.z, out, smem); break;
      case 12: pass_chunk<TA, TT, TEP, 12, PT>(pr, cd.y, cd.z, out, smem); break;
      default: pass_chunk<TA, TT, TEP, 16, PT>(pr, cd.y, cd.z, out, smem); break;
    }
  }
}

// the pass: CTAs take chunks from the iteration's queue (costliest first)
template <typename TA, bool MIXED>
__global__ void __launch_bounds__(PT, 1) bpass_kernel(BatchArgs a, int force_exact) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int next;
  const int it = *(volatile int*)a.iter;
  int* head = a.qhead + it % 3;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(head, 1);
    __syncthreads();
    const int u = next;
    __syncthreads();
    if (u >= a.nchunks) break;
    pass_one<TA, MIXED>(a, a.order[u], force_exact != 0, it, smem);
  }
}

#include "bring.cuh"

// sum of the chunk partials of problem pr at offset `off` within each chunk's block (fixed
// order); a problem's chunks are consecutive and their partial blocks equally spaced
__device__ __forceinline__ double chunk_sum(const BatchArgs& a, const BProb& pr, int off) {
  const double* base = a.part + a.part_off[pr.chunk0] + off;
  const int64_t stride = (int64_t)pr.kp * pr.dp + pr.kp;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int ch = 0;
  for (; ch + 8 <= pr.nchunk; ch += 8) {
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] += base[(ch + q) * stride];
  }
  for (; ch < pr.nchunk; ++ch) s[0] += base[ch * stride];
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

__device__ __forceinline__ double chunk_sum_warp(const BatchArgs& a, const BProb& pr, int off) {
  const int lane = threadIdx.x & 31;
  const double* base = a.part + a.part_off[pr.chunk0] + off;
  const int64_t stride = (int64_t)pr.kp * pr.dp + pr.kp;
  double s = 0.0;
  for (int ch = lane; ch < pr.nchunk; ch += 32) s += base[ch * stride];
  return warp_sum_d(s);
}

// t = W^T r (phase 1) or z = W t and the block's partial r^T z (phase 2) for the 32 rows of one
// block, one CTA: lane = row; t_i = sum_{c <= i} W[c][i] r_c reads rows of W, z_i =
// sum_{c >= i} W^T[c][i] t_c reads rows of W^T (contiguous loads, broadcast vector entries); the
// warps take consecutive slices of the columns and their sums are added in warp order.
template <int PHASE>
__global__ void __launch_bounds__(BT) bprec_kernel(BatchArgs a) {
  __shared__ double red[BW][KPMAX][32];
  const int it = *(volatile int*)a.iter;
  const int cur = it & 1;
  const int2 bk = a.blocks[blockIdx.x];
  const BProb& pr = a.probs[bk.x];
  if (!prob_active(pr, it)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = pr.d, dp = pr.dp, blk = bk.y;
  const int i = blk * 32 + lane;
  const bool row_ok = i < d;
  unsigned act = 0;
  for (int j = 0; j < pr.k; ++j)
    if (pr.flags[cur * pr.kp + j] & F_ACTIVE) act |= 1u << j;
  const double* M = PHASE == 1 ? pr.W : pr.WT;
  const double* vin = PHASE == 1 ? pr.R : pr.T;
  const int c_lo = PHASE == 1 ? 0 : blk * 32;
  const int c_hi = PHASE == 1 ? min(d, blk * 32 + 32) : d;
  const int span = (c_hi - c_lo + BW - 1) / BW;
  const int w_lo = c_lo + warp * span, w_hi = min(c_hi, w_lo + span);
  const int ic = row_ok ? i : 0;
  double s[KPMAX];
#pragma unroll
  for (int j = 0; j < KPMAX; ++j) s[j] = 0.0;
  for (int c = w_lo; c < w_hi; ++c) {
    const double w = __ldg(M + (int64_t)c * d + ic);
#pragma unroll
    for (int j = 0; j < KPMAX; ++j)
      if (act & (1u << j)) s[j] = fma(w, vin[j * dp + c], s[j]);
  }
#pragma unroll
  for (int j = 0; j < KPMAX; ++j) red[warp][j][lane] = s[j];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < KPMAX; ++j) {
      if (!(act & (1u << j))) continue;
      double v = 0.0;
      for (int w = 0; w < BW; ++w) v += red[w][j][lane];
      if (PHASE == 1) {
        if (row_ok) pr.T[j * dp + i] = v;
      } else {
        if (row_ok) pr.Z[j * dp + i] = v;
        // a breakdown marked by the update survives in the block's r^T z slot
        const double rz = warp_sum_d(row_ok ? pr.R[j * dp + i] * v : 0.0);
        if (lane == 0) {
          double* sl = pr.slot + (blk * 2 + 1) * pr.kp + j;
          if (!isnan(*sl)) *sl = rz;
        }
      }
    }
  }
}

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
      // a drop-triggered replacement within 10^2 (in norm) of the tolerance is left to the one
      // that confirms convergence a few iterations later -- unless the drop since the last
      // exact residual passes FP32's resolution (10^7 in norm), where the recursive residual
      // is rounding noise
      const bool near = rz <= 1e4 * pr.tol2 * bx && rz >= 1e-14 * pr.rz_rep[j];
      if (a.mixed && !after_exact && fin[j] &&
          (conv[j] || (!near && rz <= a.replace2 * pr.rz_rep[j]) || it + 1 - pr.it_last[j] >= a.refresh_every))
        need = true;
    }
  }
  if (need) {
    // the problem's next iteration replaces its residuals by b - H x before the directions
    // are updated
    split_x_block(pr, blk);
    if (blk == 0 && lane == 0) {
      for (int j = 0; j < kp; ++j) {  // the state carries over unchanged into the exact step
        pr.flags[nxt * kp + j] = pr.flags[cur * kp + j];
        pr.rz[nxt * kp + j] = pr.rz[cur * kp + j];
      }
      pr.pstate[4 + nxt] = 1;
      set_left(pr, it + 1, 1);
      atomicAdd(active_cnt, 1);
      atomicOr(any_exact, 1);
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
        pr.rz[nxt * kp + j] = rzn[j];
      }
      continue;
    }
    ++left;
    // after an exact residual more than twice (in norm) the recursive one of the previous
    // iteration, the old direction is not trusted: restart from the preconditioned residual
    const double beta = (after_exact && rzn[j] > 4.0 * pr.rz[cur * kp + j]) ? 0.0 : rzn[j] / pr.rz[cur * kp + j];
    if (c < pr.d) {
      const double p = pr.Z[j * dp + c] + beta * pr.P[j * dp + c];
      pr.P[j * dp + c] = p;
      pr.Pf[c * kp + j] = (float)p;
    }
    if (w0) {
      pr.flags[nxt * kp + j] = F_ACTIVE;
      pr.rz[nxt * kp + j] = rzn[j];
      if (after_exact) {
        pr.rz_rep[j] = rzn[j];
        pr.it_last[j] = it + 1;
      }
    }
  }
  if (blk == 0 && lane == 0) {
    set_left(pr, it + 1, left);
    pr.pstate[4 + nxt] = 0;
    if (left) atomicAdd(active_cnt, 1);
  }
}


// set-up per block: r = b (x0 = 0) or the split of x0 for the exact pass; state of iteration 0
template <bool MIXED>
__global__ void __launch_bounds__(BT) binit_kernel(BatchArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * BW + (threadIdx.x >> 5);
  if (w >= a.nblocks) return;
  const int2 bk = a.blocks[w];
  const BProb& pr = a.probs[bk.x];
  const int c = bk.y * 32 + lane;
  for (int j = 0; j < pr.kp; ++j) {
    if (c < pr.dp) {
      const bool in = c < pr.d && j < pr.k;
      if (in && a.x0_zero) pr.X[j * pr.d + c] = 0.0;
      pr.R[j * pr.dp + c] = in ? pr.B[j * pr.d + c] : 0.0;
      pr.P[j * pr.dp + c] = (in && !MIXED) ? pr.X[j * pr.d + c] : 0.0;  // the FP64 exact pass reads P
      pr.Pf[c * pr.kp + j] = 0.f;
      pr.Z[j * pr.dp + c] = 0.0;
      pr.T[j * pr.dp + c] = 0.0;
    }
  }
  if (!a.x0_zero && MIXED) split_x_block(pr, bk.y);
  // <b, x0>, and r^T z slots cleared
  for (int j = 0; j < pr.k; ++j) {
    const double bx = warp_sum_d(c < pr.d ? pr.B[j * pr.d + c] * pr.X[j * pr.d + c] : 0.0);
    if (lane == 0) {
      pr.slot[(bk.y * 2 + 0) * pr.kp + j] = bx;
      pr.slot[(bk.y * 2 + 1) * pr.kp + j] = 0.0;
    }
  }
  if (bk.y == 0 && lane == 0) {
    set_left(pr, 0, 1);
    pr.pstate[2] = 0;
    pr.pstate[3] = -1;
    pr.pstate[4] = 0;
    pr.pstate[5] = 0;
    for (int j = 0; j < pr.kp; ++j) {
      pr.flags[j] = j < pr.k ? F_ACTIVE : 0;  // parity 0: iteration 0 reads it
      pr.flags[pr.kp + j] = 0;
      pr.its[j] = 0;
      pr.st[j] = LSQ_ERR_MAXIT;
      pr.it_last[j] = 0;
    }
  }
}

// r0 = b - A^T A x0 from the exact pass
template <bool MIXED>
__global__ void __launch_bounds__(BT) bresid_kernel(BatchArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * BW + (threadIdx.x >> 5);
  if (w >= a.nblocks) return;
  const int2 bk = a.blocks[w];
  const BProb& pr = a.probs[bk.x];
  const int c = bk.y * 32 + lane;
  for (int j = 0; j < pr.k; ++j) {
    const double v = c < pr.d ? chunk_sum(a, pr, j * pr.dp + c) : 0.0;
    if (c < pr.d) {
      pr.R[j * pr.dp + c] = pr.B[j * pr.d + c] - v;
      if (!MIXED) pr.P[j * pr.dp + c] = 0.0;
    }
  }
}

// p = z, r^T z and the stopping rule at x0
__global__ void __launch_bounds__(BT) binitdir_kernel(BatchArgs a) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * BW + (threadIdx.x >> 5);
  if (w >= a.nblocks) return;
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
        pr.flags[j] = 0;  // parity 0 (no other block reads it in this kernel)
        pr.st[j] = conv ? LSQ_OK : (isfinite(rz) ? LSQ_ERR_MAXIT : LSQ_ERR_BREAKDOWN);
      }
    }
  }
  if (bk.y == 0 && lane == 0) {
    set_left(pr, 0, left);
    if (left) atomicAdd(a.cnt, 1);
  }
}

// x += alpha p, r -= alpha v, <b, x>; or r = b - H x in an exact residual step.  One CTA per
// block of 32 columns; warp w takes the right-hand sides j = w, w + 8, ... (lane = column), so
// the sums over a problem's chunk partials run on all warps.
__global__ void __launch_bounds__(BT) bupdate_kernel(BatchArgs a) {
  const int it = *(volatile int*)a.iter;
  const int cur = it & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int2 bk = a.blocks[blockIdx.x];
  const BProb& pr = a.probs[bk.x];
  if (!prob_active(pr, it)) return;
  const int c = bk.y * 32 + lane;
  const bool exact = exact_step(pr, it);
  for (int j = warp; j < pr.k; j += BW) {
    if (!(pr.flags[cur * pr.kp + j] & F_ACTIVE)) continue;
    if (exact) {
      if (c < pr.d) pr.R[j * pr.dp + c] = pr.B[j * pr.d + c] - chunk_sum(a, pr, j * pr.dp + c);
      if (lane == 0) pr.slot[(bk.y * 2 + 1) * pr.kp + j] = 0.0;
      continue;
    }
    const double q = chunk_sum_warp(a, pr, pr.kp * pr.dp + j);
    const double rz = pr.rz[cur * pr.kp + j];
    if (!(q > 0.0) || !isfinite(q)) {
      // breakdown: stop this right-hand side (the direction kernel sees r^T z = NaN)
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
    if (lane == 0) {
      pr.slot[(bk.y * 2 + 0) * pr.kp + j] = bxp;
      pr.slot[(bk.y * 2 + 1) * pr.kp + j] = 0.0;
      if (bk.y == 0) pr.its[j] += 1;
    }
  }
}

__global__ void __launch_bounds__(BT) bdir_kernel(BatchArgs a) {
  const int it = *(volatile int*)a.iter;
  const int w = blockIdx.x * BW + (threadIdx.x >> 5);
  if (w >= a.nblocks) return;
  const int2 bk = a.blocks[w];
  const BProb& pr = a.probs[bk.x];
  if (prob_active(pr, it))
    direction_block(a, pr, bk.y, it, exact_step(pr, it), a.anyx + (it + 1) % 3, a.cnt + (it + 1) % 3);
}

// end of an iteration: counters of the next one, then the iteration index; inside the
// device-driven loop (use_cond) also whether the loop goes on: some problem is still active in
// the next iteration and the iteration limit is not reached, so the loop always ends
__global__ void btick_kernel(BatchArgs a, cudaGraphConditionalHandle cond, int use_cond) {
  const int it = *a.iter;
  a.stats[0] += 1;
  if (a.anyx[it % 3]) a.stats[1] += 1;
  const int nx = it + 1;
  a.qhead[nx % 3] = 0;
  a.cnt[(nx + 1) % 3] = 0;
  a.anyx[(nx + 1) % 3] = 0;
  *a.iter = nx;
  if (use_cond) cudaGraphSetConditional(cond, (nx < a.maxit && a.cnt[nx % 3] > 0) ? 1u : 0u);
}

// before the device-driven loop: whether iteration 0 runs at all
__global__ void bcond_kernel(BatchArgs a, cudaGraphConditionalHandle cond) {
  const int it = *a.iter;
  cudaGraphSetConditional(cond, (it < a.maxit && a.cnt[it % 3] > 0) ? 1u : 0u);
}

int kp_of(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 12 ? 12 : 16)); }
int dp_of(int d) {
  int e = 1;
  while (32 * e < d) e <<= 1;
  return 32 * e;
}

// The work units of the pass: chunks of rows (problem, row0, row1), the offsets of their
// partial sums, each problem's first chunk and count, and the queue order (decreasing cost:
// rows x columns, scaled by the directions per element under the FP32 arithmetic).
struct ChunkPlan {
  int64_t elems;  // target elements of A per chunk
  std::vector<int4> chunks;
  std::vector<int64_t> part_off;
  std::vector<int> chunk0, nchunk, order;
  int64_t part_total;
};

ChunkPlan plan_chunks(const lsq_problem* probs, int nprob, int chunk_rows_opt, int64_t elems, bool mixed) {
  ChunkPlan pl;
  pl.elems = elems;
  pl.part_total = 0;
  pl.chunk0.resize(nprob);
  pl.nchunk.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    const int d = (int)probs[p].A.d, dp = dp_of(d), kp = kp_of(probs[p].k);
    const int rows = chunk_rows_opt > 0 ? ((chunk_rows_opt + 31) / 32) * 32
                                        : std::max<int>(256, (int)std::min<int64_t>(elems / dp, 1 << 30));
    pl.chunk0[p] = (int)pl.chunks.size();
    for (int64_t r0 = 0; r0 < probs[p].A.n; r0 += rows) {
      pl.chunks.push_back(make_int4(p, (int)r0, (int)std::min<int64_t>(probs[p].A.n, r0 + rows), 0));
      pl.part_off.push_back(pl.part_total);
      pl.part_total += (int64_t)kp * dp + kp;
    }
    pl.nchunk[p] = (int)pl.chunks.size() - pl.chunk0[p];
  }
  const int nch = (int)pl.chunks.size();
  pl.order.resize(nch);
  std::vector<double> cost(nch);
  for (int c = 0; c < nch; ++c) {
    pl.order[c] = c;
    const lsq_problem& q = probs[pl.chunks[c].x];
    const double rows = pl.chunks[c].z - pl.chunks[c].y;
    cost[c] = rows * (double)dp_of((int)q.A.d) * std::max(1.0, kp_of(q.k) / (mixed ? 6.0 : 1.0));
  }
  std::stable_sort(pl.order.begin(), pl.order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  return pl;
}

// The autotuner's choices, per device and batch shape (FNV-1a over the shapes), for the process
struct TunedPass {
  int64_t elems;
  int grid;
};
std::mutex g_tuned_mu;
std::map<uint64_t, TunedPass> g_tuned;

uint64_t batch_signature(int device, const lsq_problem* probs, int nprob, int dtype, bool mixed) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xFFu;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)device);
  mix((uint64_t)dtype);
  mix(mixed ? 1u : 0u);
  mix((uint64_t)nprob);
  for (int p = 0; p < nprob; ++p) {
    mix((uint64_t)probs[p].A.n);
    mix((uint64_t)probs[p].A.d);
    mix((uint64_t)probs[p].k);
  }
  return h;
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
  o->refresh_every = 40;
  o->chunk_rows = 0;
  o->grid_blocks = 0;
  o->profile_phases = 0;
  o->autotune = 1;
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
  for (int p = 0; p < nprob; ++p) {
    const lsq_problem& q = probs[p];
    if (!q.A.data || !q.B || !q.X) return LSQ_ERR_ARG;
    if (q.A.n < 1 || q.A.n >= (1ll << 31) || q.A.d < 1 || q.A.d > 512 || q.A.ld < q.A.d) return LSQ_ERR_ARG;
    if (q.A.dtype != LSQ_F64 && q.A.dtype != LSQ_F32) return LSQ_ERR_ARG;
    if (dtype >= 0 && q.A.dtype != dtype) return LSQ_ERR_ARG;  // one storage type per batch
    dtype = q.A.dtype;
    if (q.k < 1 || q.k > LSQ_MAX_RHS) return LSQ_ERR_ARG;
    const int64_t m = std::max<int64_t>(q.A.d, (int64_t)ceil(o.m_factor * (double)q.A.d));
  }
  // work unit of the pass: about `elems` elements of A (default 2^20, 4 MB of FP32), at least 256
  // rows, so narrow problems do not spread over thousands of partial sums; the autotuner tries
  // several sizes (and pass grids) on the first batch of a shape and keeps the fastest
  std::vector<int64_t> elems_cand = {(int64_t)1 << 20};
  if (o.chunk_rows <= 0 && o.autotune) elems_cand = {(int64_t)1 << 20, (int64_t)1 << 19, (int64_t)1 << 21};
  std::vector<ChunkPlan> plans;
  for (int64_t e : elems_cand) plans.push_back(plan_chunks(probs, nprob, o.chunk_rows, e, mixed));
  size_t max_nch = 0;
  int64_t max_part = 0;
  for (const ChunkPlan& pl : plans) {
    max_nch = std::max(max_nch, pl.chunks.size());
    max_part = std::max(max_part, pl.part_total);
  }

  // ---- layout of the state arena
  std::vector<int2> blocks;
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
    for (int b = 0; b < nblk; ++b) blocks.push_back(make_int2(p, b));
  }
  const ChunkPlan* plan = &plans[0];

  // ---- the pass kernel: dynamic shared memory for the largest problem shape
  // FP32 A in the mixed precision with contiguous, 16-byte aligned rows: the ring pass (rows
  // staged by bulk copies); otherwise the tiled pass
  bool ring = dtype == LSQ_F32 && mixed;
  for (int p = 0; p < nprob && ring; ++p)
    ring = probs[p].A.ld == probs[p].A.d && ((uintptr_t)probs[p].A.data % 16) == 0;
  void* kpass = ring ? (void*)bpass_ring_kernel
                     : dtype == LSQ_F64 ? (mixed ? (void*)bpass_kernel<double, true> : (void*)bpass_kernel<double, false>)
                                        : (mixed ? (void*)bpass_kernel<float, true> : (void*)bpass_kernel<float, false>);
  const int pass_threads = ring ? RT : PT;
  size_t smem = 0;
  if (ring) {
    smem = RSMEM;
  } else {
    for (int p = 0; p < nprob; ++p) {
      const int dpp = dp_of((int)probs[p].A.d), kpp = kp_of(probs[p].k);
      smem = std::max(smem, pass_smem_shape(mixed, dtype == LSQ_F64, dpp, kpp));
    }
  }
  if (smem > 227 * 1024) return LSQ_ERR_ARG;
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kpass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kpass, pass_threads, smem));
  if (per_sm < 1) return LSQ_ERR_CUDA;
  const int G_full = per_sm * ctx->sm_count;
  int G = G_full;
  if (o.grid_blocks > 0) G = std::min(G, o.grid_blocks);
  // the pass grids the autotuner tries: all resident CTAs, one per SM
  std::vector<int> grid_cand = {G};
  if (o.grid_blocks <= 0 && o.autotune && per_sm > 1) grid_cand.push_back(ctx->sm_count);

  const size_t o_probs = add(sizeof(BProb) * nprob);
  const size_t o_chunks = add(sizeof(int4) * max_nch);
  const size_t o_poff = add(sizeof(int64_t) * max_nch);
  const size_t o_order = add(sizeof(int) * max_nch);
  const size_t o_blocks = add(sizeof(int2) * blocks.size());
  const size_t o_part = add((size_t)max_part * 8);
  const size_t o_ctl = add(256);
  std::vector<size_t> sa_off(nprob);
  for (int p = 0; p < nprob; ++p) {
    const int64_t dd = probs[p].A.d;
    const int64_t m = std::max<int64_t>(dd, (int64_t)ceil(o.m_factor * (double)dd));
    sa_off[p] = add((size_t)m * dd * 8);
  }
  lsq_status st = lsq_ensure_state(ctx, need);
  if (st != LSQ_OK) return st;
  char* base = reinterpret_cast<char*>(ctx->state);
  cudaStream_t s = ctx->stream;
  LSQ_CUDA_TRY(cudaEventRecord(ctx->ev0, s));

  // ---- sketch every problem (instance t = p of the seed), then factor them all at once
  cudaEvent_t e1, e2;
  LSQ_CUDA_TRY(cudaEventCreate(&e1));
  LSQ_CUDA_TRY(cudaEventCreate(&e2));
  std::vector<int> prob_status(nprob, LSQ_OK);
  lsq_status first_err = LSQ_OK;
  std::vector<const double*> sa_ptr(nprob);
  std::vector<double*> w_ptr(nprob), wt_ptr(nprob);
  std::vector<int> m_of(nprob), d_of(nprob);
  cudaEventRecord(e1, s);
  // SJLT in FP32 (or over BF16-rounded A): every problem's sketch in one launch
  const bool one_launch = o.sketch_type == LSQ_SKETCH_SJLT &&
                          (o.sketch_precision == LSQ_SKETCH_F32 || o.sketch_precision == LSQ_SKETCH_BF16);
  if (one_launch) {
    std::vector<lsq_matrix> mats(nprob);
    std::vector<int> ms(nprob);
    std::vector<double*> sas(nprob);
    for (int p = 0; p < nprob; ++p) {
      const int d = (int)probs[p].A.d;
      mats[p] = probs[p].A;
      ms[p] = (int)std::max<int64_t>(d, (int64_t)ceil(o.m_factor * (double)d));
      sas[p] = reinterpret_cast<double*>(base + sa_off[p]);
    }
    st = lsq_sjlt_batched(ctx, nprob, mats.data(), ms.data(), o.s > 0 ? o.s : 8, o.seed, sas.data(),
                          o.sketch_precision == LSQ_SKETCH_BF16);
    if (st != LSQ_OK) return st;
  }
  for (int p = 0; p < nprob; ++p) {
    const int d = (int)probs[p].A.d;
    const int64_t m = std::max<int64_t>(d, (int64_t)ceil(o.m_factor * (double)d));
    double* SA = reinterpret_cast<double*>(base + sa_off[p]);
    sa_ptr[p] = SA;
    w_ptr[p] = reinterpret_cast<double*>(base + off[p].W);
    wt_ptr[p] = reinterpret_cast<double*>(base + off[p].WT);
    m_of[p] = (int)m;
    d_of[p] = d;
    if (one_launch) continue;
    lsq_sketch_opts so = {};
    so.t = (uint32_t)p;
    so.s = (int)std::min<int64_t>(o.s > 0 ? o.s : 8, m);  // an SJLT column has at most m nonzeros
    so.precision = o.sketch_precision;
    so.a32 = nullptr;
    so.ld32 = 0;
    st = lsq_sketch(ctx, &probs[p].A, o.sketch_type, m, o.seed, &so, SA);
    if (st != LSQ_OK) return st;
  }
  cudaEventRecord(e2, s);
  st = lsq_factor_batched(ctx, nprob, sa_ptr.data(), m_of.data(), d_of.data(), w_ptr.data(), wt_ptr.data(), mixed,
                          prob_status.data());
  if (st != LSQ_OK) return st;
  for (int p = 0; p < nprob; ++p) {
    if (prob_status[p] == LSQ_ERR_RANK) {
      if (first_err == LSQ_OK) first_err = LSQ_ERR_RANK;
      const size_t dd = (size_t)d_of[p] * d_of[p] * 8;
      LSQ_CUDA_TRY(cudaMemsetAsync(w_ptr[p], 0, dd, s));
      LSQ_CUDA_TRY(cudaMemsetAsync(wt_ptr[p], 0, dd, s));
    }
  }
  float ms_sketch = 0.f, ms_factor = 0.f;
  {
    cudaEvent_t e3;
    LSQ_CUDA_TRY(cudaEventCreate(&e3));
    cudaEventRecord(e3, s);
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&ms_sketch, e1, e2);
    cudaEventElapsedTime(&ms_factor, e2, e3);
    cudaEventDestroy(e3);
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
    {
      const size_t es = q.A.dtype == LSQ_F64 ? 8 : 4;
      b.vec = (((uintptr_t)q.A.data % 16) == 0 && ((size_t)q.A.ld * es) % 16 == 0) ? 1 : 0;
    }
    b.chunk0 = plan->chunk0[p];
    b.nchunk = plan->nchunk[p];
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
  // the chunk tables of a plan (the caller makes sure no pass still reads the old ones)
  auto upload_plan = [&](const ChunkPlan& pl) -> lsq_status {
    const size_t nc = pl.chunks.size();
    LSQ_CUDA_TRY(cudaMemcpy(base + o_chunks, pl.chunks.data(), sizeof(int4) * nc, cudaMemcpyHostToDevice));
    LSQ_CUDA_TRY(cudaMemcpy(base + o_poff, pl.part_off.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice));
    LSQ_CUDA_TRY(cudaMemcpy(base + o_order, pl.order.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
    return LSQ_OK;
  };
  st = upload_plan(*plan);
  if (st != LSQ_OK) return st;
  LSQ_CUDA_TRY(cudaMemcpy(base + o_blocks, blocks.data(), sizeof(int2) * blocks.size(), cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemsetAsync(base + o_ctl, 0, 256, s));

  BatchArgs a;
  a.probs = reinterpret_cast<BProb*>(base + o_probs);
  a.nprob = nprob;
  a.chunks = reinterpret_cast<const int4*>(base + o_chunks);
  a.part_off = reinterpret_cast<const int64_t*>(base + o_poff);
  a.order = reinterpret_cast<const int*>(base + o_order);
  a.nchunks = (int)plan->chunks.size();
  a.blocks = reinterpret_cast<const int2*>(base + o_blocks);
  a.nblocks = (int)blocks.size();
  a.part = reinterpret_cast<double*>(base + o_part);
  int* ctl = reinterpret_cast<int*>(base + o_ctl);
  a.iter = ctl + 0;
  a.qhead = ctl + 4;   // [3]
  a.cnt = ctl + 8;     // [4]
  a.anyx = ctl + 12;   // [3]
  a.stats = ctl + 16;  // [2]
  a.err = ctl + 20;
  a.smem_bytes = (int)smem;
  a.maxit = maxit;
  a.mixed = mixed ? 1 : 0;
  a.x0_zero = o.x0_zero ? 1 : 0;
  a.refresh_every = o.refresh_every > 0 ? o.refresh_every : 40;
  // one replacement after a 10^5 drop of the residual norm and one to confirm convergence:
  // the FP32 passes' drift after the first (~1e-7 of that level) stays below 1e-10 overall
  a.replace2 = 1e-10;

  const int nbk = (int)blocks.size();
  const int gblk = (nbk + BW - 1) / BW;
  auto launch_pass = [&](int force_exact, bool count) -> lsq_status {
    void* args[] = {&a, &force_exact};
    LSQ_CUDA_TRY(cudaLaunchKernel(kpass, dim3(G), dim3(pass_threads), args, smem, s));
    if (count) lsq_count_launch();
    return LSQ_OK;
  };
  // phase timers (opts.profile_phases): events around each kernel of the iteration, no graph
  const bool prof = o.profile_phases != 0;
  double ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  cudaEvent_t pe[7];
  if (prof)
    for (auto& e : pe) LSQ_CUDA_TRY(cudaEventCreate(&e));
  // (LSQ_LAUNCH_CHECK counts the launch; in the captured iteration the replays are counted)
#define ITER_CHECK()                                               \
  do {                                                             \
    if (cudaGetLastError() != cudaSuccess) return LSQ_ERR_CUDA;    \
    if (timed) lsq_count_launch();                                 \
  } while (0)
  cudaGraphConditionalHandle cond = 0;
  auto iteration = [&](bool timed) -> lsq_status {
    if (timed) cudaEventRecord(pe[0], s);
    lsq_status r = launch_pass(0, timed);
    if (r != LSQ_OK) return r;
    if (timed) cudaEventRecord(pe[1], s);
    bupdate_kernel<<<nbk, BT, 0, s>>>(a);
    ITER_CHECK();
    if (timed) cudaEventRecord(pe[2], s);
    bprec_kernel<1><<<nbk, BT, 0, s>>>(a);
    ITER_CHECK();
    if (timed) cudaEventRecord(pe[3], s);
    bprec_kernel<2><<<nbk, BT, 0, s>>>(a);
    ITER_CHECK();
    if (timed) cudaEventRecord(pe[4], s);
    bdir_kernel<<<gblk, BT, 0, s>>>(a);
    ITER_CHECK();
    btick_kernel<<<1, 1, 0, s>>>(a, cond, timed ? 0 : 1);
    ITER_CHECK();
    if (timed) cudaEventRecord(pe[5], s);
    return LSQ_OK;
  };

#undef ITER_CHECK
  cudaEvent_t e3;
  LSQ_CUDA_TRY(cudaEventCreate(&e3));
  cudaEventRecord(e1, s);
  // ---- set-up: r0, z0, p0 and the stopping rule at x0
  if (mixed) binit_kernel<true><<<gblk, BT, 0, s>>>(a);
  else binit_kernel<false><<<gblk, BT, 0, s>>>(a);
  LSQ_LAUNCH_CHECK();
  int passes = 0, exact_passes = 0;
  if (!o.x0_zero) {
    st = launch_pass(1, true);
    if (st != LSQ_OK) return st;
    ++passes;
    ++exact_passes;
    LSQ_CUDA_TRY(cudaMemsetAsync(a.qhead, 0, sizeof(int), s));
    if (mixed) bresid_kernel<true><<<gblk, BT, 0, s>>>(a);
    else bresid_kernel<false><<<gblk, BT, 0, s>>>(a);
    LSQ_LAUNCH_CHECK();
  }
  bprec_kernel<1><<<nbk, BT, 0, s>>>(a);
  LSQ_LAUNCH_CHECK();
  bprec_kernel<2><<<nbk, BT, 0, s>>>(a);
  LSQ_LAUNCH_CHECK();
  binitdir_kernel<<<gblk, BT, 0, s>>>(a);
  LSQ_LAUNCH_CHECK();

  // ---- autotuner: on the first batch of this shape on this device, one timed pass (after a
  // warm-up pass) of iteration 0 at each candidate chunk size and pass grid; the fastest is kept
  // for the process.  A pass only writes its partial sums (the iteration's own pass rewrites
  // them) and takes chunks from the iteration's queue head, which is reset after each trial.
  int tuned = 0;
  if (maxit > 0 && (plans.size() > 1 || grid_cand.size() > 1)) {
    const uint64_t sig = batch_signature(ctx->device, probs, nprob, dtype, mixed);
    TunedPass tp{plans[0].elems, grid_cand[0]};
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      auto f = g_tuned.find(sig);
      if (f != g_tuned.end()) {
        tp = f->second;
        have = true;
      }
    }
    if (!have) {
      cudaEvent_t t0, t1;
      LSQ_CUDA_TRY(cudaEventCreate(&t0));
      LSQ_CUDA_TRY(cudaEventCreate(&t1));
      float best = 1e30f;
      for (const ChunkPlan& pl : plans) {
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));  // no pass still reads the tables being replaced
        st = upload_plan(pl);
        if (st != LSQ_OK) return st;
        a.nchunks = (int)pl.chunks.size();
        for (int g : grid_cand) {
          G = g;
          for (int rep = 0; rep < 2; ++rep) {
            LSQ_CUDA_TRY(cudaMemsetAsync(a.qhead, 0, sizeof(int), s));
            if (rep == 1) LSQ_CUDA_TRY(cudaEventRecord(t0, s));
            st = launch_pass(0, true);
            if (st != LSQ_OK) return st;
            if (rep == 1) LSQ_CUDA_TRY(cudaEventRecord(t1, s));
          }
          LSQ_CUDA_TRY(cudaEventSynchronize(t1));
          float ms = 0.f;
          cudaEventElapsedTime(&ms, t0, t1);
          if (ms < best) {
            best = ms;
            tp = TunedPass{pl.elems, g};
          }
        }
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      std::lock_guard<std::mutex> lk(g_tuned_mu);
      g_tuned[sig] = tp;
      tuned = 1;
    }
    // the chosen plan and grid for the iterations
    for (const ChunkPlan& pl : plans)
      if (pl.elems == tp.elems) plan = &pl;
    G = tp.grid;
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    st = upload_plan(*plan);
    if (st != LSQ_OK) return st;
    a.nchunks = (int)plan->chunks.size();
    for (int p = 0; p < nprob; ++p) {
      hp[p].chunk0 = plan->chunk0[p];
      hp[p].nchunk = plan->nchunk[p];
    }
    LSQ_CUDA_TRY(cudaMemcpy(base + o_probs, hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice));
    LSQ_CUDA_TRY(cudaMemsetAsync(a.qhead, 0, sizeof(int), s));
  }

  // ---- iterations: one CUDA graph whose conditional WHILE node runs the iteration body (pass,
  // update, the two triangular products, directions, tick) until no problem is active or maxit
  // iterations have run -- the tick kernel decides on the device, so the whole loop is one
  // launch with no host round trip.  With opts.profile_phases the host drives the iterations
  // one by one instead, timing each kernel.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int it = 0;
  if (!prof && maxit > 0) {
    LSQ_CUDA_TRY(cudaGraphCreate(&graph, 0));
    auto fail = [&](lsq_status r) {
      if (graph) cudaGraphDestroy(graph);
      (void)cudaGetLastError();
      return r;
    };
    if (cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      return fail(LSQ_ERR_CUDA);
    // the first node sets the condition of iteration 0
    cudaGraphNode_t kn;
    cudaKernelNodeParams kp = {};
    void* cargs[] = {&a, &cond};
    kp.func = (void*)bcond_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = cargs;
    if (cudaGraphAddKernelNode(&kn, graph, nullptr, 0, &kp) != cudaSuccess) return fail(LSQ_ERR_CUDA);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn;
    if (cudaGraphAddNode(&wn, graph, &kn, nullptr, 1, &cp) != cudaSuccess) return fail(LSQ_ERR_CUDA);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // the body is captured on the context's own non-blocking stream (the caller's may be the
    // legacy default stream, which cannot be captured); the graph runs on the caller's stream
    if (!ctx->capture && cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking) != cudaSuccess)
      return fail(LSQ_ERR_CUDA);
    const cudaStream_t s_user = s;
    s = ctx->capture;
    if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      s = s_user;
      return fail(LSQ_ERR_CUDA);
    }
    st = iteration(false);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &captured);
    s = s_user;
    if (st != LSQ_OK || ce != cudaSuccess) return fail(st != LSQ_OK ? st : LSQ_ERR_CUDA);
    if (cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) return fail(LSQ_ERR_CUDA);
    LSQ_CUDA_TRY(cudaGraphLaunch(gexec, s));
  } else if (prof) {
    int* host_cnt = ctx->host_status + 14;
    while (it < maxit) {
      // active problems for iteration it: cnt[it % 3]
      LSQ_CUDA_TRY(cudaMemcpyAsync(host_cnt, a.cnt + it % 3, sizeof(int), cudaMemcpyDeviceToHost, s));
      LSQ_CUDA_TRY(cudaStreamSynchronize(s));
      if (*host_cnt == 0) break;
      st = iteration(true);
      if (st != LSQ_OK) return st;
      LSQ_CUDA_TRY(cudaStreamSynchronize(s));
      float t = 0.f;
      for (int q = 0; q < 5; ++q) {
        cudaEventElapsedTime(&t, pe[q], pe[q + 1]);
        ph[q] += t;
      }
      ++it;
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (prof)
    for (auto& e : pe) cudaEventDestroy(e);
  cudaEventRecord(e3, s);
  cudaEventRecord(ctx->ev1, s);
  LSQ_CUDA_TRY(cudaStreamSynchronize(s));
  float ms_solve = 0.f, ms_total = 0.f;
  cudaEventElapsedTime(&ms_solve, e1, e3);
  cudaEventElapsedTime(&ms_total, ctx->ev0, ctx->ev1);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  cudaEventDestroy(e3);
  int hdr[24];
  LSQ_CUDA_TRY(cudaMemcpy(hdr, ctl, sizeof(hdr), cudaMemcpyDeviceToHost));
  passes += hdr[16];
  exact_passes += mixed ? hdr[17] : hdr[16];
  // the device-driven loop launched the condition kernel and six kernels per iteration it ran
  if (!prof && maxit > 0)
    for (int q = 0; q < 1 + 6 * hdr[16]; ++q) lsq_count_launch();
  const int errc = hdr[20];
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
    info->passes = passes;
    info->exact_passes = exact_passes;
    info->ms_total = ms_total;
    info->ms_sketch = ms_sketch;
    info->ms_factor = ms_factor;
    info->ms_solve = ms_solve;
    for (int q = 0; q < 8; ++q) info->ms_phase[q] = q < 5 ? ph[q] : 0.0;
    info->pass_chunk_elems = plan->elems;
    info->pass_grid = G;
    info->tuned = tuned;
  }
  return overall;
}
