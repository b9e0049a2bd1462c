// factor.cu -- H_S = (SA)^T (SA) = R^T R and W = R^{-1} (Section 1, PCG paragraph;
// Section 6: a factorisation of H_S costs O(m d^2) and makes each solve with H_S O(d^2)).
//
// (1) Gram G = (SA)^T (SA) in FP64: split-K tiles over the upper triangle, fixed-order
//     reduction, padded to dp = 32 ceil(d/32) with an identity block.
// (2) One cooperative kernel: right-looking blocked Cholesky with 32 x 32 blocks
//     (diagonal block on one CTA, panel and trailing update as 32 x 8 tile tasks over
//     the whole grid), then W = R^{-1} by recursive doubling over a binary tree of the
//     diagonal blocks: for R = [[A, B], [0, C]], R^{-1} = [[A^-1, -A^-1 B C^-1], [0, C^-1]].
//     Phases are separated by bounded grid barriers.
#include <algorithm>
#include <type_traits>
#include <math.h>
#include <vector>

#include "apass.cuh"
#include "common.cuh"

namespace {

constexpr int TB = 64, TK = 16;

// One TK-row step of a 64 x 64 Gram tile in double-FP32 (DF): each thread's 4 x 4 outputs are
// (head, tail) FP32 pairs; the operands were split into a 21-bit head and the FP32 rounding of
// the rest (about 45 significant bits), products are exact through an FMA (TwoProduct) and the
// sums are carried with TwoSum (Dekker 1971; Knuth) -- on the FP32 pipe, which does ~70x the
// FP64 pipe's FMA rate on this part.
__device__ __forceinline__ void df_gram_step(const float2 (*Xa)[TB], const float2 (*Xb)[TB], int ty, int tx,
                                             float (&ah)[4][4], float (&al)[4][4]) {
#pragma unroll 4
  for (int k = 0; k < TK; ++k) {
    float2 x[4], y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = Xa[k][ty + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = Xb[k][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) lsq_apass::df_fma(x[i].x, x[i].y, y[j].x, y[j].y, ah[i][j], al[i][j]);
  }
}

__device__ __forceinline__ float2 df_split(double v) {
  float h, t;
  lsq_apass::split_df(v, h, t);
  return make_float2(h, t);
}

// part[split][dp][dp] (upper tiles only) = sum over the split's rows of SA^T SA, in FP64 or,
// with DF, in double-FP32
template <bool DF>
__global__ void __launch_bounds__(256) gram_kernel(const double* __restrict__ SA, int m, int d, int dp,
                                                   int rows_per_split, const int2* __restrict__ tiles,
                                                   double* __restrict__ part) {
  using E = typename std::conditional<DF, float2, double>::type;
  __shared__ E Xa[TK][TB];
  __shared__ E Xb[TK][TB];
  const int2 tl = tiles[blockIdx.x];
  const int a0 = tl.x * TB, b0 = tl.y * TB;
  const int r_begin = blockIdx.y * rows_per_split;
  const int r_end = min(m, r_begin + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  float ah[4][4] = {}, al[4][4] = {};
  for (int r0 = r_begin; r0 < r_end; r0 += TK) {
    for (int e = threadIdx.x; e < TK * TB; e += 256) {
      const int k = e / TB, c = e % TB;
      const int r = r0 + k;
      const double va = (r < r_end && a0 + c < d) ? SA[(int64_t)r * d + a0 + c] : 0.0;
      const double vb = (r < r_end && b0 + c < d) ? SA[(int64_t)r * d + b0 + c] : 0.0;
      if constexpr (DF) {
        Xa[k][c] = df_split(va);
        Xb[k][c] = df_split(vb);
      } else {
        Xa[k][c] = va;
        Xb[k][c] = vb;
      }
    }
    __syncthreads();
    if constexpr (DF) {
      df_gram_step(Xa, Xb, ty, tx, ah, al);
    } else {
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        double x[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = Xa[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = Xb[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * dp * dp;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      const double v = DF ? (double)ah[i][j] + (double)al[i][j] : acc[i][j];
      if (a < dp && b < dp) out[(int64_t)a * dp + b] = v;
    }
}

// G = sum of the splits on the upper tiles, mirrored; identity on the padded diagonal
__global__ void gram_reduce_kernel(const double* __restrict__ part, int splits, int d, int dp, double* __restrict__ G) {
  const int64_t total = (int64_t)dp * dp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / dp), b = (int)(e % dp);
    double v;
    if (a >= d || b >= d) {
      v = (a == b) ? 1.0 : 0.0;
    } else {
      const int lo = min(a, b), hi = max(a, b);
      // the tile holding (lo, hi) is an upper tile (tile row <= tile column)
      const int64_t idx = (int64_t)lo * dp + hi;
      const bool upper_tile = (lo / TB) <= (hi / TB);
      const int64_t src = upper_tile ? idx : (int64_t)hi * dp + lo;
      v = 0.0;
      for (int g = 0; g < splits; ++g) v += part[(int64_t)g * dp * dp + src];
    }
    G[e] = v;
  }
}

// ------------------------------------------------------------------------------------
// 32 x 8 tile task: out(r, c) = (acc ? out(r, c) : 0) + alpha * sum_k X(r, k) Y(k, c),
// X(r, k) = Xm[r*ld + k] (or Xm[k*ld + r] when transX), Y(k, c) = Ym[k*ld + c], k < K.
// ------------------------------------------------------------------------------------
struct TileSmem {
  double X[2][32][33];
  double Y[2][32][8];
};

// the diagonal-block routines' arrays
struct DiagSmem {
  double a[32][33], b[32][33], c[32][33];
  double rinv[32], pinv[32];
  int bad;
};

// one shared workspace: a CTA runs one of these routines at a time
union FactorSmem {
  TileSmem tile;
  DiagSmem diag;
};

// 8-byte asynchronous copies global -> shared (the thread does not wait for the data)
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tile_load(TileSmem& sm, int buf, const double* Xm, bool transX, const double* Ym,
                                          int k0, int ld) {
  for (int e = threadIdx.x; e < 1024; e += 256) {
    if (transX) {
      const int kk = e >> 5, rr = e & 31;
      cp_async8(&sm.X[buf][rr][kk], Xm + (int64_t)(k0 + kk) * ld + rr);
    } else {
      const int rr = e >> 5, kk = e & 31;
      cp_async8(&sm.X[buf][rr][kk], Xm + (int64_t)rr * ld + k0 + kk);
    }
  }
  const int kk = threadIdx.x >> 3, cc = threadIdx.x & 7;
  cp_async8(&sm.Y[buf][kk][cc], Ym + (int64_t)(k0 + kk) * ld + cc);
  cp_async_commit();
}

// the next 32-deep block is loaded while the current one is multiplied
__device__ void tile_task(TileSmem& sm, double* out, const double* Xm, bool transX, const double* Ym, int K, int ld,
                          double alpha, bool acc) {
  const int r = threadIdx.x >> 3, c = threadIdx.x & 7;
  double sum = 0.0;
  tile_load(sm, 0, Xm, transX, Ym, 0, ld);
  cp_async_wait_all();
  __syncthreads();
  for (int k0 = 0, buf = 0; k0 < K; k0 += 32, buf ^= 1) {
    if (k0 + 32 < K) tile_load(sm, buf ^ 1, Xm, transX, Ym, k0 + 32, ld);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) sum = fma(sm.X[buf][r][kk], sm.Y[buf][kk][c], sum);
    cp_async_wait_all();
    __syncthreads();
  }
  double* o = out + (int64_t)r * ld + c;
  *o = (acc ? *o : 0.0) + alpha * sum;
}

// Upper-triangle task index e -> (a, b), 0 <= a <= b, e = b (b + 1) / 2 + a.
__device__ __forceinline__ void tri_decode(int e, int& a, int& b) {
  int bb = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (bb * (bb + 1) / 2 > e) --bb;
  while ((bb + 1) * (bb + 2) / 2 <= e) ++bb;
  b = bb;
  a = e - bb * (bb + 1) / 2;
}

// Cholesky of one 32 x 32 diagonal block by the whole CTA: R into Rkk, and 1 / R[i][i] into the
// block's own diagonal in G (the block is not read again).  FP64 instructions are costly on
// this part (a warp instruction holds a sub-partition's FP64 unit for ~70 cycles whatever its
// active lanes), so the factorisation is right-looking with the live entries of each step
// packed densely onto threads, one barrier per step:
//   step j: R[j][l] = G[j][l] / sqrt(G[j][j]) and G[i][l] -= G[j][i] G[j][l] / G[j][j] for
//   j < i <= l; the thread that updates G[j+1][j+1] also takes its reciprocal square root, so
//   the next pivot is ready at the barrier.
// Sets *err to LSQ_ERR_RANK on a non-positive or non-finite pivot.
__device__ void diag_chol(DiagSmem& sm, double* Gkk, double* Rkk, int ld, int* err) {
  double (*Gs)[33] = sm.a;
  double (*Rs)[33] = sm.b;
  double* rinv = sm.rinv;
  double* pinv = sm.pinv;
  int& bad = sm.bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < 1024; e += nt) {
    Gs[e >> 5][e & 31] = Gkk[(int64_t)(e >> 5) * ld + (e & 31)];
    Rs[e >> 5][e & 31] = 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  if (tid == 0) {
    const double g = Gs[0][0];
    if (!(g > 0.0) || !isfinite(g)) bad = 1;
    const double r = rsqrt(g);
    rinv[0] = r;
    pinv[0] = r * r;
  }
  __syncthreads();
  for (int j = 0; j < 32; ++j) {
    const int S = 31 - j, T = S * (S + 1) / 2;
    const double ri = rinv[j], pv = pinv[j];
    for (int e = tid; e < T + 32 - j; e += nt) {
      if (e < T) {
        int a, b;
        tri_decode(e, a, b);
        const int i = j + 1 + a, l = j + 1 + b;
        const double g = fma(-(Gs[j][i] * pv), Gs[j][l], Gs[i][l]);
        Gs[i][l] = g;
        if (e == 0) {  // (i, l) = (j + 1, j + 1): the next pivot
          if (!(g > 0.0) || !isfinite(g)) bad = 1;
          const double r = rsqrt(g);
          rinv[j + 1] = r;
          pinv[j + 1] = r * r;
        }
      } else {
        const int l = j + (e - T);
        Rs[j][l] = Gs[j][l] * ri;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < 1024; e += nt) Rkk[(int64_t)(e >> 5) * ld + (e & 31)] = Rs[e >> 5][e & 31];
  if (tid < 32) Gkk[(int64_t)tid * ld + tid] = rinv[tid];
  if (tid == 0 && bad) atomicCAS(err, 0, (int)LSQ_ERR_RANK);
  __syncthreads();
}

// W = R^{-1} of one 32 x 32 upper triangular block (Rkk; 1 / R[i][i] on the block's diagonal in
// G), right-looking from the bottom row, one barrier per step:
//   W[i][l] = (delta_il - S[i][l]) / R[i][i] for l >= i, then S[k][l] += R[k][i] W[i][l], k < i <= l.
__device__ void diag_inv(DiagSmem& sm, const double* Gkk, const double* Rkk, double* Wkk, int ld) {
  double (*Rs)[33] = sm.a;
  double (*Ss)[33] = sm.b;
  double (*Ws)[33] = sm.c;
  double* rinv = sm.rinv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < 1024; e += nt) {
    Rs[e >> 5][e & 31] = Rkk[(int64_t)(e >> 5) * ld + (e & 31)];
    Ss[e >> 5][e & 31] = 0.0;
    Ws[e >> 5][e & 31] = 0.0;
  }
  if (tid < 32) rinv[tid] = Gkk[(int64_t)tid * ld + tid];
  __syncthreads();
  for (int i = 31; i >= 0; --i) {
    const int w = 32 - i;
    const double ri = rinv[i];
    for (int e = tid; e < (i + 1) * w; e += nt) {
      const int k = e / w, l = i + e % w;
      const double wil = ((i == l ? 1.0 : 0.0) - Ss[i][l]) * ri;
      if (k == i) Ws[i][l] = wil;
      else Ss[k][l] = fma(Rs[k][i], wil, Ss[k][l]);
    }
    __syncthreads();
  }
  for (int e = tid; e < 1024; e += nt) Wkk[(int64_t)(e >> 5) * ld + (e & 31)] = Ws[e >> 5][e & 31];
  __syncthreads();
}

// 32 x 8 panel task: out = R^{-T} Gt (R = Rkk upper, 1 / R[i][i] on the diagonal of Gkk) by
// forward substitution: warp c solves column c, lane i keeps row i's running value, and each
// step's new unknown is broadcast by a shuffle (no CTA barrier inside the solve).
__device__ void trsm_task(TileSmem& sm, double* out, const double* Rkk, const double* Gt, const double* Gkk, int ld) {
  const int tid = threadIdx.x, lane = tid & 31, c = tid >> 5;
  for (int e = tid; e < 1024; e += blockDim.x) sm.X[0][e >> 5][e & 31] = Rkk[(int64_t)(e >> 5) * ld + (e & 31)];
  __syncthreads();
  if (c < 8) {
    double acc = Gt[(int64_t)lane * ld + c];
    const double di = Gkk[(int64_t)lane * ld + lane];
    double x = 0.0;
#pragma unroll 4
    for (int p = 0; p < 32; ++p) {
      const double xp = __shfl_sync(0xffffffffu, acc * di, p);
      if (lane == p) x = xp;
      if (lane > p) acc = fma(-sm.X[0][p][lane], xp, acc);
    }
    out[(int64_t)lane * ld + c] = x;
  }
  __syncthreads();
}

// The blocked Cholesky and inverse on a group of `nb` CTAs (this CTA has rank `rank`) that
// synchronise through `bar`; the single-problem launch uses the whole grid as one group.
__device__ void chol_inv_body(double* __restrict__ G, double* __restrict__ Rf, double* __restrict__ Wf,
                              double* __restrict__ Tb, int nblk, const int4* __restrict__ nodes,
                              const int* __restrict__ level_start, int nlevels, unsigned* bar, unsigned nb,
                              unsigned rank, int* err) {
  __shared__ FactorSmem fsm;
  TileSmem& sm = fsm.tile;
  const int dp = nblk * 32;
  // the group's barriers: a count that only grows (bar[2..3], zeroed before the launch)
  unsigned long long bar_target = 0;
  auto gsync = [&]() -> int {
    return grid_sync_count(reinterpret_cast<unsigned long long*>(bar + 2), bar_target, nb, err);
  };
  // Look-ahead: CTA 0 applies the trailing update to the next diagonal block first and
  // factors it at once, while the other CTAs update the rest of the trailing matrix; each
  // panel then needs two grid barriers.
  if (rank == 0) diag_chol(fsm.diag, G, Rf, dp, err);
  if (gsync()) return;
  for (int k = 0; k < nblk; ++k) {
    const int64_t kk = (int64_t)k * 32;
    const int rest = nblk - 1 - k;
    // panel: R[k][j] = R[k][k]^{-T} G[k][j] (forward substitution; the inverses of the
    // diagonal blocks are taken after the factorisation, off this chain)
    for (int task = rank; task < rest * 4; task += nb) {
      const int j = k + 1 + task / 4, q = task % 4;
      const int64_t col = (int64_t)j * 32 + q * 8;
      trsm_task(sm, Rf + kk * dp + col, Rf + kk * dp + kk, G + kk * dp + col, G + kk * dp + kk, dp);
    }
    if (gsync()) return;
    if (rest == 0) break;
    // trailing update: G[i][j] -= R[k][i]^T R[k][j], k < i <= j; pair 0 is the next
    // diagonal block (k+1, k+1)
    const int pairs = rest * (rest + 1) / 2;
    const int64_t k1 = (int64_t)(k + 1) * 32;
    // the next diagonal block's update is split over `nd` CTAs (one 32 x 8 tile each: it is
    // 32^3 FP64 FMAs, ~9 us on one SM); CTAs 1 .. nd-1 count themselves done on bar[4] and
    // CTA 0 waits for them (bounded) before it factors the block
    const unsigned nd = nb >= 4 ? 4u : 1u;
    if (rank < nd) {
      for (unsigned q = rank; q < 4; q += nd)
        tile_task(sm, G + k1 * dp + k1 + q * 8, Rf + kk * dp + k1, true, Rf + kk * dp + k1 + q * 8, 32, dp, -1.0,
                  true);
      __syncthreads();
      if (rank > 0 && threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar + 4, 1u);
      }
    }
    if (rank == 0) {
      if (nd > 1 && threadIdx.x == 0) {
        const unsigned target = (unsigned)(k + 1) * (nd - 1);
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire_u32(bar + 4) < target) {
          if (*(volatile int*)err != 0) break;
          if (++spins > LSQ_SPIN_LIMIT || global_ns() - t0 > LSQ_WAIT_NS) {
            atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
      }
      __syncthreads();
      if (*(volatile int*)err == 0) diag_chol(fsm.diag, G + k1 * dp + k1, Rf + k1 * dp + k1, dp, err);
    }
    const int others = nb > 1 ? (int)nb - 1 : 1;
    const int first = nb > 1 ? (int)rank - 1 : 0;
    if (nb == 1 || rank > 0) {
      for (int task = 4 + first; task < pairs * 4; task += others) {
        int p = task / 4;
        const int q = task % 4;
        int i = 0;
        while (p >= rest - i) { p -= rest - i; ++i; }
        const int bi = k + 1 + i, bj = bi + p;
        const int64_t col = (int64_t)bj * 32 + q * 8;
        tile_task(sm, G + (int64_t)bi * 32 * dp + col, Rf + kk * dp + (int64_t)bi * 32, true, Rf + kk * dp + col, 32,
                  dp, -1.0, true);
      }
    }
    if (gsync()) return;
  }
  // the inverses of the diagonal blocks, all at once
  for (int k = (int)rank; k < nblk; k += (int)nb) {
    const int64_t kk = (int64_t)k * 32;
    diag_inv(fsm.diag, G + kk * dp + kk, Rf + kk * dp + kk, Wf + kk * dp + kk, dp);
  }
  if (gsync()) return;
  // W = R^{-1}: merge sibling blocks bottom-up
  for (int lev = 0; lev < nlevels; ++lev) {
    const int n0 = level_start[lev], n1 = level_start[lev + 1];
    // phase 1: T[a:mid, mid:b] = R[a:mid, mid:b] W[mid:b, mid:b]
    int base = 0;
    for (int nd = n0; nd < n1; ++nd) {
      const int4 t = nodes[nd];
      const int rows = t.y - t.x, cols4 = (t.z - t.y) * 4;
      for (int task = (int)((rank + nb - (unsigned)(base % nb)) % nb); task < rows * cols4; task += nb) {
        const int rb = task / cols4, cs = task % cols4;
        const int64_t r0 = (int64_t)(t.x + rb) * 32, c0 = (int64_t)t.y * 32 + cs * 8;
        tile_task(sm, Tb + r0 * dp + c0, Rf + r0 * dp + (int64_t)t.y * 32, false, Wf + (int64_t)t.y * 32 * dp + c0,
                  (t.z - t.y) * 32, dp, 1.0, false);
      }
      base += rows * cols4;
    }
    if (gsync()) return;
    // phase 2: W[a:mid, mid:b] = -W[a:mid, a:mid] T[a:mid, mid:b]
    base = 0;
    for (int nd = n0; nd < n1; ++nd) {
      const int4 t = nodes[nd];
      const int rows = t.y - t.x, cols4 = (t.z - t.y) * 4;
      for (int task = (int)((rank + nb - (unsigned)(base % nb)) % nb); task < rows * cols4; task += nb) {
        const int rb = task / cols4, cs = task % cols4;
        const int64_t r0 = (int64_t)(t.x + rb) * 32, c0 = (int64_t)t.y * 32 + cs * 8;
        tile_task(sm, Wf + r0 * dp + c0, Wf + r0 * dp + (int64_t)t.x * 32, false, Tb + (int64_t)t.x * 32 * dp + c0,
                  (t.y - t.x) * 32, dp, -1.0, false);
      }
      base += rows * cols4;
    }
    if (gsync()) return;
  }
}

__global__ void __launch_bounds__(256, 2) chol_inv_kernel(double* __restrict__ G, double* __restrict__ Rf,
                                                       double* __restrict__ Wf, double* __restrict__ Tb, int nblk,
                                                       const int4* __restrict__ nodes, const int* __restrict__ level_start,
                                                       int nlevels, unsigned* bar, int* err) {
  chol_inv_body(G, Rf, Wf, Tb, nblk, nodes, level_start, nlevels, bar, gridDim.x, blockIdx.x, err);
}

__global__ void copy_out_kernel(const double* __restrict__ Rf, const double* __restrict__ Wf, int d, int dp,
                                double* __restrict__ R, double* __restrict__ W) {
  const int64_t total = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / d), b = (int)(e % d);
    const bool up = b >= a;
    R[e] = up ? Rf[(int64_t)a * dp + b] : 0.0;
    W[e] = up ? Wf[(int64_t)a * dp + b] : 0.0;
  }
}

static void build_tree(int a, int b, int depth, std::vector<std::vector<int4>>& by_depth) {
  if (b - a <= 1) return;
  const int mid = a + (b - a) / 2;
  build_tree(a, mid, depth + 1, by_depth);
  build_tree(mid, b, depth + 1, by_depth);
  if ((int)by_depth.size() <= depth) by_depth.resize(depth + 1);
  by_depth[depth].push_back(make_int4(a, mid, b, 0));
}

}  // namespace

extern "C" lsq_status lsq_factor(lsq_ctx* ctx, const double* SA, int64_t m, int64_t d, double* R, double* W) {
  return lsq_factor_ex(ctx, SA, m, d, R, W, LSQ_PREC_F64);
}

extern "C" lsq_status lsq_factor_ex(lsq_ctx* ctx, const double* SA, int64_t m, int64_t d, double* R, double* W,
                                    int32_t gram_precision) {
  if (!ctx || !SA || !R || !W) return LSQ_ERR_ARG;
  if (gram_precision != LSQ_PREC_F64 && gram_precision != LSQ_PREC_MIXED) return LSQ_ERR_ARG;
  if (d < 1 || d > LSQ_MAX_D || m < d || m > (1ll << 31) - 1) return LSQ_ERR_ARG;
  const int di = (int)d, mi = (int)m;
  const int nblk = (di + 31) / 32, dp = nblk * 32;

  // Gram tiles (upper triangle of 64 x 64 tiles) and split-K
  const int nt = (dp + TB - 1) / TB;
  std::vector<int2> tiles;
  for (int a = 0; a < nt; ++a)
    for (int b = a; b < nt; ++b) tiles.push_back(make_int2(a, b));
  int splits = std::max(1, (2 * ctx->sm_count + (int)tiles.size() - 1) / (int)tiles.size());
  splits = std::min(splits, std::max(1, mi / 64));
  splits = std::min(splits, std::max(1, (int)(((int64_t)128 << 20) / ((int64_t)dp * dp * 8))));
  const int rows_per_split = ((mi + splits - 1) / splits + TK - 1) / TK * TK;
  splits = (mi + rows_per_split - 1) / rows_per_split;

  // inverse tree levels, deepest first
  std::vector<std::vector<int4>> by_depth;
  build_tree(0, nblk, 0, by_depth);
  std::vector<int4> nodes;
  std::vector<int> level_start;
  for (int dep = (int)by_depth.size() - 1; dep >= 0; --dep) {
    level_start.push_back((int)nodes.size());
    for (auto& t : by_depth[dep]) nodes.push_back(t);
  }
  level_start.push_back((int)nodes.size());
  const int nlevels = (int)level_start.size() - 1;

  const size_t mat = (size_t)dp * dp;
  size_t need = lsq_align256((size_t)splits * mat * 8) + 4 * lsq_align256(mat * 8) + lsq_align256(tiles.size() * 8) +
                lsq_align256(std::max<size_t>(1, nodes.size()) * 16) + lsq_align256(level_start.size() * 4) +
                lsq_align256(64);
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  double* part = cv.take<double>((size_t)splits * mat);
  double* G = cv.take<double>(mat);
  double* Rf = cv.take<double>(mat);
  double* Wf = cv.take<double>(mat);
  double* Tb = cv.take<double>(mat);
  int2* d_tiles = cv.take<int2>(tiles.size());
  int4* d_nodes = cv.take<int4>(std::max<size_t>(1, nodes.size()));
  int* d_levels = cv.take<int>(level_start.size());
  unsigned* bar = cv.take<unsigned>(16);
  int* err = reinterpret_cast<int*>(bar + 8);
  cudaStream_t s = ctx->stream;

  LSQ_CUDA_TRY(cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  if (!nodes.empty())
    LSQ_CUDA_TRY(cudaMemcpyAsync(d_nodes, nodes.data(), nodes.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  LSQ_CUDA_TRY(cudaMemcpyAsync(d_levels, level_start.data(), level_start.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  LSQ_CUDA_TRY(cudaMemsetAsync(bar, 0, 64, s));
  LSQ_CUDA_TRY(cudaMemsetAsync(Rf, 0, mat * 8, s));
  LSQ_CUDA_TRY(cudaMemsetAsync(Wf, 0, mat * 8, s));

  const dim3 ggrid((unsigned)tiles.size(), (unsigned)splits);
  if (gram_precision == LSQ_PREC_MIXED)
    gram_kernel<true><<<ggrid, 256, 0, s>>>(SA, mi, di, dp, rows_per_split, d_tiles, part);
  else
    gram_kernel<false><<<ggrid, 256, 0, s>>>(SA, mi, di, dp, rows_per_split, d_tiles, part);
  LSQ_LAUNCH_CHECK();
  gram_reduce_kernel<<<std::min(4 * ctx->sm_count, (int)((mat + 255) / 256)), 256, 0, s>>>(part, splits, di, dp, G);
  LSQ_LAUNCH_CHECK();

  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_inv_kernel, 256, 0));
  if (per_sm < 1) return LSQ_ERR_CUDA;
  int grid = std::min(per_sm, 2) * ctx->sm_count;
  const int max_tasks = std::max(4 * nblk * nblk, 8);
  grid = std::max(1, std::min(grid, max_tasks));
  void* args[] = {&G, &Rf, &Wf, &Tb, (void*)&nblk, &d_nodes, &d_levels, (void*)&nlevels, &bar, &err};
  int nblk_v = nblk, nlev_v = nlevels;
  args[4] = &nblk_v;
  args[7] = &nlev_v;
  LSQ_CUDA_TRY(cudaLaunchCooperativeKernel((void*)chol_inv_kernel, dim3(grid), dim3(256), args, 0, s));
  lsq_count_launch();
  copy_out_kernel<<<std::min(4 * ctx->sm_count, (int)((d * d + 255) / 256)), 256, 0, s>>>(Rf, Wf, di, dp, R, W);
  LSQ_LAUNCH_CHECK();
  if (ctx->defer_checks) return lsq_defer_status(ctx, err, 1);  // the rank check, reported later
  LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  LSQ_CUDA_TRY(cudaStreamSynchronize(s));
  const int code = *ctx->host_status;
  if (code == LSQ_ERR_RANK) return LSQ_ERR_RANK;
  if (code != 0) return (lsq_status)code;
  return LSQ_OK;
}

// ------------------------------------------------------------------------------------
// Many factorisations at once (batched solves): one launch for every Gram matrix (a 64 x 64
// tile of one problem per CTA, all rows of its SA; FP64, or double-FP32 under the mixed
// precision), one cooperative launch in which each problem's Cholesky and inverse run on a
// group of CTAs sized by its d^3 with a barrier of its own, one launch writing W and W^T.
// ------------------------------------------------------------------------------------
namespace {

struct GramJob {
  const double* SA;
  double* G;
  int m, d, dp;
};

struct CholJob {
  double *G, *Rf, *Wf, *Tb;
  const int4* nodes;
  const int* level_start;
  int nlevels, nblk, cta0, ncta;
  unsigned* bar;
  int* err;
  double* W;   // d x d output
  double* WT;  // d x d output
  int d;
};

template <bool DF>
__global__ void __launch_bounds__(256) gram_batched_kernel(const GramJob* __restrict__ jobs,
                                                           const int4* __restrict__ units) {
  const int4 u = units[blockIdx.x];
  const GramJob jb = jobs[u.x];
  const int a0 = u.y * TB, b0 = u.z * TB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int d = jb.d, dp = jb.dp;
  double res[4][4];
  if constexpr (!DF) {
    __shared__ double Xa[TK][TB];
    __shared__ double Xb[TK][TB];
    double acc[4][4] = {};
    for (int r0 = 0; r0 < jb.m; r0 += TK) {
      for (int e = threadIdx.x; e < TK * TB; e += 256) {
        const int k = e / TB, c = e % TB;
        const int r = r0 + k;
        Xa[k][c] = (r < jb.m && a0 + c < d) ? jb.SA[(int64_t)r * d + a0 + c] : 0.0;
        Xb[k][c] = (r < jb.m && b0 + c < d) ? jb.SA[(int64_t)r * d + b0 + c] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        double x[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = Xa[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = Xb[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) res[i][j] = acc[i][j];
  } else {
    // double-FP32 (df_gram_step)
    __shared__ float2 Xa[TK][TB];
    __shared__ float2 Xb[TK][TB];
    float ah[4][4] = {}, al[4][4] = {};
    for (int r0 = 0; r0 < jb.m; r0 += TK) {
      for (int e = threadIdx.x; e < TK * TB; e += 256) {
        const int k = e / TB, c = e % TB;
        const int r = r0 + k;
        Xa[k][c] = df_split((r < jb.m && a0 + c < d) ? jb.SA[(int64_t)r * d + a0 + c] : 0.0);
        Xb[k][c] = df_split((r < jb.m && b0 + c < d) ? jb.SA[(int64_t)r * d + b0 + c] : 0.0);
      }
      __syncthreads();
      df_gram_step(Xa, Xb, ty, tx, ah, al);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) res[i][j] = (double)ah[i][j] + (double)al[i][j];
  }
  // the tile and its mirror; the padding of the last block is the identity
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < dp && b < dp) {
        const double v = (a < d && b < d) ? res[i][j] : (a == b ? 1.0 : 0.0);
        jb.G[(int64_t)a * dp + b] = v;
        jb.G[(int64_t)b * dp + a] = v;
      }
    }
}

__global__ void __launch_bounds__(256) chol_inv_batched_kernel(const CholJob* __restrict__ jobs,
                                                               const int* __restrict__ cta_job) {
  const CholJob& j = jobs[cta_job[blockIdx.x]];
  chol_inv_body(j.G, j.Rf, j.Wf, j.Tb, j.nblk, j.nodes, j.level_start, j.nlevels, j.bar, (unsigned)j.ncta,
                blockIdx.x - (unsigned)j.cta0, j.err);
}

// W (upper part of Wf) and W^T for problem blockIdx.y; rows strided over blockIdx.x
__global__ void w_out_batched_kernel(const CholJob* __restrict__ jobs) {
  const CholJob& j = jobs[blockIdx.y];
  const int d = j.d, dp = j.nblk * 32;
  for (int i = blockIdx.x; i < d; i += gridDim.x) {
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
      const double w = c >= i ? j.Wf[(int64_t)i * dp + c] : 0.0;
      j.W[(int64_t)i * d + c] = w;
      j.WT[(int64_t)c * d + i] = w;
    }
  }
}

}  // namespace

// Factors the sketches SA_p (device, m_p x d_p) of nprob problems: W_p = R_p^{-1} and its
// transpose into the caller's buffers; status_out[p] = LSQ_OK or LSQ_ERR_RANK (host array).
lsq_status lsq_factor_batched(lsq_ctx* ctx, int nprob, const double* const* SA, const int* m, const int* d,
                              double* const* W, double* const* WT, bool df_gram, int* status_out) {
  cudaStream_t s = ctx->stream;
  // the scratch arena is rewritten below by synchronous copies: earlier work must be done
  LSQ_CUDA_TRY(cudaStreamSynchronize(s));
  // trees of the inverse, one per distinct block count
  std::vector<int4> nodes;
  std::vector<int> levels;
  std::vector<int> tree_node0(33, -1), tree_lev0(33, -1), tree_nlev(33, 0);
  for (int p = 0; p < nprob; ++p) {
    const int nblk = (d[p] + 31) / 32;
    if (tree_node0[nblk] >= 0) continue;
    std::vector<std::vector<int4>> by_depth;
    build_tree(0, nblk, 0, by_depth);
    tree_node0[nblk] = (int)nodes.size();
    tree_lev0[nblk] = (int)levels.size();
    const int base = (int)nodes.size();
    for (int dep = (int)by_depth.size() - 1; dep >= 0; --dep) {
      levels.push_back((int)nodes.size() - base);
      for (auto& t : by_depth[dep]) nodes.push_back(t);
    }
    levels.push_back((int)nodes.size() - base);
    tree_nlev[nblk] = (int)by_depth.size();
  }
  // Gram units and the scratch layout
  std::vector<int4> units;
  size_t mats = 0;
  for (int p = 0; p < nprob; ++p) {
    const int dp = ((d[p] + 31) / 32) * 32, nt = (dp + TB - 1) / TB;
    for (int a = 0; a < nt; ++a)
      for (int b = a; b < nt; ++b) units.push_back(make_int4(p, a, b, 0));
    mats += lsq_align256((size_t)dp * dp * 8);
  }
  // CTA groups of the cooperative launch: sizes by d^3, at least one CTA each, problems in waves
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_inv_batched_kernel, 256, 0));
  if (per_sm < 1) return LSQ_ERR_CUDA;
  const int cta_per_sm = std::min(per_sm, 4);
  const int gmax = cta_per_sm * ctx->sm_count;
  size_t need = 4 * mats + lsq_align256(sizeof(GramJob) * nprob) + lsq_align256(sizeof(CholJob) * nprob) +
                lsq_align256(sizeof(int4) * units.size()) + lsq_align256(sizeof(int4) * std::max<size_t>(1, nodes.size())) +
                lsq_align256(sizeof(int) * levels.size()) + lsq_align256(sizeof(int) * gmax) +
                lsq_align256((size_t)nprob * 64);
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  char* mbase = cv.take<char>(4 * mats);
  GramJob* d_gj = cv.take<GramJob>(nprob);
  CholJob* d_cj = cv.take<CholJob>(nprob);
  int4* d_units = cv.take<int4>(units.size());
  int4* d_nodes = cv.take<int4>(std::max<size_t>(1, nodes.size()));
  int* d_levels = cv.take<int>(levels.size());
  int* d_ctajob = cv.take<int>(gmax);
  unsigned* d_bars = cv.take<unsigned>((size_t)nprob * 16);
  std::vector<GramJob> gj(nprob);
  std::vector<CholJob> cj(nprob);
  size_t off = 0;
  for (int p = 0; p < nprob; ++p) {
    const int nblk = (d[p] + 31) / 32, dp = nblk * 32;
    const size_t mb = lsq_align256((size_t)dp * dp * 8);
    double* G = reinterpret_cast<double*>(mbase + off);
    double* Rf = reinterpret_cast<double*>(mbase + mats + off);
    double* Wf = reinterpret_cast<double*>(mbase + 2 * mats + off);
    double* Tb = reinterpret_cast<double*>(mbase + 3 * mats + off);
    off += mb;
    gj[p] = GramJob{SA[p], G, m[p], d[p], dp};
    cj[p].G = G;
    cj[p].Rf = Rf;
    cj[p].Wf = Wf;
    cj[p].Tb = Tb;
    cj[p].nodes = d_nodes + tree_node0[nblk];
    cj[p].level_start = d_levels + tree_lev0[nblk];
    cj[p].nlevels = tree_nlev[nblk];
    cj[p].nblk = nblk;
    cj[p].bar = d_bars + (size_t)p * 16;
    cj[p].err = reinterpret_cast<int*>(d_bars + (size_t)p * 16 + 8);
    cj[p].W = W[p];
    cj[p].WT = WT[p];
    cj[p].d = d[p];
  }
  LSQ_CUDA_TRY(cudaMemsetAsync(mbase + mats, 0, 2 * mats, s));  // Rf, Wf
  LSQ_CUDA_TRY(cudaMemsetAsync(d_bars, 0, (size_t)nprob * 64, s));
  LSQ_CUDA_TRY(cudaMemcpy(d_gj, gj.data(), sizeof(GramJob) * nprob, cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemcpy(d_units, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice));
  if (!nodes.empty()) LSQ_CUDA_TRY(cudaMemcpy(d_nodes, nodes.data(), sizeof(int4) * nodes.size(), cudaMemcpyHostToDevice));
  LSQ_CUDA_TRY(cudaMemcpy(d_levels, levels.data(), sizeof(int) * levels.size(), cudaMemcpyHostToDevice));
  if (df_gram)
    gram_batched_kernel<true><<<(unsigned)units.size(), 256, 0, s>>>(d_gj, d_units);
  else
    gram_batched_kernel<false><<<(unsigned)units.size(), 256, 0, s>>>(d_gj, d_units);
  LSQ_LAUNCH_CHECK();
  // CTA groups sized so that every problem takes about the same time T: its FP64 work (the
  // Cholesky and the inverse, 2 d^3 / 3 FMAs) at the rate of g CTAs, but no less than its chain
  // of diagonal blocks; T is the longest chain or the whole work spread over the grid, whichever
  // is larger.  The largest problems first, in waves that fill the cooperative grid.
  std::vector<int> order(nprob);
  for (int p = 0; p < nprob; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return d[x] > d[y]; });
  const double cta_rate = 1.75 * 2.0e9 / cta_per_sm;  // FP64 FMA per second of a CTA
  auto work = [&](int p) { const double dd = ((d[p] + 31) / 32) * 32.0; return 2.0 / 3.0 * dd * dd * dd; };
  double total_work = 0.0, longest_chain = 0.0;
  for (int p = 0; p < nprob; ++p) {
    total_work += work(p);
    longest_chain = std::max(longest_chain, ((d[p] + 31) / 32) * 60e-6);
  }
  std::vector<int> gsize(nprob);
  auto size_groups = [&](double T) {
    long long sum = 0;
    for (int p = 0; p < nprob; ++p) {
      const int nblk = (d[p] + 31) / 32;
      const int cap = std::min(gmax, std::max(1, 4 * nblk * nblk));
      gsize[p] = std::max(1, std::min(cap, (int)std::ceil(work(p) / (T * cta_rate))));
      sum += gsize[p];
    }
    return sum;
  };
  if (nprob <= gmax) {
    // one wave: the shortest T whose groups fill the grid (bisection on T)
    double lo = longest_chain, hi = std::max(lo, total_work / cta_rate);
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (size_groups(mid) <= gmax) hi = mid;
      else lo = mid;
    }
    size_groups(hi);
  } else {
    size_groups(std::max(longest_chain, total_work / (gmax * cta_rate)));
  }
  size_t next = 0;
  while (next < order.size()) {
    const size_t w0 = next;
    size_t w1 = w0;
    int used = 0;
    while (w1 < order.size() && used + gsize[order[w1]] <= gmax) used += gsize[order[w1++]];
    std::vector<int> ctajob;
    for (size_t i = w0; i < w1; ++i) {
      const int p = order[i];
      const int g = gsize[p];
      cj[p].cta0 = (int)ctajob.size();
      cj[p].ncta = g;
      for (int q = 0; q < g; ++q) ctajob.push_back(p);
    }
    LSQ_CUDA_TRY(cudaMemcpy(d_cj, cj.data(), sizeof(CholJob) * nprob, cudaMemcpyHostToDevice));
    LSQ_CUDA_TRY(cudaMemcpy(d_ctajob, ctajob.data(), sizeof(int) * ctajob.size(), cudaMemcpyHostToDevice));
    const CholJob* jp = d_cj;
    const int* cp = d_ctajob;
    void* args[] = {(void*)&jp, (void*)&cp};
    LSQ_CUDA_TRY(cudaLaunchCooperativeKernel((void*)chol_inv_batched_kernel, dim3((unsigned)ctajob.size()), dim3(256),
                                             args, 0, s));
    lsq_count_launch();
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));  // the tables are rewritten for the next wave
    next = w1;
  }
  LSQ_CUDA_TRY(cudaMemcpy(d_cj, cj.data(), sizeof(CholJob) * nprob, cudaMemcpyHostToDevice));
  w_out_batched_kernel<<<dim3(64, (unsigned)nprob), 256, 0, s>>>(d_cj);
  LSQ_LAUNCH_CHECK();
  std::vector<unsigned> bars((size_t)nprob * 16);
  LSQ_CUDA_TRY(cudaMemcpyAsync(bars.data(), d_bars, bars.size() * 4, cudaMemcpyDeviceToHost, s));
  LSQ_CUDA_TRY(cudaStreamSynchronize(s));
  lsq_status overall = LSQ_OK;
  for (int p = 0; p < nprob; ++p) {
    const int code = (int)bars[(size_t)p * 16 + 8];
    status_out[p] = code;
    if (code != 0 && code != LSQ_ERR_RANK && overall == LSQ_OK) overall = (lsq_status)code;
  }
  return overall;
}
