// apass.cuh -- the fused pass over A (v = A^T (A p), q = ||A p||^2, one read of each row)
// shared by the solver and the standalone pass entry points.  Internal, not part of the ABI.
#pragma once

#include "common.cuh"

namespace lsq_apass {

template <typename TA>
__device__ __forceinline__ double ld_elem(const TA* p) {
  return (double)__ldg(p);
}

// ------------------------------------------------------------------------------------
// Fused pass over the rows [r0, r1): per-warp accumulators of v = A^T (A p) in
// registers (lane owns columns lane + 32 k), q = sum (a_i . p)^2; then a fixed-order
// CTA reduction into part[c * P + cta].  The next row is loaded before the current
// one is used so that each warp keeps two rows in flight.
// ------------------------------------------------------------------------------------
template <typename TA, int EPL, bool ALLOW_PREFETCH = true>
__device__ void fused_pass(const TA* __restrict__ A, int64_t ld, int d, int dp, int64_t r0, int64_t r1,
                           const double* vec_s, double* wred, double* qred, double* part, int P, int cta) {
  constexpr bool PV_REG = EPL <= 8;   // keep p in registers while they are plentiful
  constexpr bool PREFETCH = ALLOW_PREFETCH && EPL <= 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double pv[PV_REG ? EPL : 1], acc[EPL], cur[EPL], nxt[PREFETCH ? EPL : 1];
  bool ok[EPL];
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = lane + 32 * k;
    ok[k] = c < d;
    if (PV_REG) pv[k] = ok[k] ? vec_s[c] : 0.0;
    acc[k] = 0.0;
  }
  double q = 0.0;
  int64_t i = r0 + warp;
  if (PREFETCH && i < r1) {
    const TA* a = A + i * ld;
#pragma unroll
    for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? ld_elem(a + lane + 32 * k) : 0.0;
  }
  for (; i < r1; i += LSQ_WARPS) {
    if (PREFETCH) {
      const int64_t inext = i + LSQ_WARPS;
      if (inext < r1) {
        const TA* a = A + inext * ld;
#pragma unroll
        for (int k = 0; k < (PREFETCH ? EPL : 1); ++k) nxt[k] = ok[k] ? ld_elem(a + lane + 32 * k) : 0.0;
      }
    } else {
      const TA* a = A + i * ld;
#pragma unroll
      for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? ld_elem(a + lane + 32 * k) : 0.0;
    }
    double w = 0.0;
#pragma unroll
    for (int k = 0; k < EPL; ++k) w = fma(cur[k], PV_REG ? pv[PV_REG ? k : 0] : vec_s[lane + 32 * k], w);
    w = warp_sum(w);
#pragma unroll
    for (int k = 0; k < EPL; ++k) acc[k] = fma(w, cur[k], acc[k]);
    q = fma(w, w, q);
    if (PREFETCH) {
#pragma unroll
      for (int k = 0; k < EPL; ++k) cur[k] = nxt[PREFETCH ? k : 0];
    }
  }
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = lane + 32 * k;
    if (c < dp) wred[warp * dp + c] = acc[k];
  }
  if (lane == 0) qred[warp] = q;
  __syncthreads();
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < LSQ_WARPS; ++w) s += wred[w * dp + c];
    part[(int64_t)c * P + cta] = s;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < LSQ_WARPS; ++w) s += qred[w];
    part[(int64_t)dp * P + cta] = s;
  }
  __syncthreads();
}


// ------------------------------------------------------------------------------------
// FP32 arithmetic variant of the pass (the inner passes of the mixed-precision solve).
// FP64 elements are narrowed to FP32 by integer operations on their bit pattern (the
// FP64->FP32 conversion instruction runs at the FP64 rate, about 2 per clock per SM on
// this part, below the ~3 elements per clock per SM that the HBM rate needs):
// mantissa truncated to 23 bits, exponent clamped so that values below the FP32 normal
// range become (tiny) subnormal-or-zero patterns and values above it become non-finite,
// which the solver reports as a breakdown.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float narrow_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t lo = (uint32_t)u, hi = (uint32_t)(u >> 32);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t ec = min(max(e, 896u), 1151u) - 896u;
  const uint32_t mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
  return __uint_as_float((ec << 23) | mant | (hi & 0x80000000u));
}

__device__ __forceinline__ float narrow_f32(float x) { return x; }

// column of element k of a lane's row slice: lane + 32 k, or, at EPL >= 16, 128 (k / 4) + 4 lane + k % 4
// (four adjacent columns per lane, the layout of the bulk-copy pass below, so both compute with
// the same values in the same order)
template <int EPL>
__device__ __forceinline__ int f32_col(int k, int lane) {
  return EPL >= 16 ? 128 * (k >> 2) + 4 * lane + (k & 3) : lane + 32 * k;
}

template <typename TA, int EPL>
__device__ void fused_pass_f32(const TA* __restrict__ A, int64_t ld, int d, int dp, int64_t r0, int64_t r1,
                               const double* vec_s, double* wred, double* qred, double* part, int P, int cta) {
  // two rows in flight per warp while the registers allow it (raw FP64 rows are 2 registers
  // per element); p from shared memory at the widest rows
  constexpr bool PREFETCH = sizeof(TA) == 4 || EPL <= 16;
  constexpr bool PV_REG = EPL <= 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // FP32 copy of p in the (not yet used) reduction buffer: one conversion per entry per pass
  float* pf = reinterpret_cast<float*>(wred);
  for (int c = threadIdx.x; c < dp; c += blockDim.x) pf[c] = (float)vec_s[c];
  __syncthreads();
  float pv[PV_REG ? EPL : 1], acc[EPL];
  TA cur[EPL];
  bool ok[EPL];
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = f32_col<EPL>(k, lane);
    ok[k] = c < d;
    if (PV_REG) pv[PV_REG ? k : 0] = ok[k] ? pf[c] : 0.0f;
    acc[k] = 0.0f;
  }
  double q = 0.0;
  int64_t i = r0 + warp;
  if (PREFETCH && i < r1) {
    const TA* a = A + i * ld;
#pragma unroll
    for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? __ldg(a + f32_col<EPL>(k, lane)) : (TA)0;
  }
  for (; i < r1; i += LSQ_WARPS) {
    if (!PREFETCH) {
      const TA* a = A + i * ld;
#pragma unroll
      for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? __ldg(a + f32_col<EPL>(k, lane)) : (TA)0;
    }
    // narrow the row first (its raw registers die here), then put the next row in flight
    float af[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) af[k] = narrow_f32(cur[k]);
    if (PREFETCH) {
      const int64_t inext = i + LSQ_WARPS;
      if (inext < r1) {
        const TA* a = A + inext * ld;
#pragma unroll
        for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? __ldg(a + f32_col<EPL>(k, lane)) : (TA)0;
      }
    }
    float w = 0.0f;
#pragma unroll
    for (int k = 0; k < EPL; ++k) w = fmaf(af[k], PV_REG ? pv[PV_REG ? k : 0] : pf[f32_col<EPL>(k, lane)], w);
    w = warp_sumf(w);
#pragma unroll
    for (int k = 0; k < EPL; ++k) acc[k] = fmaf(w, af[k], acc[k]);
    q = fma((double)w, (double)w, q);
  }
  __syncthreads();  // every warp is done with pf before wred is overwritten
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = f32_col<EPL>(k, lane);
    if (c < dp) wred[warp * dp + c] = (double)acc[k];
  }
  if (lane == 0) qred[warp] = q;
  __syncthreads();
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < LSQ_WARPS; ++w2) s += wred[w2 * dp + c];
    part[(int64_t)c * P + cta] = s;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w2 = 0; w2 < LSQ_WARPS; ++w2) s += qred[w2];
    part[(int64_t)dp * P + cta] = s;
  }
  __syncthreads();
}


// ------------------------------------------------------------------------------------
// The FP32 pass for wide FP32 rows (256 < d <= 1024, d a multiple of 4, 16-byte aligned rows)
// with the rows staged by bulk copies: each warp keeps RING_NS of its rows in flight in a ring
// of shared-memory slots, one cp.async.bulk per row started by lane 0 and counted in bytes on
// the slot's mbarrier, instead of one row prefetched in registers.  The registers that frees
// hold p, and the deeper queue keeps HBM busy with one 256-thread CTA per SM.  Lane l owns the
// columns 128 k + 4 l + t (k < 8, t < 4) and reads them as eight 16-byte vectors per row.
// Every wait is bounded: on a time-out the pass records LSQ_ERR_TIMEOUT, waits (bounded) for
// its copies still in flight and returns; the caller checks the flag at its next barrier.
// ------------------------------------------------------------------------------------
constexpr int RING_NS = 4;
constexpr uint32_t RING_SPIN = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32a(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ring_init(uint64_t* bars) {
  // thread 0, before a CTA barrier: one arrival (the expect-tx) per phase
  for (int e = 0; e < LSQ_WARPS * RING_NS; ++e)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32a(bars + e)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void ring_issue(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32a(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32a(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32a(bar))
      : "memory");
}

__device__ __forceinline__ bool ring_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t spins = 0; spins < RING_SPIN; ++spins) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32a(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// ring: LSQ_WARPS x RING_NS slots of `slot_floats` floats; bars: LSQ_WARPS x RING_NS mbarriers;
// phase: this thread's parity bits of its warp's slots (kept across passes by the caller)
template <int EPL>
__device__ inline void fused_pass_f32_ring(const float* __restrict__ A, int64_t ld, int d, int dp, int64_t r0,
                                           int64_t r1, const double* vec_s, double* wred, double* qred, double* part,
                                           int P, int cta, float* ring, int slot_floats, uint64_t* bars,
                                           uint32_t& phase, int* err) {
  static_assert(EPL == 16 || EPL == 32, "rows of 512 or 1024 padded columns");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* pf = reinterpret_cast<float*>(wred);
  for (int c = threadIdx.x; c < dp; c += blockDim.x) pf[c] = (float)vec_s[c];
  __syncthreads();
  float pv[EPL], acc[EPL];
  bool okc[EPL / 4];
#pragma unroll
  for (int k = 0; k < EPL / 4; ++k) {
    const int c0 = 128 * k + 4 * lane;
    okc[k] = c0 < d;  // d is a multiple of 4: the four columns are in or out together
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      pv[4 * k + t] = okc[k] ? pf[c0 + t] : 0.0f;
      acc[4 * k + t] = 0.0f;
    }
  }
  double q = 0.0;
  float* slots = ring + (size_t)warp * RING_NS * slot_floats;
  uint64_t* bar = bars + warp * RING_NS;
  const uint32_t bytes = (uint32_t)d * 4u;
  const int64_t first = r0 + warp;
  // rows first + LSQ_WARPS j of this warp; slot j % RING_NS
  int64_t issued = 0, done = 0;
  const int64_t nrows = first < r1 ? (r1 - first + LSQ_WARPS - 1) / LSQ_WARPS : 0;
  for (; issued < nrows && issued < RING_NS; ++issued)
    if (lane == 0) ring_issue(slots + issued * slot_floats, A + (first + LSQ_WARPS * issued) * ld, bytes, bar + issued);
  bool good = true;
  for (; done < nrows; ++done) {
    const int s = (int)(done % RING_NS);
    const bool landed = __all_sync(0xffffffffu, ring_wait(bar + s, (phase >> s) & 1u));
    if (!landed) {
      good = false;
      break;
    }
    phase ^= 1u << s;
    const float4* row = reinterpret_cast<const float4*>(slots + s * slot_floats);
    float af[EPL];
#pragma unroll
    for (int k = 0; k < EPL / 4; ++k) {
      const float4 v = okc[k] ? row[32 * k + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      af[4 * k] = v.x;
      af[4 * k + 1] = v.y;
      af[4 * k + 2] = v.z;
      af[4 * k + 3] = v.w;
    }
    __syncwarp();  // every lane has its values: the slot may be refilled
    if (issued < nrows) {
      if (lane == 0) ring_issue(slots + s * slot_floats, A + (first + LSQ_WARPS * issued) * ld, bytes, bar + s);
      ++issued;
    }
    float w = 0.0f;
#pragma unroll
    for (int k = 0; k < EPL; ++k) w = fmaf(af[k], pv[k], w);
    w = warp_sumf(w);
#pragma unroll
    for (int k = 0; k < EPL; ++k) acc[k] = fmaf(w, af[k], acc[k]);
    q = fma((double)w, (double)w, q);
  }
  if (!good) {
    if (lane == 0) atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
    // the copies still in flight land before the slots are given up (bounded)
    for (; done < issued; ++done) {
      const int s = (int)(done % RING_NS);
      if (ring_wait(bar + s, (phase >> s) & 1u)) phase ^= 1u << s;
    }
  }
  __syncthreads();  // every warp is done with pf before wred is overwritten
#pragma unroll
  for (int k = 0; k < EPL / 4; ++k) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 128 * k + 4 * lane + t;
      if (c < dp) wred[warp * dp + c] = (double)acc[4 * k + t];
    }
  }
  if (lane == 0) qred[warp] = q;
  __syncthreads();
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    double s2 = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < LSQ_WARPS; ++w2) s2 += wred[w2 * dp + c];
    part[(int64_t)c * P + cta] = s2;
  }
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int w2 = 0; w2 < LSQ_WARPS; ++w2) s2 += qred[w2];
    part[(int64_t)dp * P + cta] = s2;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// Exact pass in double-FP32 arithmetic (the residual replacements of the mixed solve).
// Each FP64 element a is split into a head of 21 significant bits and the FP32 rounding
// of its remaining 32 mantissa bits (about 45 significant bits in all); products are made
// error-free with an FMA (TwoProduct) and sums are carried as unevaluated (hi, lo) FP32
// pairs with Knuth's TwoSum (Dekker 1971; Knuth, TAOCP vol. 2).  v = A^T (A x) comes out
// with a relative error of a few 1e-14 per component, far below what the solver's
// tolerance needs, at the throughput of the FP32 and integer pipes.
// Elements with |a| < 2^-74 keep only their head (their tail would underflow FP32).
// ------------------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ void split_df(double x, float& head, float& tail) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t lo32 = (uint32_t)u, hi32 = (uint32_t)(u >> 32);
  const uint32_t sign = hi32 & 0x80000000u;
  const uint32_t e = (hi32 >> 20) & 0x7FFu;
  const uint32_t ec = min(max(e, 896u), 1151u);
  head = __uint_as_float(sign | ((ec - 896u) << 23) | ((hi32 & 0xFFFFFu) << 3));
  // tail = lo32 * 2^(e - 1075), sign of x; zero when that scale leaves the FP32 range
  const float scale = __uint_as_float(sign | ((e - 948u) << 23));
  tail = (e >= 949u && e <= 1151u) ? __fmul_rn(__uint2float_rn(lo32), scale) : 0.0f;
}

__device__ __forceinline__ void split_df(float x, float& head, float& tail) {
  head = x;
  tail = 0.0f;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += (ah + al) * (bh + bl), dropping only al * bl
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  const float cross = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pe));
  float s, e;
  two_sum(sh, p, s, e);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, cross));
}

__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, bl));
}

// v partials only (the residual needs no q); part[dp * P + cta] is written as 0
template <typename TA, int EPL>
__device__ void fused_pass_df(const TA* __restrict__ A, int64_t ld, int d, int dp, int64_t r0, int64_t r1,
                              const double* vec_s, double* wred, double* qred, double* part, int P, int cta) {
  constexpr bool PREFETCH = sizeof(TA) == 4 || EPL <= 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* xs = reinterpret_cast<float2*>(wred);  // (head, tail) of x, dp entries
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    const double xv = vec_s[c];
    const float xh = (float)xv;
    xs[c] = make_float2(xh, (float)(xv - (double)xh));
  }
  __syncthreads();
  float vh[EPL], vl[EPL];
  TA cur[EPL];
  bool ok[EPL];
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    ok[k] = lane + 32 * k < d;
    vh[k] = 0.0f;
    vl[k] = 0.0f;
  }
  int64_t i = r0 + warp;
  if (PREFETCH && i < r1) {
    const TA* a = A + i * ld;
#pragma unroll
    for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? __ldg(a + lane + 32 * k) : (TA)0;
  }
  for (; i < r1; i += LSQ_WARPS) {
    if (!PREFETCH) {
      const TA* a = A + i * ld;
#pragma unroll
      for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? __ldg(a + lane + 32 * k) : (TA)0;
    }
    float ah[EPL], al[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) split_df(cur[k], ah[k], al[k]);
    if (PREFETCH) {
      const int64_t inext = i + LSQ_WARPS;
      if (inext < r1) {
        const TA* a = A + inext * ld;
#pragma unroll
        for (int k = 0; k < EPL; ++k) cur[k] = ok[k] ? __ldg(a + lane + 32 * k) : (TA)0;
      }
    }
    float wh = 0.0f, wl = 0.0f;
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      const float2 xv = xs[lane + 32 * k];
      df_fma(ah[k], al[k], xv.x, xv.y, wh, wl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, wh, o);
      const float ol = __shfl_xor_sync(0xffffffffu, wl, o);
      df_add(wh, wl, oh, ol);
    }
    // renormalise w to a clean (head, tail) pair
    float nh, nl;
    two_sum(wh, wl, nh, nl);
#pragma unroll
    for (int k = 0; k < EPL; ++k) df_fma(ah[k], al[k], nh, nl, vh[k], vl[k]);
  }
  __syncthreads();  // every warp is done with xs before wred is overwritten
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = lane + 32 * k;
    if (c < dp) wred[warp * dp + c] = (double)vh[k] + (double)vl[k];
  }
  if (lane == 0) qred[warp] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < LSQ_WARPS; ++w2) sum += wred[w2 * dp + c];
    part[(int64_t)c * P + cta] = sum;
  }
  if (threadIdx.x == 0) part[(int64_t)dp * P + cta] = 0.0;
  __syncthreads();
}

// The same pass for FP64 rows, staged through shared memory: each warp has one row slot
// (slots: LSQ_WARPS x dp doubles, which may lie in wred past its first dp entries) and, as
// soon as the current row is split into registers, has the next row copied into the slot
// with cp.async while it computes, so a row is in flight without holding registers (the
// split row and the double-FP32 accumulators already fill them).  Each lane copies and reads
// only its own elements (columns lane + 32 k): its own cp.async.wait_group orders the data,
// and a __syncwarp (which orders the memory operations of the lanes it joins) separates the
// loads of the current row from the copy of the next one into the same slot.  Same
// arithmetic, in the same order, as fused_pass_df.
__device__ __forceinline__ void cp_async_8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_none() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int EPL>
__device__ void fused_pass_df_staged(const double* __restrict__ A, int64_t ld, int d, int dp, int64_t r0, int64_t r1,
                                     const double* vec_s, double* wred, double* qred, double* part, int P, int cta,
                                     double* slots) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* xs = reinterpret_cast<float2*>(wred);  // (head, tail) of x, dp entries
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    const double xv = vec_s[c];
    const float xh = (float)xv;
    xs[c] = make_float2(xh, (float)(xv - (double)xh));
  }
  double* slot = slots + (int64_t)warp * dp + lane;
  float vh[EPL], vl[EPL];
  bool ok[EPL];
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    ok[k] = lane + 32 * k < d;
    vh[k] = 0.0f;
    vl[k] = 0.0f;
    // columns at or past d are never copied: zero in the slot for the whole pass
    if (!ok[k]) slot[32 * k] = 0.0;
  }
  __syncthreads();  // xs complete; no warp still reads wred from before the pass
  int64_t i = r0 + warp;
  if (i < r1) {
    const double* a = A + i * ld + lane;
#pragma unroll
    for (int k = 0; k < EPL; ++k)
      if (ok[k]) cp_async_8(slot + 32 * k, a + 32 * k);
  }
  cp_async_commit_group();
  for (; i < r1; i += LSQ_WARPS) {
    cp_async_wait_none();  // row i has landed
    float ah[EPL], al[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) split_df(slot[32 * k], ah[k], al[k]);
    __syncwarp();
    const int64_t inext = i + LSQ_WARPS;
    if (inext < r1) {
      const double* a = A + inext * ld + lane;
#pragma unroll
      for (int k = 0; k < EPL; ++k)
        if (ok[k]) cp_async_8(slot + 32 * k, a + 32 * k);
    }
    cp_async_commit_group();
    float wh = 0.0f, wl = 0.0f;
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      const float2 xv = xs[lane + 32 * k];
      df_fma(ah[k], al[k], xv.x, xv.y, wh, wl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, wh, o);
      const float ol = __shfl_xor_sync(0xffffffffu, wl, o);
      df_add(wh, wl, oh, ol);
    }
    float nh, nl;
    two_sum(wh, wl, nh, nl);
#pragma unroll
    for (int k = 0; k < EPL; ++k) df_fma(ah[k], al[k], nh, nl, vh[k], vl[k]);
  }
  cp_async_wait_none();
  __syncthreads();  // every warp is done with xs and its slot before wred is overwritten
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = lane + 32 * k;
    if (c < dp) wred[warp * dp + c] = (double)vh[k] + (double)vl[k];
  }
  if (lane == 0) qred[warp] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < LSQ_WARPS; ++w2) sum += wred[w2 * dp + c];
    part[(int64_t)c * P + cta] = sum;
  }
  if (threadIdx.x == 0) part[(int64_t)dp * P + cta] = 0.0;
  __syncthreads();
}

// sum_{j < P} src[j] by one warp, fixed order
__device__ __forceinline__ double warp_sum_strip(const double* src, int P) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int j = lane; j < P; j += 32) s += src[j];
  return warp_sum(s);
}

// standalone pass: CTA b handles rows [b * rows_per_cta, (b + 1) * rows_per_cta)
template <typename TA, int EPL>
__global__ void __launch_bounds__(LSQ_THREADS, 1) hmatvec_kernel(const void* A, int64_t n, int d, int dp, int64_t ld,
                                                                  int64_t rows_per_cta, const double* p, double* part) {
  extern __shared__ __align__(16) double smem[];
  double* vec = smem;
  double* wred = vec + dp;
  double* qred = wred + LSQ_WARPS * dp;
  for (int c = threadIdx.x; c < dp; c += blockDim.x) vec[c] = c < d ? p[c] : 0.0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(n, r0 + rows_per_cta);
  fused_pass<TA, EPL>(reinterpret_cast<const TA*>(A), ld, d, dp, r0, r1, vec, wred, qred, part, gridDim.x,
                      blockIdx.x);
}

// v[c] = sum_j part[c][j] (c < d), q = sum_j part[dp][j]; one warp per output, fixed order
static __global__ void reduce_part_kernel(const double* part, int P, int d, int dp, double* v, double* q) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c <= d; c += nw) {
    const int src = c < d ? c : dp;
    const double s = warp_sum_strip(part + (int64_t)src * P, P);
    if (lane == 0) {
      if (c < d) v[c] = s;
      else *q = s;
    }
  }
}

// elements per lane: the smallest power of two with 32 * EPL >= d
static inline int epl_for(int d) {
  int e = 1;
  while (32 * e < d) e <<= 1;
  return e;
}

template <typename TA>
static void* pick_hmv(int epl) {
  switch (epl) {
    case 1: return (void*)hmatvec_kernel<TA, 1>;
    case 2: return (void*)hmatvec_kernel<TA, 2>;
    case 4: return (void*)hmatvec_kernel<TA, 4>;
    case 8: return (void*)hmatvec_kernel<TA, 8>;
    case 16: return (void*)hmatvec_kernel<TA, 16>;
    default: return (void*)hmatvec_kernel<TA, 32>;
  }
}

static inline size_t hmatvec_smem_bytes(int dp) { return (size_t)(dp + LSQ_WARPS * dp + LSQ_WARPS) * 8; }

}  // namespace lsq_apass
