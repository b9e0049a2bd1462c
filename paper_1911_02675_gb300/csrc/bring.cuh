// bring.cuh -- the batched pass over FP32 A with contiguous, 16-byte aligned rows (included by
// batch.cu inside its namespace, after BProb / BatchArgs).
//
// The same sums as pass_chunk / pass_chunk_df (part[j dp + c] = sum_rows a_c (a . p_j) and
// q_j = sum_rows (a . p_j)^2, Section 1 eq. (PCG) per right-hand side), with a different
// schedule: a chunk's rows stream into a ring of RNS shared-memory stages of 32 KB, one
// cp.async.bulk per stage (see rp_issue) counted in bytes on the stage's `full` mbarrier; the
// eight warps release a stage on its `empty` mbarrier once they have read it, and thread 0 refills
// it with the stage RNS - 1 ahead.  In the exact (SIMT) pass, warp w owns the right-hand sides
// jg JG .. jg JG + JG - 1 (jg = w mod J, J = kp / JG) and every J-th group of rows; inside a
// warp, L = dp / EPL lanes share a row (32 / L rows at a time) and lane l owns the columns
// l mod L + L e (e < EPL).  Per row: the lanes' partial dots with their registers of X, a
// butterfly sum over the L lanes (every lane ends with all JG dots), then acc += a y^T in
// registers, all in the double-FP32 products and sums of pass_chunk_df.  The FP32 pass runs on
// the tensor cores (rp_chunk_mma below).
// Every wait is bounded; on a time-out the CTA records it, waits (bounded) for its copies still
// in flight and stops.
#pragma once

constexpr int RW = 8;                  // warps of a CTA (two per SM sub-partition: up to 255 registers)
constexpr int RT = RW * 32;            // threads of a CTA
constexpr int RNS = 6;                 // stages in the ring
constexpr int RSTAGE = 8256;           // floats per stage (16 rows of 512 and the alignment slack)
// the FP32 pass on the tensor cores: the stage-1 partial tiles (RYP), Y split in two (RY each),
// per-thread q (RQF)
constexpr int RYP = 8 * 256, RY = 128 * 16, RQF = 256;
constexpr size_t RSMEM = ((size_t)RNS * RSTAGE + RYP + 2 * RY + RQF) * 4;  // dynamic shared memory
constexpr uint32_t RSPIN = 1u << 24;   // polls of a wait before it gives up

__device__ __forceinline__ bool rp_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t spins = 0; spins < RSPIN; ++spins) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(lsq_apass::smem_u32a(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void rp_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(lsq_apass::smem_u32a(bar)) : "memory");
}

__device__ __forceinline__ void rp_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// (sh, sl) += a (bh + bl) with a exact in FP32: TwoProduct by FMA, the tail product folded into
// the error term, TwoSum into the head (Dekker 1971; Knuth)
__device__ __forceinline__ void rp_df_fma(float a, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(a, bh);
  const float cross = __fmaf_rn(a, bl, __fmaf_rn(a, bh, -p));
  float s, e;
  lsq_apass::two_sum(sh, p, s, e);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, cross));
}

// (ah, al) += (bh, bl) with the tails added first, so that two lanes exchanging their sums end
// with the same value
__device__ __forceinline__ void rp_df_add_sym(float& ah, float& al, float bh, float bl) {
  float s, e;
  lsq_apass::two_sum(ah, bh, s, e);
  ah = s;
  al = __fadd_rn(__fadd_rn(al, bl), e);
}

// Puts stage t of the chunk [r0, r1) (R rows a stage) in flight into its slot, once the warps
// have released the slot's previous stage: the stage's element range and the 8 floats after it
// (the tensor-core pass reads up to 7 of them, beside zeros of P: the matrix's own next row), the
// range rounded out to 16 bytes.  Where that would read past the matrix, the copy stops at the
// last 16-byte boundary, plain loads fetch the last < 4 elements and zeros fill the 8 floats after
// them (so that stale floats of another problem never meet this one's products), and only then
// does the thread need a proxy fence before its copy.  `released`: the caller knows that every
// warp has released the slot (a CTA barrier after their arrivals), so its wait is skipped.
// Returns false if the wait for the slot gave up.
__device__ __forceinline__ bool rp_issue(const float* A, int64_t n_elems, int d, int64_t r0, int64_t r1, int R, int t,
                                         uint32_t gs, float* ring, uint64_t* full, uint64_t* empty,
                                         bool released = false) {
  const uint32_t g = gs + (uint32_t)t;
  const int s = (int)(g % RNS);
  const uint32_t u = g / RNS;
  if (!released && u >= 1 && !rp_wait(empty + s, (u - 1) & 1u)) return false;
  const int64_t lo = r0 + (int64_t)t * R, hi = min(r1, lo + R);
  const int64_t e_lo = lo * d, e_hi = hi * d;
  const int64_t a_lo = e_lo & ~(int64_t)3;
  int64_t a_hi = (e_hi + 8 + 3) & ~(int64_t)3;
  float* buf = ring + s * RSTAGE;
  if (a_hi > n_elems) {
    a_hi = e_hi & ~(int64_t)3;
    for (int64_t e = a_hi; e < e_hi; ++e) buf[e - a_lo] = __ldg(A + e);
    const int z0 = (int)(e_hi - a_lo);
    for (int i = 0; i < 8; ++i) buf[z0 + i] = 0.f;
    rp_fence_async();  // this thread's plain stores to the ring come before its copies
  }
  const uint32_t bytes = (uint32_t)(a_hi - a_lo) * 4u;
  if (bytes) lsq_apass::ring_issue(buf, A + a_lo, bytes, full + s);
  else rp_arrive(full + s);
  return true;
}

// One exact (double-FP32) chunk, rows [r0, r1) of problem pr, stages gs .. gs + nst - 1 of this
// CTA's ring: part[j dp + c] = sum_rows a_c (a . x_j), part[kp dp + j] = 0.  Returns the number of
// stages it used.  Called by every thread of the CTA.
template <int EPL, int JG>
__device__ __forceinline__ int rp_chunk_exact(const BProb& pr, int64_t r0, int64_t r1, double* __restrict__ out,
                                              float* ring, uint64_t* full, uint64_t* empty, uint32_t gs,
                                              volatile int* s_err) {
  const int d = pr.d, dp = pr.dp, kp = pr.kp;
  const int L = dp / EPL;                 // lanes per row: 8, 16 or 32
  const int lgL = 31 - __clz(L);
  const int RPW = 32 >> lgL;              // rows a warp takes at once
  const int R = (RSTAGE - 16) / d;        // rows per stage (room for the zeros placed past them)
  const int nst = (int)((r1 - r0 + R - 1) / R);
  const int J = kp / JG;                  // groups of right-hand sides
  const int NRS = RW / J;                 // row slices of warps
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* A = reinterpret_cast<const float*>(pr.A);
  int issued = 0;  // stages put in flight (lane 0 of warp 0)
  const bool prod = tid == 0;
  // consumer roles: right-hand-side group jg, row slice rs; sub-row and lane within the row
  const int jg = warp % J, rs = warp / J;
  const bool act = rs < NRS;
  const int sub = lane >> lgL, sl = lane & (L - 1);
  auto issue = [&](int t) {
    if (rp_issue(A, pr.n * d, d, r0, r1, R, t, gs, ring, full, empty)) ++issued;
    else *s_err = 1;
  };
  if (prod)
    for (int t = 0; t < nst && t < RNS - 1 && !*s_err; ++t) issue(t);
  // head and tail of this warp's right-hand sides of X at the lane's columns; the accumulators
  float pv[EPL][JG], pl[EPL][JG], acc[EPL][JG], accl[EPL][JG];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int c = sl + L * e;
#pragma unroll
    for (int j = 0; j < JG; ++j) {
      const int jj = jg * JG + j;
      const bool in = act && c < d && jj < pr.k;
      pv[e][j] = in ? pr.Xh[c * kp + jj] : 0.f;
      pl[e][j] = in ? pr.Xl[c * kp + jj] : 0.f;
      acc[e][j] = accl[e][j] = 0.f;
    }
  }
  for (int t = 0; t < nst; ++t) {
    const uint32_t g = gs + (uint32_t)t;
    const int s = (int)(g % RNS);
    if (prod && t + RNS - 1 < nst && !*s_err) issue(t + RNS - 1);
    __syncwarp();
    // (one decision per warp: every lane takes part in the vote)
    if (!__all_sync(0xffffffffu, !*s_err && rp_wait(full + s, (g / RNS) & 1u))) {
      if (lane == 0) *s_err = 1;
      break;
    }
    if (act) {
      const int64_t lo = r0 + (int64_t)t * R;
      const int nrows = (int)(min(r1, lo + R) - lo);
      const int64_t e_lo = lo * d;
      const float* buf = ring + s * RSTAGE + (int)(e_lo - (e_lo & ~(int64_t)3));
      for (int m = rs * RPW; m < nrows; m += NRS * RPW) {
        const int i = m + sub;
        const bool valid = i < nrows;
        const float* row = buf + (valid ? i : 0) * d;
        float a[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int c = sl + L * e;
          a[e] = (valid && c < d) ? row[c] : 0.f;
        }
        {
          float yh[JG], yl[JG];
#pragma unroll
          for (int j = 0; j < JG; ++j) yh[j] = yl[j] = 0.f;
#pragma unroll
          for (int e = 0; e < EPL; ++e)
#pragma unroll
            for (int j = 0; j < JG; ++j) rp_df_fma(a[e], pv[e][j], pl[e][j], yh[j], yl[j]);
          for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < JG; ++j) {
              const float oh = __shfl_xor_sync(0xffffffffu, yh[j], o);
              const float ol = __shfl_xor_sync(0xffffffffu, yl[j], o);
              rp_df_add_sym(yh[j], yl[j], oh, ol);
            }
#pragma unroll
          for (int e = 0; e < EPL; ++e)
#pragma unroll
            for (int j = 0; j < JG; ++j) rp_df_fma(a[e], yh[j], yl[j], acc[e][j], accl[e][j]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) rp_arrive(empty + s);
  }
  __syncthreads();  // every stage has been read: the ring is free
  if (*s_err) {
    // the copies still in flight are among the last RNS issued: wait for them (bounded)
    if (prod)
      for (int t = issued > RNS ? issued - RNS : 0; t < issued; ++t) {
        const uint32_t g = gs + (uint32_t)t;
        rp_wait(full + g % RNS, (g / RNS) & 1u);
      }
    __syncthreads();
    return nst;
  }
  // per row slice partials of V (FP64), in the ring
  if (act) {
    double* red = reinterpret_cast<double*>(ring);
    const int slc = rs * RPW + sub;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int c = sl + L * e;
#pragma unroll
      for (int j = 0; j < JG; ++j) {
        red[((size_t)slc * kp + jg * JG + j) * dp + c] = (double)acc[e][j] + (double)accl[e][j];
      }
    }
  }
  __syncthreads();
  // fixed-order sums over the row slices
  const double* red = reinterpret_cast<const double*>(ring);
  const int nsl = (RW / J) * RPW;
  for (int e = tid; e < kp * dp; e += RT) {
    const int j = e / dp, c = e - j * dp;
    double sum = 0.0;
    for (int q2 = 0; q2 < nsl; ++q2) sum += red[((size_t)q2 * kp + j) * dp + c];
    out[e] = sum;
  }
  if (tid < kp) out[kp * dp + tid] = 0.0;  // the exact pass needs no q
  __syncthreads();
  // the ring again holds only finite floats (the tensor-core pass reads past a stage's rows)
  {
    float4* z = reinterpret_cast<float4*>(ring);
    const int n4 = (int)(((size_t)nsl * kp * dp * 2 + 3) / 4);
    for (int i = tid; i < n4; i += RT) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  rp_fence_async();  // the reads and writes of the reduction area come before the next copies into it
  __syncthreads();
  return nst;
}

// ------------------------------------------------------------------------------------
// The FP32 pass on the tensor cores.  Per stage of R = 16 nrt rows (at most 128), read in place
// from the ring slot:
//   stage 1  Y = A_stage P by warp-level m16n8k8 TF32 MMAs: a warp takes a 16-row tile and a run of
//            8-column k-steps (KS = 8 / nrt warps share a tile when nrt < 8), P fragments held in
//            registers for the whole chunk;
//   Y        the KS partial tiles summed in a fixed order, q_j += y_j^2, Y split for stage 2;
//   stage 2  V_stage = A_stage^T Y: a warp owns 16-column tiles of V and a slice of the stage's 8-row
//            k-steps; V_stage is added to the warp's running V by FP32 additions (the tensor
//            cores' own accumulation is kept to one stage: over thousands of steps its rounding
//            drifts), and the slot is released.
// Each product is three MMAs over a split of both operands into a TF32 head (rounded to nearest)
// and the FP32 remainder: a_h b_h + a_h b_l + a_l b_h, the dropped a_l b_l below 2^-22 of the
// product (the remainder itself is read as TF32, a relative 2^-11 of it).  Warp-level MMAs rather
// than tcgen05: a tcgen05 tile is 64 or 128 rows of the whole width (d <= 512), needed twice (as A
// and as A^T) and split in two, which does not fit in shared memory beside the ring; the pass is
// bound by HBM, and the MMAs take the multiply-adds and the per-row reductions off the SIMT pipes.
// ------------------------------------------------------------------------------------
constexpr int RKMAX = 9;  // k-steps of a stage-1 warp (checked over every width d <= 512)

__device__ __forceinline__ uint32_t tf32_head(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

__device__ __forceinline__ void mma_tf32(float (&dd)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(dd[0]), "+f"(dd[1]), "+f"(dd[2]), "+f"(dd[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void tf32_split4(const uint32_t (&a)[4], uint32_t (&h)[4], uint32_t (&l)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = tf32_head(__uint_as_float(a[i]));
    l[i] = __float_as_uint(__uint_as_float(a[i]) - __uint_as_float(h[i]));
  }
}

// Y[r][j] sits at r * 16 + (j ^ 8 ((r >> 1) & 1)): the B fragments of stage 2 (rows k8 + t, t < 4,
// columns 8 nt + g) then hit 32 distinct banks
__device__ __forceinline__ int y_at(int r, int j) { return r * 16 + (j ^ (((r >> 1) & 1) << 3)); }

template <int NT>
__device__ __forceinline__ int rp_chunk_mma(const BProb& pr, int64_t r0, int64_t r1, double* __restrict__ out,
                                            float* smf, uint64_t* full, uint64_t* empty, uint32_t gs,
                                            volatile int* s_err) {
  constexpr int KPAD = NT * 8;
  const int d = pr.d, dp = pr.dp, kp = pr.kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tq = lane & 3;
  float* ring = smf;
  float* ypart = smf + RNS * RSTAGE;
  float* yb = ypart + RYP;
  float* ysm = yb + RY;
  float* qf = ysm + RY;
  // tiling of a stage (the fragments read up to 20 floats past a stage's last row: still in the slot)
  const int nrt_max = min(128, (RSTAGE - 24) / d) >> 4;
  int nrt, KS;
  if (nrt_max >= 8) {
    nrt = nrt_max & ~7;
    KS = 1;
  } else {
    nrt = 1 << (31 - __clz(nrt_max));
    KS = RW / nrt;
  }
  const int R = nrt * 16;
  const int nst = (int)((r1 - r0 + R - 1) / R);
  const int kd = (d + 7) >> 3;
  const int kps = KS == 1 ? kd : (kd + KS - 1) / KS;
  const int nct = (d + 15) >> 4;
  // stage-1 role: row tiles rt1, rt1 + RW, ... (KS == 1) or the one tile rt1 (KS > 1); k-steps
  // k0 .. k0 + nk - 1
  const int ks = warp % KS, rt1 = warp / KS;
  const int k0 = ks * kps, nk = min(kps, kd - k0);
  // stage-2 role: column tiles ct0 + 8 i (i < ctw), row k-steps rsl, rsl + rspl, ...
  const int ctw = nct >= 8 ? (nct + 7) >> 3 : 1;
  const int rspl = nct >= 8 ? 1 : RW / nct;
  const int ct0 = nct >= 8 ? warp : warp % nct;
  const int rsl = nct >= 8 ? 0 : warp / nct;
  const bool act2 = rsl < rspl;
  const float* A = reinterpret_cast<const float*>(pr.A);
  int issued = 0;
  const bool prod = tid == 0;
  auto issue = [&](int t, bool released) {
    if (rp_issue(A, pr.n * d, d, r0, r1, R, t, gs, ring, full, empty, released)) ++issued;
    else *s_err = 1;
  };
  if (prod)
    for (int t = 0; t < nst && t < RNS - 1 && !*s_err; ++t) issue(t, false);
  // P fragments of this warp's k-steps, head and remainder: b0 = P[8 k + tq][8 nt + g],
  // b1 = P[8 k + tq + 4][..]; zero beyond d, so that the entries read there (the next row's, or
  // the zeros placed past the stage) add nothing
  uint32_t pbh[RKMAX][NT][2], pbl[RKMAX][NT][2];
#pragma unroll
  for (int kk = 0; kk < RKMAX; ++kk)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = (k0 + kk) * 8 + tq + 4 * h, j = nt * 8 + g;
        const float v = (kk < nk && c < d && j < pr.k) ? pr.Pf[c * kp + j] : 0.f;
        pbh[kk][nt][h] = tf32_head(v);
        pbl[kk][nt][h] = __float_as_uint(v - __uint_as_float(pbh[kk][nt][h]));
      }
  float vrun[4][NT][4];
#pragma unroll
  for (int ci = 0; ci < 4; ++ci)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) vrun[ci][nt][i] = 0.f;
  // q: KS == 1, this lane's columns 8 nt + 2 tq (+1) of its fragments; KS > 1, column tid % KPAD
  float qacc[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) qacc[nt][0] = qacc[nt][1] = 0.f;
  bool failed = false;
  for (int t = 0; t < nst; ++t) {
    const uint32_t gg = gs + (uint32_t)t;
    const int s = (int)(gg % RNS);
    const int64_t lo = r0 + (int64_t)t * R;
    const int nrows = (int)(min(r1, lo + R) - lo);
    const int64_t e_lo = lo * d;
    const float* raw = ring + s * RSTAGE + (int)(e_lo - (e_lo & ~(int64_t)3));
    const bool ok = __all_sync(0xffffffffu, !*s_err && rp_wait(full + s, (gg / RNS) & 1u));
    // ---- stage 1: Y tiles (rows past the stage's are stale: their Y is replaced by zeros)
    if (ok) {
      for (int rt = rt1; rt < nrt; rt += (KS == 1 ? RW : nrt)) {
        float dh[NT][4], d1[NT][4], d2[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int i = 0; i < 4; ++i) dh[nt][i] = d1[nt][i] = d2[nt][i] = 0.f;
        const float* pa = raw + (rt * 16 + g) * d + tq + k0 * 8;
        const float* pb = pa + 8 * d;
        // the next k-step's fragment is loaded before this one's MMAs are issued
        uint32_t an[4] = {0u, 0u, 0u, 0u};
        if (nk > 0) {
          an[0] = __float_as_uint(pa[0]);
          an[1] = __float_as_uint(pb[0]);
          an[2] = __float_as_uint(pa[4]);
          an[3] = __float_as_uint(pb[4]);
        }
#pragma unroll
        for (int kk = 0; kk < RKMAX; ++kk) {
          if (kk < nk) {
            const uint32_t a[4] = {an[0], an[1], an[2], an[3]};
            if (kk + 1 < nk) {
              an[0] = __float_as_uint(pa[kk * 8 + 8]);
              an[1] = __float_as_uint(pb[kk * 8 + 8]);
              an[2] = __float_as_uint(pa[kk * 8 + 12]);
              an[3] = __float_as_uint(pb[kk * 8 + 12]);
            }
            uint32_t ah[4], al[4];
            tf32_split4(a, ah, al);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              mma_tf32(dh[nt], ah, pbh[kk][nt][0], pbh[kk][nt][1]);
              mma_tf32(d1[nt], ah, pbl[kk][nt][0], pbl[kk][nt][1]);
              mma_tf32(d2[nt], al, pbh[kk][nt][0], pbh[kk][nt][1]);
            }
          }
        }
        if (KS == 1) {
          // the whole dot products: Y straight from the fragments (zero past the stage's rows)
          const int ra = rt * 16 + g, rb = ra + 8;
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int r = i < 2 ? ra : rb, j = nt * 8 + 2 * tq + (i & 1);
              const float y = r < nrows ? dh[nt][i] + (d1[nt][i] + d2[nt][i]) : 0.f;
              qacc[nt][i & 1] = fmaf(y, y, qacc[nt][i & 1]);
              const uint32_t h = tf32_head(y);
              yb[y_at(r, j)] = __uint_as_float(h);
              ysm[y_at(r, j)] = y - __uint_as_float(h);
            }
        } else {
          float* yp = ypart + (rt * KS + ks) * 256;
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            *reinterpret_cast<float2*>(yp + g * 16 + nt * 8 + 2 * tq) =
                make_float2(dh[nt][0] + (d1[nt][0] + d2[nt][0]), dh[nt][1] + (d1[nt][1] + d2[nt][1]));
            *reinterpret_cast<float2*>(yp + (g + 8) * 16 + nt * 8 + 2 * tq) =
                make_float2(dh[nt][2] + (d1[nt][2] + d2[nt][2]), dh[nt][3] + (d1[nt][3] + d2[nt][3]));
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) {  // one decision for the whole CTA
      failed = true;
      break;
    }
    // every warp is past stage 2 of stage t - 1: its slot takes stage t + RNS - 1 without a wait
    if (prod && t + RNS - 1 < nst && !*s_err) issue(t + RNS - 1, t >= 1);
    if (KS > 1) {
      // ---- Y: the KS partial tiles in order; q; the split for stage 2
      for (int e = tid; e < R * KPAD; e += RT) {
        const int r = e / KPAD, j = e - r * KPAD;
        const float* yp = ypart + (r >> 4) * KS * 256 + (r & 15) * 16 + j;
        float y = 0.f;
        for (int k2 = 0; k2 < KS; ++k2) y += yp[k2 * 256];
        if (r >= nrows) y = 0.f;
        qacc[0][0] = fmaf(y, y, qacc[0][0]);
        const uint32_t h = tf32_head(y);
        yb[y_at(r, j)] = __uint_as_float(h);
        ysm[y_at(r, j)] = y - __uint_as_float(h);
      }
      __syncthreads();
    }
    // ---- stage 2: V_stage = A^T Y (columns past d give rows of V that are not written out), added
    // to the running V; then the slot is released
    if (act2) {
      float vh[4][NT][4], vx[4][NT][4];
#pragma unroll
      for (int ci = 0; ci < 4; ++ci)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int i = 0; i < 4; ++i) vh[ci][nt][i] = vx[ci][nt][i] = 0.f;
      for (int kr = rsl; kr < R / 8; kr += rspl) {
        const int rr = kr * 8 + tq;
        uint32_t ybh[NT][2], ybl[NT][2];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int j = nt * 8 + g;
          ybh[nt][0] = __float_as_uint(yb[y_at(rr, j)]);
          ybh[nt][1] = __float_as_uint(yb[y_at(rr + 4, j)]);
          ybl[nt][0] = __float_as_uint(ysm[y_at(rr, j)]);
          ybl[nt][1] = __float_as_uint(ysm[y_at(rr + 4, j)]);
        }
        // rows past the stage's are stale (zero Y rows would not cancel a non-finite entry)
        const bool ina = rr < nrows, inb = rr + 4 < nrows;
        const float* alo = raw + rr * d + g + ct0 * 16;
        const float* ahi = alo + 4 * d;
#pragma unroll
        for (int ci = 0; ci < 4; ++ci) {
          if (ci < ctw && ct0 + 8 * ci < nct) {
            const int c = ci * 128;
            const uint32_t a[4] = {__float_as_uint(ina ? alo[c] : 0.f), __float_as_uint(ina ? alo[c + 8] : 0.f),
                                   __float_as_uint(inb ? ahi[c] : 0.f), __float_as_uint(inb ? ahi[c + 8] : 0.f)};
            uint32_t ah[4], al[4];
            tf32_split4(a, ah, al);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              mma_tf32(vh[ci][nt], ah, ybh[nt][0], ybh[nt][1]);
              mma_tf32(vx[ci][nt], ah, ybl[nt][0], ybl[nt][1]);
              mma_tf32(vx[ci][nt], al, ybh[nt][0], ybh[nt][1]);
            }
          }
        }
      }
#pragma unroll
      for (int ci = 0; ci < 4; ++ci)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int i = 0; i < 4; ++i) vrun[ci][nt][i] += vh[ci][nt][i] + vx[ci][nt][i];
    }
    __syncwarp();
    if (lane == 0) rp_arrive(empty + s);
    // the next stage's stage 1 writes Y only after this stage's readers have passed the next
    // barrier (KS == 1: the Y writes of stage t + 1 come before that barrier -- so a barrier here)
    if (KS == 1) __syncthreads();
  }
  if (failed) {
    if (tid == 0) *s_err = 1;
    if (prod)
      for (int t = issued > RNS ? issued - RNS : 0; t < issued; ++t) {
        const uint32_t gg = gs + (uint32_t)t;
        rp_wait(full + gg % RNS, (gg / RNS) & 1u);
      }
    __syncthreads();
    return nst;
  }
  __syncthreads();  // every stage has been read: the ring is free for the reduction
  // ---- V partials (FP64) of the row slices in the ring; q per thread
  double* red = reinterpret_cast<double*>(ring);
  if (act2) {
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
      const int ct = ct0 + 8 * ci;
      if (ci < ctw && ct < nct) {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int c = ct * 16 + g, j = nt * 8 + 2 * tq;
          double* rb = red + (size_t)(rsl * KPAD + j) * dp + c;
          rb[0] = (double)vrun[ci][nt][0];
          rb[dp] = (double)vrun[ci][nt][1];
          rb[8] = (double)vrun[ci][nt][2];
          rb[dp + 8] = (double)vrun[ci][nt][3];
        }
      }
    }
  }
  if (KS == 1) {
    // per-lane q of columns 8 nt + 2 tq (+1): into qf[j * 32 + lane-slot] as warp sums
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v = qacc[nt][h];
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (g == 0) qf[warp * 16 + nt * 8 + 2 * tq + h] = v;  // lanes 0..3: this warp's sum for j
      }
  } else {
    qf[tid] = qacc[0][0];
  }
  __syncthreads();
  for (int e = tid; e < kp * dp; e += RT) {
    const int j = e / dp, c = e - j * dp;
    double sum = 0.0;
    if (c < d)
      for (int q2 = 0; q2 < rspl; ++q2) sum += red[(size_t)(q2 * KPAD + j) * dp + c];
    out[e] = sum;
  }
  if (tid < kp) {
    double sum = 0.0;
    if (KS == 1)
      for (int w2 = 0; w2 < RW; ++w2) sum += (double)qf[w2 * 16 + tid];
    else
      for (int i = tid; i < RT; i += KPAD) sum += (double)qf[i];
    out[kp * dp + tid] = sum;
  }
  __syncthreads();
  // the ring again holds only finite floats: zero the reduction area
  {
    float4* z = reinterpret_cast<float4*>(ring);
    const int n4 = (int)(((size_t)rspl * KPAD * dp * 2 + 3) / 4);
    for (int i = tid; i < n4; i += RT) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  rp_fence_async();  // the reduction area's reads and writes come before the next copies into it
  __syncthreads();
  return nst;
}

// FP32 passes on the tensor cores (one or two 8-column tiles of right-hand sides); exact passes
// by the SIMT schedule with (EPL, JG): EPL columns per lane (dp / EPL lanes per row), JG
// right-hand sides per warp, sized so that a lane's operand and accumulator registers (4 EPL JG
// floats in double-FP32) stay within the budget of one CTA per SM
__device__ __forceinline__ int rp_run(const BProb& pr, int64_t r0, int64_t r1, double* out, bool exact, float* ring,
                                      uint64_t* full, uint64_t* empty, uint32_t gs,
                                      volatile int* s_err) {
  const int dp = pr.dp, kp = pr.kp;
#define RP_CALL(E, G) return rp_chunk_exact<E, G>(pr, r0, r1, out, ring, full, empty, gs, s_err)
  if (!exact) return kp <= 8 ? rp_chunk_mma<1>(pr, r0, r1, out, ring, full, empty, gs, s_err)
                            : rp_chunk_mma<2>(pr, r0, r1, out, ring, full, empty, gs, s_err);
  if (dp <= 128) {
    switch (kp) {
      case 4: RP_CALL(4, 4);
      case 12: RP_CALL(4, 6);
      default: RP_CALL(4, 8);
    }
  }
  if (dp == 256) {
    if (kp == 12) RP_CALL(8, 3);
    RP_CALL(8, 4);
  }
  RP_CALL(16, 2);
#undef RP_CALL
}

// The pass: CTAs take chunks from the iteration's queue (costliest first), as bpass_kernel does.
__global__ void __launch_bounds__(RT, 1) bpass_ring_kernel(BatchArgs a, int force_exact) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[RNS], empty[RNS];
  __shared__ int next;
  __shared__ volatile int s_err;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RNS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(lsq_apass::smem_u32a(full + s)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(lsq_apass::smem_u32a(empty + s)), "r"(RW)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_err = 0;
  }
  float* ring = reinterpret_cast<float*>(smem);
  // every float of the shared memory starts finite (zero): the tensor-core pass reads a little
  // past a stage's rows and multiplies what it finds there by zeros
  for (int i = threadIdx.x; i < (int)(RSMEM / 16); i += RT)
    reinterpret_cast<float4*>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  rp_fence_async();
  __syncthreads();
  const int it = *(volatile int*)a.iter;
  int* head = a.qhead + it % 3;
  uint32_t gs = 0;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(head, 1);
    __syncthreads();
    const int u = next;
    __syncthreads();
    if (u >= a.nchunks) break;
    const int ch = a.order[u];
    const int4 cd = a.chunks[ch];
    const BProb& pr = a.probs[cd.x];
    if (!prob_active(pr, it)) continue;
    const bool exact = force_exact != 0 || exact_step(pr, it);
    gs += (uint32_t)rp_run(pr, cd.y, cd.z, a.part + a.part_off[ch], exact, ring, full, empty, gs, &s_err);
    if (s_err) {
      if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)LSQ_ERR_TIMEOUT);
      break;
    }
  }
}
