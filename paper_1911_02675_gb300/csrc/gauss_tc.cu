// gauss_tc.cu -- Gaussian sketch SA = S A on the 5th-generation tensor cores (tcgen05),
// BF16 operands and FP32 accumulation in tensor memory (Section 2: a Gaussian embedding is
// a dense m x n matrix, so S A is a true dense contraction).
//
// A CTA owns a 128 x NT tile of SA (NT = 256 or 512 accumulator columns in TMEM) and a
// contiguous range of rows of A (split-K).  Per stage of 64 rows:
//   * all threads generate the 128 x 64 tile of S from Philox4x32-10 + Box-Muller (FP32,
//     rounded to BF16) and narrow the 64 x NT tile of A to BF16, writing both into shared
//     memory in the canonical K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per
//     core matrix; K-adjacent core matrices 128 bytes apart, 8-row groups 256 bytes apart);
//   * one thread issues the tcgen05.mma instructions (M = 128, N = 256, K = 16 each) and
//     commits them to the stage's mbarrier, which the producers wait on (bounded) before
//     they overwrite the stage.
// The epilogue reads the accumulator with tcgen05.ld and writes FP32 partials; a fixed-order
// reduction over the splits (sketch.cu) scales by 1/sqrt(m) and writes SA in FP64.
// S is never stored in global memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "apass.cuh"
#include "common.cuh"

namespace {

constexpr int TC_M = 128;
constexpr int TC_KS = 64;  // rows of A per stage (4 MMAs of K = 16)
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_SPIN = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; on time-out records the error and returns false
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > TC_SPIN) {
      atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// descriptor version 1 (bits 46..48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24
constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// z(j, i) pair for j = 2q (cosine) and 2q + 1 (sine) in FP32, from the same Philox words as
// the FP64 definition; the uniforms keep the top 24 of their 53 bits (BF16 keeps 8)
__device__ __forceinline__ void gauss_pair_f32(uint64_t seed, uint32_t i, uint32_t q, uint32_t t, float& zc,
                                               float& zs) {
  const uint4 w = philox_at(seed, i, q, t, TAG_GAUSS);
  const float u1 = __fmaf_rn((float)(w.x >> 8), 0x1p-24f, 0x1p-25f);
  const float u2 = __fmaf_rn((float)(w.z >> 8), 0x1p-24f, 0x1p-25f);
  const float rad = sqrtf(-2.0f * __logf(u1));
  float s, c;
  __sincosf(6.28318530717958647692f * u2, &s, &c);
  zc = rad * c;
  zs = rad * s;
}

// byte offset of element (row r, k) of a K-major operand tile with R rows and TC_KS columns
// (K-step kk = k / 16 occupies R * 32 bytes)
__device__ __forceinline__ uint32_t core_offset(int R, int r, int kgroup) {
  const int kk = kgroup >> 1, kc = kgroup & 1;  // 8-wide K groups: 2 per K-step
  return (uint32_t)(kk * R * 32 + (r >> 3) * 256 + kc * 128 + (r & 7) * 16);
}

template <typename TA, int NT, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) gauss_tc_kernel(const TA* __restrict__ A, int64_t n, int d,
                                                                 int64_t ld, int m, uint64_t seed, uint32_t t,
                                                                 int64_t rows_per_split, float* __restrict__ part,
                                                                 int* err) {
  constexpr int A_BYTES = TC_M * TC_KS * 2;
  constexpr int B_BYTES = NT * TC_KS * 2;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, 256);
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  __shared__ __align__(8) uint64_t mbar[STAGES];
  __shared__ uint32_t tmem_base_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * TC_M, c0 = blockIdx.y * NT;
  const int64_t i_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t i_end = min(n, i_begin + rows_per_split);
  const int64_t nsteps = i_end > i_begin ? (i_end - i_begin + TC_KS - 1) / TC_KS : 0;

  if (warp == 0) tmem_alloc(&tmem_base_s, NT);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  bool ok = true;

  for (int64_t step = 0; step < nsteps && ok; ++step) {
    const int s = (int)(step % STAGES);
    if (step >= STAGES) {
      // the MMAs that read this stage STAGES steps ago have completed
      ok = mbar_wait_bounded(&mbar[s], (uint32_t)(((step / STAGES) - 1) & 1), err);
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
    }
    const int64_t k0 = i_begin + step * TC_KS;
    uint8_t* stA = sA + s * A_BYTES;
    uint8_t* stB = sB + s * B_BYTES;
    // S tile: 64 pairs of sketch rows x 8 groups of 8 rows of A
    for (int u = tid; u < (TC_M / 2) * (TC_KS / 8); u += TC_THREADS) {
      const int jp = u >> 3, kg = u & 7;
      uint32_t ev[4], od[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        float c_a = 0.f, s_a = 0.f, c_b = 0.f, s_b = 0.f;
        const int64_t ia = k0 + kg * 8 + q;
        if (ia < i_end) gauss_pair_f32(seed, (uint32_t)ia, (uint32_t)((j0 >> 1) + jp), t, c_a, s_a);
        if (ia + 1 < i_end) gauss_pair_f32(seed, (uint32_t)(ia + 1), (uint32_t)((j0 >> 1) + jp), t, c_b, s_b);
        ev[q >> 1] = pack_bf16(c_a, c_b);
        od[q >> 1] = pack_bf16(s_a, s_b);
      }
      *reinterpret_cast<uint4*>(stA + core_offset(TC_M, 2 * jp, kg)) = make_uint4(ev[0], ev[1], ev[2], ev[3]);
      *reinterpret_cast<uint4*>(stA + core_offset(TC_M, 2 * jp + 1, kg)) = make_uint4(od[0], od[1], od[2], od[3]);
    }
    // A tile: NT columns x 8 groups of 8 rows, narrowed to BF16
    for (int u = tid; u < NT * (TC_KS / 8); u += TC_THREADS) {
      const int nn = u % NT, kg = u / NT;
      const int col = c0 + nn;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t i = k0 + kg * 8 + q;
        v[q] = (i < i_end && col < d) ? lsq_apass::narrow_f32(__ldg(A + i * ld + col)) : 0.f;
      }
      *reinterpret_cast<uint4*>(stB + core_offset(NT, nn, kg)) =
          make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
    // generic-proxy writes -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < TC_KS / 16; ++kk) {
        const uint64_t ad = smem_desc(smem_u32(stA + kk * TC_M * 32), 128, 256);
#pragma unroll
        for (int h = 0; h < NT / 256; ++h) {
          const uint64_t bd = smem_desc(smem_u32(stB + kk * NT * 32 + h * (256 / 8) * 256), 128, 256);
          mma_bf16(tmem + h * 256, ad, bd, IDESC, (step > 0 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(&mbar[s]);
    }
  }
  // all MMAs done: the last commit tracks every earlier one
  if (ok && nsteps > 0) {
    const int64_t last = nsteps - 1;
    ok = mbar_wait_bounded(&mbar[last % STAGES], (uint32_t)((last / STAGES) & 1), err);
  }
  ok = !__syncthreads_or(!ok);
  tc_fence_after();
  if (warp < 4) {
    const int j = j0 + 32 * warp + lane;
    float* out = part + (int64_t)blockIdx.z * m * d;
    for (int cb = 0; cb < NT; cb += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, r);
      if (j < m) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int col = c0 + cb + q;
          if (col < d) out[(int64_t)j * d + col] = (ok && nsteps > 0) ? __uint_as_float(r[q]) : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NT);
}

}  // namespace

// entry from sketch.cu: FP32 partials [splits][m][d] of the Gaussian sketch (unscaled)
lsq_status lsq_gauss_tc_partials(lsq_ctx* ctx, const lsq_matrix* A, int m, uint64_t seed, uint32_t t, float* part,
                                 int splits, int64_t rows_per_split, int nt, int* err) {
  const int d = (int)A->d;
  const int gx = (m + TC_M - 1) / TC_M, gy = (d + nt - 1) / nt;
  dim3 grid(gx, gy, splits);
  if (nt == 512) {
    constexpr int STAGES = 2;
    const size_t smem = (size_t)STAGES * (TC_M * TC_KS * 2 + 512 * TC_KS * 2);
    if (A->dtype == LSQ_F64) {
      auto k = gauss_tc_kernel<double, 512, STAGES>;
      LSQ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<grid, TC_THREADS, smem, ctx->stream>>>(reinterpret_cast<const double*>(A->data), A->n, d, A->ld, m, seed, t,
                                                 rows_per_split, part, err);
    } else {
      auto k = gauss_tc_kernel<float, 512, STAGES>;
      LSQ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<grid, TC_THREADS, smem, ctx->stream>>>(reinterpret_cast<const float*>(A->data), A->n, d, A->ld, m, seed, t,
                                                 rows_per_split, part, err);
    }
  } else {
    constexpr int STAGES = 3;
    const size_t smem = (size_t)STAGES * (TC_M * TC_KS * 2 + 256 * TC_KS * 2);
    if (A->dtype == LSQ_F64) {
      auto k = gauss_tc_kernel<double, 256, STAGES>;
      LSQ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<grid, TC_THREADS, smem, ctx->stream>>>(reinterpret_cast<const double*>(A->data), A->n, d, A->ld, m, seed, t,
                                                 rows_per_split, part, err);
    } else {
      auto k = gauss_tc_kernel<float, 256, STAGES>;
      LSQ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<grid, TC_THREADS, smem, ctx->stream>>>(reinterpret_cast<const float*>(A->data), A->n, d, A->ld, m, seed, t,
                                                 rows_per_split, part, err);
    }
  }
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}
