// gauss_tc.cu -- Gaussian sketch SA = S A on the 5th-generation tensor cores (tcgen05),
// BF16 operands and FP32 accumulation in tensor memory (Section 2: a Gaussian embedding is
// a dense m x n matrix, so S A is a true dense contraction).
//
// Two kernels per chunk of rows of A:
//   * pack_kernel narrows the chunk to BF16 and writes it in the tensor core's canonical
//     K-major, no-swizzle core-matrix layout, one contiguous blob of 64 rows x NT columns
//     per (64-row block, column tile): core matrices of 8 columns x 8 rows (16 bytes per
//     column), K-adjacent core matrices 128 bytes apart, 8-column groups 256 bytes apart,
//     16-row K-steps NT * 32 bytes apart.  A blob is then one bulk copy (cp.async.bulk).
//   * gauss_tc_kernel: a CTA owns a 128 x NT tile of SA (NT = 256 or 512 FP32 accumulator
//     columns in TMEM) and a contiguous range of 64-row blocks (split-K).  Per stage, one
//     thread starts the bulk copy of the blob into shared memory (completion counted in
//     bytes on the stage's `full` mbarrier) while every thread generates the 128 x 64 tile
//     of S from Philox4x32-10 + Box-Muller (FP32, rounded to BF16) in the same layout; then
//     one thread issues the tcgen05.mma instructions (M = 128, N = 256, K = 16) and
//     commits them to the stage's `empty` mbarrier, which the generators wait on before
//     they overwrite the stage.  Every wait is bounded and records LSQ_ERR_TIMEOUT.
// The epilogue reads the accumulator with tcgen05.ld and adds it into FP32 partials per
// split; a fixed-order reduction over the splits scales by 1/sqrt(m) and writes SA in FP64.
// S is never stored in global memory.
//
// Sketch rows j0 + 2 q' (cosine of pair q') sit in tile row q', rows j0 + 2 q' + 1 (sine)
// in tile row q' + 64, so that one thread's Philox call fills both halves and a warp's
// shared stores cover 512 contiguous bytes.
#include <cuda_bf16.h>

#include <algorithm>

#include "apass.cuh"
#include "common.cuh"

namespace {

constexpr int TC_M = 128;
constexpr int TC_KS = 64;  // rows of A per stage (4 MMAs of K = 16)
constexpr uint32_t TC_SPIN = 1u << 26;
constexpr int TC_GEN = 512;  // generating threads

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

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// one bulk global -> shared copy (16-byte aligned ends, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
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

__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait with cluster-scope acquire (the arrivals include other CTAs' releases)
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity, int* err) {
  uint32_t spins = 0;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (++spins > TC_SPIN) {
      atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      return false;
    }
  }
}

// bulk copy of `bytes` from this CTA's shared memory to a shared::cluster address (another
// CTA of the cluster), completion counted on the mbarrier at `bar` (shared::cluster)
__device__ __forceinline__ void bulk_s2peer(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "r"(smem_u32(src)), "r"(bytes), "r"(bar)
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

// Philox4x32-10 with the ten round keys computed once per thread (the same function as
// philox4x32_10: key k_r = k_0 + r * increment)
struct RoundKeys {
  uint32_t a[10], b[10];
};

__device__ __forceinline__ RoundKeys round_keys(uint64_t seed) {
  RoundKeys k;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    k.a[r] = k0;
    k.b[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return k;
}

// one Philox4x32 round (multipliers 0xD2511F53, 0xCD9E8D57) with round key (ka, kb)
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t ka, uint32_t kb) {
  const uint32_t lo0 = 0xD2511F53u * c.x;
  const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
  const uint32_t lo1 = 0xCD9E8D57u * c.z;
  const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
  return make_uint4(hi1 ^ c.y ^ ka, lo1, hi0 ^ c.w ^ kb, lo0);
}

// byte offset of element (row r, k-group kg of 8) of a K-major operand tile with R rows and
// TC_KS columns (K-step kk = kg / 2 occupies R * 32 bytes)
__host__ __device__ __forceinline__ uint32_t core_offset(int R, int r, int kgroup) {
  const int kk = kgroup >> 1, kc = kgroup & 1;
  return (uint32_t)(kk * R * 32 + (r >> 3) * 256 + kc * 128 + (r & 7) * 16);
}

// ------------------------------------------------------------------------------------
// Rows [row0, row0 + rows) of A -> BF16 blobs; blob (kb, ct) at byte ((kb * nct + ct) * NT * 128).
// Unit = 8 consecutive rows of one column (one 16-byte store); zero outside n x d.
// ------------------------------------------------------------------------------------
template <typename TA>
__global__ void __launch_bounds__(256) pack_kernel(const TA* __restrict__ A, int64_t n, int d, int64_t ld,
                                                   int64_t row0, int64_t nkb, int nt, int nct,
                                                   uint8_t* __restrict__ out) {
  const int dpad = nt * nct;
  const int64_t units = nkb * 8 * (int64_t)dpad;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(u % dpad);
    const int64_t rest = u / dpad;
    const int kg = (int)(rest & 7);
    const int64_t kb = rest >> 3;
    const int64_t i0 = row0 + kb * TC_KS + kg * 8;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t i = i0 + q;
      v[q] = (i < n && c < d) ? lsq_apass::narrow_f32(__ldg(A + i * ld + c)) : 0.f;
    }
    const int ct = c / nt, nn = c - ct * nt;
    uint8_t* blob = out + ((size_t)kb * nct + ct) * (size_t)nt * 128;
    *reinterpret_cast<uint4*>(blob + core_offset(nt, nn, kg)) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  }
}

// Warp roles: warps 0..15 generate S, warp 16 starts the bulk copies of A's blobs and issues
// the MMAs (one elected lane; the whole warp waits).  Stage s is handed over through mbarriers:
// `full` (the blob landed, bytes counted), `gen` (every generating warp of this CTA wrote its
// part of S and fenced it for the async proxy), `sfull` (CL = 2: the other CTA's half of S
// landed, bytes counted) and `empty` (the MMAs that read the stage completed, one commit per
// CTA of the cluster).  No CTA-wide barrier runs inside the loop.  CL = 2: the two CTAs of a
// cluster own adjacent column tiles of the same rows of SA, so they need the same S; CTA r
// generates the K-steps 2r and 2r + 1 of each stage (one contiguous 8 KB half) and sends it
// to the other CTA with one shared-to-shared bulk copy, so S is generated once per row tile.
//
// SJ = true: the same product with S an SJLT (Section 2, last paragraph) instead: column i of S
// holds s entries +-1 (exact in BF16; the 1/sqrt(s) scale is applied in FP64 by the reduction)
// at the rows the hash pass drew (hsj[i * s + k], sign bit k of ssj[i]; i the row of A).  Warp
// w owns tile rows 8w .. 8w + 7: per stage it zeroes them and writes the entries that land
// there, so no warp waits on another.  Every product is exact and the FP32 accumulation runs
// in a fixed order, so the sketch repeats bit for bit.
template <int NT, int STAGES, int BS, int CL, bool SJ>
__global__ void __launch_bounds__(TC_GEN + 64, 1)
    gauss_tc_kernel(const uint8_t* __restrict__ pk, int64_t nkb, int nct, int d, int m, uint64_t seed, uint32_t t,
                    int64_t row0, int64_t kb_per_split, int accumulate, float* __restrict__ part, int* err,
                    const int32_t* __restrict__ hsj, const uint32_t* __restrict__ ssj, int s_sj, int64_t n_rows) {
  constexpr int A_BYTES = TC_M * TC_KS * 2;
  constexpr int B_BYTES = NT * TC_KS * 2;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, 256);
  constexpr int UNITS = (TC_M / 2) * (TC_KS / 8);  // 512 (pair of rows, k-group) per stage
  constexpr int PER = 8 / CL;                      // K-columns of a unit this CTA generates
  constexpr int GW = TC_GEN / 32;                  // generating warps
  static_assert(CL == 1 || CL == 2, "a single CTA or a CTA pair");
  static_assert(UNITS == TC_GEN, "one unit (or two half units) per generating thread and stage");
  constexpr uint32_t HALF_A = A_BYTES / 2;        // one CTA's part of a stage of S (CL = 2)
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;  // BS slots of the B operand (blobs of A)
  __shared__ __align__(8) uint64_t full[BS];
  __shared__ __align__(8) uint64_t bempty[BS];  // this CTA's MMAs that read the B slot are done
  __shared__ __align__(8) uint64_t gen[STAGES];
  __shared__ __align__(8) uint64_t sfull[STAGES];
  __shared__ __align__(8) uint64_t empty[STAGES];
  __shared__ __align__(8) uint64_t zeroed[STAGES];  // SJ: every generating warp zeroed its rows
  __shared__ uint32_t tmem_base_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * TC_M, ct = blockIdx.y;
  const int64_t kb_begin = (int64_t)blockIdx.z * kb_per_split;
  const int64_t kb_end = min(nkb, kb_begin + kb_per_split);
  const int64_t nsteps = kb_end > kb_begin ? kb_end - kb_begin : 0;
  const uint32_t rank = CL > 1 ? cluster_rank() : 0u;

  if (warp == 0) tmem_alloc(&tmem_base_s, NT);
  if (tid == 0) {
    for (int b = 0; b < BS; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&bempty[b], 1);
    }
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&gen[s], GW);
      mbar_init(&sfull[s], 1);
      mbar_init(&empty[s], CL);
      mbar_init(&zeroed[s], GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  // every CTA of the cluster has initialised its barriers before any remote access
  if (CL > 1) cluster_sync_all();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  bool ok = true;
  int64_t copies = 0;  // bulk copies of blobs started (MMA warp)
  int64_t armed = 0;   // CL = 2: stages armed for the other CTA's half of S (exchange warp)

  if (SJ && warp < GW) {
    // ---- SJLT generators.  Per stage: warp w zeroes tile rows 8w .. 8w + 7 of this CTA's
    // K-columns, the warps meet on the stage's `zeroed` mbarrier (bounded), then each lane
    // writes its (K-column, target) pairs, whose target rows and signs it loaded a stage ahead
    constexpr int KC = TC_KS / CL;                 // K-columns of a stage this CTA writes
    constexpr int PMAX = KC * 32 / TC_GEN;         // pairs per lane at s = 32 (4 or 2)
    const int kc0 = CL == 1 ? 0 : KC * (int)rank;  // first of them
    const int npairs = KC * s_sj;
    const uint16_t plus = 0x3F80u, minus = 0xBF80u;  // BF16 +1, -1
    int32_t tgt[PMAX];
    uint16_t val[PMAX];
    // pair p of the stage: K-column p / s, target p % s; this thread takes p = tid + TC_GEN q
    auto fetch = [&](int64_t step) {
      const int64_t ib = (row0 + (kb_begin + step) * TC_KS) + kc0;  // row of A of K-column kc0
#pragma unroll
      for (int q = 0; q < PMAX; ++q) {
        const int p = tid + TC_GEN * q;
        tgt[q] = -1;
        if (step < nsteps && p < npairs) {
          const int k = p / s_sj, e = p - k * s_sj;
          const int64_t i = ib + k;
          if (i < n_rows) {
            const int off = __ldg(hsj + i * s_sj + e) - j0;
            if (off >= 0 && off < TC_M) {
              const int L = (off & 1) ? 64 + (off >> 1) : (off >> 1);  // the tile row of sketch row j0 + off
              const int kcol = kc0 + k;
              tgt[q] = (int32_t)(core_offset(TC_M, L, kcol >> 3) + (kcol & 7) * 2);
              val[q] = ((__ldg(ssj + i) >> e) & 1u) ? minus : plus;
            }
          }
        }
      }
    };
    fetch(0);
    for (int64_t step = 0; step < nsteps; ++step) {
      const int s = (int)(step % STAGES);
      const uint32_t par = (uint32_t)((step / STAGES) & 1);
      if (step >= STAGES &&
          !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((step / STAGES) - 1) & 1), err))) {
        ok = false;
        break;
      }
      uint8_t* stA = sA + s * A_BYTES;
      // rows 8w .. 8w + 7 of K-step kk form 256 contiguous bytes at kk * TC_M * 32 + w * 256
      for (int b = lane; b < (KC / 16) * 16; b += 32) {
        const int kk = (kc0 >> 4) + (b >> 4);
        *reinterpret_cast<uint4*>(stA + kk * TC_M * 32 + warp * 256 + (b & 15) * 16) = make_uint4(0u, 0u, 0u, 0u);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&zeroed[s]);
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&zeroed[s], par, err))) {
        ok = false;
        break;
      }
#pragma unroll
      for (int q = 0; q < PMAX; ++q)
        if (tgt[q] >= 0) *reinterpret_cast<uint16_t*>(stA + tgt[q]) = val[q];
      fetch(step + 1);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&gen[s]);
    }
  } else if (!SJ && warp < GW) {
    // ---- generators
    const RoundKeys keys = round_keys(seed);
    // CL = 1: thread -> unit (row pair jp, k-group kg), a warp's stores fill 512 contiguous
    // bytes.  CL = 2: thread -> half unit (k-values 4 hq .. 4 hq + 3) of the 256 units of this
    // CTA's K-steps 2 rank, 2 rank + 1; a warp's 8-byte stores fill 256 contiguous bytes.
    const int u = CL == 1 ? tid : tid >> 1, hq = CL == 1 ? 0 : tid & 1;
    const int ln = u & 31, blk = u >> 5;
    const int kk = CL == 1 ? (blk & 3) : 2 * (int)rank + (blk & 1);
    const int gpair = CL == 1 ? blk >> 2 : blk >> 1;
    const int r8 = ln & 7, kc = (ln >> 3) & 1, gsub = ln >> 4;
    const int jp = 8 * (2 * gpair + gsub) + r8;
    const int kg = 2 * kk + kc;
    const uint32_t qq = (uint32_t)((j0 >> 1) + jp);
    const uint32_t off_e = core_offset(TC_M, jp, kg) + hq * (PER * 2);
    const uint32_t off_o = core_offset(TC_M, jp + 64, kg) + hq * (PER * 2);
    for (int64_t step = 0; step < nsteps; ++step) {
      const int s = (int)(step % STAGES);
      // the MMAs (of every CTA of the cluster) that read this stage STAGES steps ago are done
      // (the warp decides together, so that it stays converged)
      if (step >= STAGES &&
          !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((step / STAGES) - 1) & 1), err))) {
        ok = false;
        break;
      }
      uint8_t* stA = sA + s * A_BYTES;
      // z(2q, i) (cosine) and z(2q + 1, i) (sine) in FP32 from the same Philox words as the
      // FP64 definition (the uniforms keep the top 24 of their 53 bits; BF16 keeps 8); the
      // PER Philox streams of the unit advance round by round together
      const uint32_t ia0 = (uint32_t)(row0 + (kb_begin + step) * TC_KS) + (uint32_t)(kg * 8) + hq * PER;
      uint4 w[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) w[q] = make_uint4(ia0 + (uint32_t)q, qq, t, TAG_GAUSS);
#pragma unroll
      for (int r = 0; r < 10; ++r) {
#pragma unroll
        for (int q = 0; q < PER; ++q) w[q] = philox_round(w[q], keys.a[r], keys.b[r]);
      }
      uint32_t ev[PER / 2], od[PER / 2];
#pragma unroll
      for (int q = 0; q < PER; q += 2) {
        float zc[2], zs[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float u1 = __fmaf_rn((float)(w[q + h].x >> 8), 0x1p-24f, 0x1p-25f);
          const float u2 = __fmaf_rn((float)(w[q + h].z >> 8), 0x1p-24f, 0x1p-25f);
          const float rad = sqrtf(-2.0f * __logf(u1));
          float sn, cs;
          __sincosf(6.28318530717958647692f * u2, &sn, &cs);
          zc[h] = rad * cs;
          zs[h] = rad * sn;
        }
        ev[q >> 1] = pack_bf16(zc[0], zc[1]);
        od[q >> 1] = pack_bf16(zs[0], zs[1]);
      }
      if constexpr (CL == 1) {
        *reinterpret_cast<uint4*>(stA + off_e) = make_uint4(ev[0], ev[1], ev[2], ev[3]);
        *reinterpret_cast<uint4*>(stA + off_o) = make_uint4(od[0], od[1], od[2], od[3]);
      } else {
        *reinterpret_cast<uint2*>(stA + off_e) = make_uint2(ev[0], ev[1]);
        *reinterpret_cast<uint2*>(stA + off_o) = make_uint2(od[0], od[1]);
      }
      // generic-proxy writes -> visible to the async proxy (tensor core, bulk copy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&gen[s]);
    }
  } else if (warp == GW) {
    // ---- copies and MMAs: the whole warp waits, lane 0 issues.  The B operand has a ring of its
    // own (BS slots): blob k + BS - 1 is copied into the slot of blob k - 1 right after the MMAs of
    // step k are issued and those of step k - 1 are done, so a copy has BS - 1 steps of MMAs to
    // land.  The S slots are the generators' and the exchange warp's to wait for.
    auto blob = [&](int64_t k) { return pk + ((size_t)(kb_begin + k) * nct + ct) * (size_t)B_BYTES; };
    for (int64_t k = 0; k < nsteps && k < BS; ++k) {
      if (lane == 0) {
        mbar_expect_tx(&full[k], (uint32_t)B_BYTES);
        bulk_g2s(sB + k * B_BYTES, blob(k), (uint32_t)B_BYTES, &full[k]);
      }
      ++copies;
    }
    for (int64_t step = 0; step < nsteps; ++step) {
      const int s = (int)(step % STAGES);
      const int b = (int)(step % BS);
      uint8_t* stA = sA + s * A_BYTES;
      uint8_t* stB = sB + b * B_BYTES;
      const uint32_t par = (uint32_t)((step / STAGES) & 1);
      bool got = mbar_wait_bounded(&gen[s], par, err);
      // CL = 2: the other CTA's half of S, sent by its exchange warp
      if constexpr (CL > 1) got = got && mbar_wait_cluster_bounded(&sfull[s], par, err);
      got = got && mbar_wait_bounded(&full[b], (uint32_t)((step / BS) & 1), err);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      if (lane == 0) {
        tc_fence_after();
#pragma unroll
        for (int k2 = 0; k2 < TC_KS / 16; ++k2) {
          const uint64_t ad = smem_desc(smem_u32(stA + k2 * TC_M * 32), 128, 256);
#pragma unroll
          for (int h = 0; h < NT / 256; ++h) {
            const uint64_t bd = smem_desc(smem_u32(stB + k2 * NT * 32 + h * (256 / 8) * 256), 128, 256);
            mma_bf16(tmem + h * 256, ad, bd, IDESC, (step > 0 || k2 > 0) ? 1u : 0u);
          }
        }
        if constexpr (CL > 1) mma_commit_mc(&empty[s], (uint16_t)((1u << CL) - 1u));
        else mma_commit(&empty[s]);
        mma_commit(&bempty[b]);
      }
      __syncwarp();
      // refill the B slot of step - 1 with blob step - 1 + BS once that step's MMAs are done
      if (step >= 1 && step - 1 + BS < nsteps) {
        const int bp = (int)((step - 1) % BS);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bempty[bp], (uint32_t)(((step - 1) / BS) & 1), err))) {
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_expect_tx(&full[bp], (uint32_t)B_BYTES);
          bulk_g2s(sB + bp * B_BYTES, blob(step - 1 + BS), (uint32_t)B_BYTES, &full[bp]);
        }
        ++copies;
      }
    }
  } else if (CL > 1 && warp == GW + 1) {
    // ---- exchange (CL = 2): as soon as this CTA's generators have written their half of a
    // stage, one shared-to-shared bulk copy sends it to the other CTA (whose stage s is free:
    // `empty` counts both CTAs' MMA commits), and the stage is armed for the other half
    for (int64_t step = 0; step < nsteps; ++step) {
      const int s = (int)(step % STAGES);
      const uint32_t par = (uint32_t)((step / STAGES) & 1);
      if (step >= STAGES &&
          !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((step / STAGES) - 1) & 1), err))) {
        ok = false;
        break;
      }
      const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&gen[s], par, err));
      if (lane == 0) {
        uint8_t* stA = sA + s * A_BYTES;
        const uint32_t peer = rank ^ 1u;
        if (got) bulk_s2peer(peer_addr(smem_u32(stA + rank * HALF_A), peer), stA + rank * HALF_A, HALF_A,
                             peer_addr(smem_u32(&sfull[s]), peer));
        mbar_expect_tx(&sfull[s], HALF_A);
      }
      ++armed;
      __syncwarp();
      if (!got) {
        ok = false;
        break;
      }
    }
  }
  // all MMAs done: the final phase of every stage counts the last commits of every CTA
  ok = !__syncthreads_or(!ok);
  if (ok && nsteps > 0) {
    const int64_t first = nsteps > STAGES ? nsteps - STAGES : 0;
    for (int64_t st = first; st < nsteps && ok; ++st)
      ok = mbar_wait_bounded(&empty[st % STAGES], (uint32_t)((st / STAGES) & 1), err);
    // and this CTA's own last MMAs, through the B slot commit of the last step
    if (ok) ok = mbar_wait_bounded(&bempty[(nsteps - 1) % BS], (uint32_t)(((nsteps - 1) / BS) & 1), err);
  }
  ok = !__syncthreads_or(!ok);
  // a failed run may leave bulk copies in flight (blobs, and the other CTA's halves of S into
  // this CTA): wait (bounded) for each slot's last one
  if (!ok && warp == GW)
    for (int64_t c = (copies > BS ? copies - BS : 0); c < copies; ++c)
      (void)mbar_wait_bounded(&full[c % BS], (uint32_t)((c / BS) & 1), err);
  if (!ok && warp == GW + 1)
    for (int64_t c = (armed > STAGES ? armed - STAGES : 0); c < armed; ++c)
      (void)mbar_wait_bounded(&sfull[c % STAGES], (uint32_t)((c / STAGES) & 1), err);
  __syncwarp();
  tc_fence_after();
  if (warp < GW) {
    if (ok && nsteps > 0) {
      // warp w reads TMEM lanes 32 (w % 4) .. + 31; the warps sharing a lane group split the columns
      constexpr int GROUPS = GW / 4;
      const int lg = warp & 3, cg = warp >> 2;
      const int L = 32 * lg + lane;
      const int j = j0 + (L < 64 ? 2 * L : 2 * (L - 64) + 1);
      float* out = part + (int64_t)blockIdx.z * m * d;
      for (int cb = 16 * cg; cb < NT; cb += 16 * GROUPS) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)cb, r);
        const int col0 = ct * NT + cb;
        if (j < m && col0 < d) {
          float* o = out + (int64_t)j * d + col0;
          if ((d & 3) == 0 && col0 + 16 <= d) {
#pragma unroll
            for (int q = 0; q < 16; q += 4) {
              float4 v = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]), __uint_as_float(r[q + 2]),
                                     __uint_as_float(r[q + 3]));
              if (accumulate) {
                const float4 p = *reinterpret_cast<const float4*>(o + q);
                v.x += p.x;
                v.y += p.y;
                v.z += p.z;
                v.w += p.w;
              }
              *reinterpret_cast<float4*>(o + q) = v;
            }
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (col0 + q < d) o[q] = (accumulate ? o[q] : 0.f) + __uint_as_float(r[q]);
          }
        }
      }
    } else if (!accumulate) {
      // nothing accumulated (no rows, or a failed run): the partial tile is zero
      float* out = part + (int64_t)blockIdx.z * m * d;
      for (int e = tid; e < TC_M * NT; e += TC_GEN) {
        const int row = e / NT, col = ct * NT + e % NT;
        const int jj = j0 + (row < 64 ? 2 * row : 2 * (row - 64) + 1);
        if (jj < m && col < d) out[(int64_t)jj * d + col] = 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NT);
  // no CTA leaves while another CTA of its cluster may still write into its shared memory
  if (CL > 1) cluster_sync_all();
}

// out[e] = scale * sum_g part[g][e], fixed order in g
__global__ void reduce_tc_kernel(const float* __restrict__ part, int splits, int64_t md, double scale,
                                 double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < md; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < splits; ++g) s += (double)part[(int64_t)g * md + e];
    out[e] = scale * s;
  }
}

struct SjltHashes {
  const int32_t* h;     // n x s target rows (draw order)
  const uint32_t* sgn;  // n sign words
  int s;
  int64_t n;
};

template <int NT, int STAGES, int BS, int CL, bool SJ>
lsq_status launch_tc(lsq_ctx* ctx, dim3 grid, const uint8_t* pk, int64_t nkb, int nct, int d, int m, uint64_t seed,
                     uint32_t t, int64_t row0, int64_t kb_per_split, int accumulate, float* part, int* err,
                     const SjltHashes& hs) {
  const size_t smem = (size_t)STAGES * (TC_M * TC_KS * 2) + (size_t)BS * (NT * TC_KS * 2);
  auto k = gauss_tc_kernel<NT, STAGES, BS, CL, SJ>;
  LSQ_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (CL == 1) {
    k<<<grid, TC_GEN + (CL > 1 ? 64 : 32), smem, ctx->stream>>>(pk, nkb, nct, d, m, seed, t, row0, kb_per_split, accumulate, part,
                                                err, hs.h, hs.sgn, hs.s, hs.n);
  } else {
    // clusters of CL CTAs along the column tiles (grid.y is a multiple of CL)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(TC_GEN + 64);  // a CTA pair: the generators, the MMA warp and the exchange warp
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CL;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LSQ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, pk, nkb, nct, d, m, seed, t, row0, kb_per_split, accumulate, part, err,
                                    hs.h, hs.sgn, hs.s, hs.n));
  }
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

// split count whose CTA count fills whole waves best (one CTA per SM)
int pick_splits(int tiles, int sms, int64_t kb_total, int64_t cap) {
  int best = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= 64 && s <= kb_total && s <= cap; ++s) {
    const int64_t ctas = (int64_t)tiles * s;
    const int64_t waves = (ctas + sms - 1) / sms;
    double eff = (double)ctas / (double)(waves * sms);
    if (waves < 2) eff *= 0.9;  // prefer at least two waves' worth of CTAs
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

}  // namespace

lsq_status lsq_sjlt_hash_launch(lsq_ctx* ctx, int64_t n, int m, int s, uint64_t seed, uint32_t t, int64_t grow0,
                                int32_t* h, uint32_t* signs);

// Both sketches share the driver: sjlt_s = 0 the Gaussian, sjlt_s > 0 the SJLT with s nonzeros
// per column (its target rows drawn first by the hash pass of lsq_sketch's SJLT)
static lsq_status tc_sketch_run(lsq_ctx* ctx, const lsq_matrix* A, int m, uint64_t seed, uint32_t t, double* SA,
                                lsq_rows_hook rows_ready, void* hook_user, int64_t grow0, int sjlt_s) {
  const int d = (int)A->d;
  const int nt = d > 256 ? 512 : 256;
  const int nct = (d + nt - 1) / nt;
  const int tiles_m = (m + TC_M - 1) / TC_M;
  const int tiles = tiles_m * nct;
  const size_t blob = (size_t)nt * TC_KS * 2;
  // chunks of at most 1 GiB of packed A
  int64_t kb_chunk = std::max<int64_t>(1, ((int64_t)1 << 30) / (int64_t)(blob * nct));
  const int64_t kb_total = (A->n + TC_KS - 1) / TC_KS;
  kb_chunk = std::min(kb_chunk, kb_total);
  const int64_t cap = std::max<int64_t>(1, ((int64_t)512 << 20) / ((int64_t)m * d * 4));
  const int splits = pick_splits(tiles, ctx->sm_count, kb_chunk, cap);
  const int64_t kb_per_split = (kb_chunk + splits - 1) / splits;
  const bool sj = sjlt_s > 0;
  const size_t hash_bytes = sj ? lsq_align256((size_t)A->n * sjlt_s * 4) + lsq_align256((size_t)A->n * 4) : 0;
  // more than one chunk: two packed-chunk buffers, so that chunk k + 1 is packed (on the
  // auxiliary stream) while the tensor cores work on chunk k
  const int64_t nchunks = (kb_total + kb_chunk - 1) / kb_chunk;
  const bool two = nchunks > 1;
  const size_t pk_bytes = (size_t)kb_chunk * nct * blob;
  const size_t need = lsq_align256(pk_bytes) * (two ? 2 : 1) + lsq_align256((size_t)splits * m * d * 4) + 256 +
                      hash_bytes;
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  uint8_t* pkb[2];
  pkb[0] = cv.take<uint8_t>(pk_bytes);
  pkb[1] = two ? cv.take<uint8_t>(pk_bytes) : pkb[0];
  float* part = cv.take<float>((size_t)splits * m * d);
  int* err = cv.take<int>(1);
  SjltHashes hs{nullptr, nullptr, 0, A->n};
  if (sj) {
    int32_t* h = cv.take<int32_t>((size_t)A->n * sjlt_s);
    uint32_t* sg = cv.take<uint32_t>((size_t)A->n);
    st = lsq_sjlt_hash_launch(ctx, A->n, m, sjlt_s, seed, t, grow0, h, sg);
    if (st != LSQ_OK) return st;
    hs = SjltHashes{h, sg, sjlt_s, A->n};
  }
  LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  // the packing stream: the context stream, or the auxiliary one, which first waits for the work
  // already queued on the context stream (it may write A)
  cudaStream_t ps = ctx->stream;
  if (two) {
    if (!ctx->aux) LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ctx->ev_aux)
      if (!e) LSQ_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    LSQ_CUDA_TRY(cudaEventRecord(ctx->ev_aux[4], ctx->stream));
    LSQ_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_aux[4], 0));
    ps = ctx->aux;
  }
  // on an early return the context stream still waits for everything queued on the packing stream
  auto join = [&](lsq_status r) {
    if (two && cudaEventRecord(ctx->ev_aux[4], ctx->aux) == cudaSuccess)
      cudaStreamWaitEvent(ctx->stream, ctx->ev_aux[4], 0);
    return r;
  };
  const dim3 grid(tiles_m, nct, splits);
  int64_t c = 0;
  for (int64_t kb0 = 0; kb0 < kb_total; kb0 += kb_chunk, ++c) {
    const int64_t nkb = std::min(kb_chunk, kb_total - kb0);
    const int64_t row0 = kb0 * TC_KS;  // of A; grow0 + row0 in the whole matrix (the generator's index)
    const int buf = (int)(c & 1);
    uint8_t* pk = pkb[buf];
    // the buffer was last read by the MMAs of chunk c - 2
    if (two && c >= 2 && cudaStreamWaitEvent(ps, ctx->ev_aux[2 + buf], 0) != cudaSuccess) return join(LSQ_ERR_CUDA);
    if (rows_ready) {
      st = rows_ready(hook_user, row0, std::min<int64_t>(A->n, row0 + nkb * TC_KS), ps);
      if (st != LSQ_OK) return join(st);
    }
    const int64_t units = nkb * 8 * (int64_t)nt * nct;
    const int pgrid = (int)std::min<int64_t>((units + 255) / 256, 16 * (int64_t)ctx->sm_count);
    if (A->dtype == LSQ_F64)
      pack_kernel<double><<<pgrid, 256, 0, ps>>>(reinterpret_cast<const double*>(A->data), A->n, d, A->ld, row0, nkb,
                                                 nt, nct, pk);
    else
      pack_kernel<float><<<pgrid, 256, 0, ps>>>(reinterpret_cast<const float*>(A->data), A->n, d, A->ld, row0, nkb, nt,
                                                nct, pk);
    if (cudaGetLastError() != cudaSuccess) return join(LSQ_ERR_CUDA);
    lsq_count_launch();
    if (two && (cudaEventRecord(ctx->ev_aux[buf], ps) != cudaSuccess ||
                cudaStreamWaitEvent(ctx->stream, ctx->ev_aux[buf], 0) != cudaSuccess))
      return join(LSQ_ERR_CUDA);
    const int acc = kb0 > 0 ? 1 : 0;
    // the Gaussian generator indexes rows of the whole matrix; the SJLT's hashes are A's own rows
    const int64_t r0 = sj ? row0 : grow0 + row0;
    // a CTA pair shares S when d needs two 512-column tiles (nt = 256 only for d <= 256)
    if (nt == 512 && nct % 2 == 0)
      st = sj ? launch_tc<512, 2, 3, 2, true>(ctx, grid, pk, nkb, nct, d, m, seed, t, r0, kb_per_split, acc, part, err, hs)
              : launch_tc<512, 2, 3, 2, false>(ctx, grid, pk, nkb, nct, d, m, seed, t, r0, kb_per_split, acc, part, err, hs);
    else if (nt == 512)
      st = sj ? launch_tc<512, 2, 3, 1, true>(ctx, grid, pk, nkb, nct, d, m, seed, t, r0, kb_per_split, acc, part, err, hs)
              : launch_tc<512, 2, 3, 1, false>(ctx, grid, pk, nkb, nct, d, m, seed, t, r0, kb_per_split, acc, part, err, hs);
    else
      st = sj ? launch_tc<256, 4, 4, 1, true>(ctx, grid, pk, nkb, nct, d, m, seed, t, r0, kb_per_split, acc, part, err, hs)
              : launch_tc<256, 4, 4, 1, false>(ctx, grid, pk, nkb, nct, d, m, seed, t, r0, kb_per_split, acc, part, err, hs);
    if (st != LSQ_OK) return join(st);
    if (two && cudaEventRecord(ctx->ev_aux[2 + buf], ctx->stream) != cudaSuccess) return join(LSQ_ERR_CUDA);
  }
  const int64_t md = (int64_t)m * d;
  const int rgrid = (int)std::min<int64_t>((md + 255) / 256, 4 * (int64_t)ctx->sm_count);
  reduce_tc_kernel<<<rgrid, 256, 0, ctx->stream>>>(part, splits, md, 1.0 / sqrt((double)(sj ? sjlt_s : m)), SA);
  LSQ_LAUNCH_CHECK();
  // a timed-out wait inside the tensor-core kernel is reported here (or deferred)
  if (ctx->defer_checks) return lsq_defer_status(ctx, err, 0);
  LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 13, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LSQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ctx->host_status[13] ? (lsq_status)ctx->host_status[13] : LSQ_OK;
}

// BF16 tensor-core Gaussian sketch into SA (FP64, m x d); called by lsq_sketch.  `rows_ready`
// (may be null) is called with each chunk's row range [r0, r1) before the chunk is read, in row
// order, so that a caller can queue the upload of those rows and make the context stream wait
// for them (lsq_upload_sketch): the copy of chunk k + 1 then overlaps the work on chunk k.
lsq_status lsq_gauss_tc_run(lsq_ctx* ctx, const lsq_matrix* A, int m, uint64_t seed, uint32_t t, double* SA,
                            lsq_rows_hook rows_ready, void* hook_user, int64_t grow0) {
  return tc_sketch_run(ctx, A, m, seed, t, SA, rows_ready, hook_user, grow0, 0);
}

// The SJLT with s nonzeros per column of S on the tensor cores (BF16 A, exact +-1 entries,
// FP32 accumulation in a fixed order, 1/sqrt(s) in FP64); arguments as lsq_gauss_tc_run.
lsq_status lsq_sjlt_tc_run(lsq_ctx* ctx, const lsq_matrix* A, int m, int s, uint64_t seed, uint32_t t, double* SA,
                           lsq_rows_hook rows_ready, void* hook_user, int64_t grow0) {
  return tc_sketch_run(ctx, A, m, seed, t, SA, rows_ready, hook_user, grow0, s);
}
