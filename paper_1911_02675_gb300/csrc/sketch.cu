// sketch.cu -- SA = S A for the three embeddings of Section 2 (Gaussian, SRHT, SJLT).
//
// Every kernel streams A once (Gaussian: once per 64-row slab of S) and generates its
// randomness on the fly from Philox4x32-10; S is never stored.  Partial sums go to a
// per-split scratch slab and a fixed-order reduction writes SA, so results repeat run
// to run (SJLT: up to the order of its shared-memory additions).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "apass.cuh"
#include "common.cuh"

namespace {

// ------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T load_as(const void* base, int64_t idx, int dtype) {
  if (dtype == LSQ_F64) return (T)__ldg(reinterpret_cast<const double*>(base) + idx);
  return (T)__ldg(reinterpret_cast<const float*>(base) + idx);
}

// FP32 arithmetic on FP64 data: narrow with integer operations (the FP64->FP32 conversion
// instruction runs at the FP64 rate on this part)
template <>
__device__ __forceinline__ float load_as<float>(const void* base, int64_t idx, int dtype) {
  if (dtype == LSQ_F64) return lsq_apass::narrow_f32(__ldg(reinterpret_cast<const double*>(base) + idx));
  return __ldg(reinterpret_cast<const float*>(base) + idx);
}

// 53 random bits -> (k + 1/2) 2^-53 in the open unit interval
__device__ __forceinline__ double unit_open53(uint32_t hi, uint32_t lo) {
  const unsigned long long k = ((((unsigned long long)hi) << 32) | lo) >> 11;
  return ((double)k + 0.5) * 0x1p-53;
}

// Box-Muller pair (cosine branch, sine branch) in the arithmetic type T
template <typename T>
__device__ __forceinline__ void box_muller(uint4 w, T& z_cos, T& z_sin);

template <>
__device__ __forceinline__ void box_muller<double>(uint4 w, double& zc, double& zs) {
  const double u1 = unit_open53(w.x, w.y);
  const double u2 = unit_open53(w.z, w.w);
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  zc = rad * c;
  zs = rad * s;
}

template <>
__device__ __forceinline__ void box_muller<float>(uint4 w, float& zc, float& zs) {
  // the same 53-bit uniforms, evaluated in FP32 (u1 > 0 is kept by the +1/2 offset)
  const float u1 = (float)unit_open53(w.x, w.y);
  const float u2 = (float)unit_open53(w.z, w.w);
  const float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  zc = rad * c;
  zs = rad * s;
}

// out[j*d + c] = scale * sum_g part[g][j][c]   (fixed order in g).  FP32 partials are summed as
// (head, tail) FP32 pairs (TwoSum: exact up to the final rounding of the pair) on the FP32 pipe,
// which does ~70x the FP64 pipe's adds on this part; FP64 partials in FP64.
template <typename TP>
__global__ void reduce_splits_kernel(const TP* __restrict__ part, int splits, int64_t md, double scale,
                                     double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < md; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if constexpr (sizeof(TP) == 4) {
      float h = 0.f, t = 0.f;
      for (int g = 0; g < splits; ++g) lsq_apass::df_add(h, t, part[(int64_t)g * md + e], 0.f);
      s = (double)h + (double)t;
    } else {
      for (int g = 0; g < splits; ++g) s += (double)part[(int64_t)g * md + e];
    }
    out[e] = scale * s;
  }
}

// ------------------------------------------------------------------------------------
// Gaussian: SA = S A, S[j,i] = z(j,i)/sqrt(m).  Split-K GEMM over the rows of A; each
// CTA owns a 64 x 64 tile of SA and a contiguous range of rows, regenerates its 64 x 16
// tile of S per step (one Philox call per pair of sketch rows) and accumulates 4 x 4
// outputs per thread.  Scaling by 1/sqrt(m) happens in the reduction.
// ------------------------------------------------------------------------------------
constexpr int GM = 64, GD = 64, GK = 16;

template <typename T>
__global__ void __launch_bounds__(256) gauss_sketch_kernel(const void* __restrict__ A, int dtype, int64_t n, int d,
                                                          int64_t ld, int m, uint64_t seed, uint32_t t,
                                                          int64_t rows_per_split, T* __restrict__ part,
                                                          int64_t grow0) {
  __shared__ T Ss[GK][GM];
  __shared__ T As[GK][GD];
  const int j0 = blockIdx.x * GM, c0 = blockIdx.y * GD;
  const int64_t i_begin = (int64_t)blockIdx.z * rows_per_split;
  const int64_t i_end = min(n, i_begin + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;

  for (int64_t i0 = i_begin; i0 < i_end; i0 += GK) {
    for (int e = threadIdx.x; e < (GM / 2) * GK; e += 256) {
      const int jp = e / GK, k = e % GK;
      const int64_t i = i0 + k;
      T zc = (T)0, zs = (T)0;
      if (i < i_end)
        box_muller<T>(philox_at(seed, (uint32_t)(i + grow0), (uint32_t)((j0 >> 1) + jp), t, TAG_GAUSS), zc, zs);
      Ss[k][2 * jp] = zc;
      Ss[k][2 * jp + 1] = zs;
    }
    for (int e = threadIdx.x; e < GK * GD; e += 256) {
      const int k = e / GD, c = e % GD;
      const int64_t i = i0 + k;
      As[k][c] = (i < i_end && c0 + c < d) ? load_as<T>(A, i * ld + c0 + c, dtype) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      T s[4], a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) s[r] = Ss[k][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = As[k][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(s[r], a[c], acc[r][c]);
    }
    __syncthreads();
  }
  T* out = part + (int64_t)blockIdx.z * m * d;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int j = j0 + ty + 16 * r;
    if (j >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = c0 + tx + 16 * c;
      if (col < d) out[(int64_t)j * d + col] = acc[r][c];
    }
  }
}

// ------------------------------------------------------------------------------------
// SRHT: S = (1/sqrt m) P H E on N = 2^ceil(log2 n) zero-padded rows.
//   (1) keys/signs: sample key and sign bit of every row i < N;
//   (2) radix select: the m-th smallest (key, index) by four 16-bit digit rounds;
//   (3) compaction: the selected rows in ascending index order;
//   (4) two-level transform: N = N1 * N2, i = i1 * N2 + i2, and
//       (H x)[k1 N2 + k2] = sum_{i1} (-1)^{popc(k1 & i1)} (H_{N2} x_{i1})[k2],
//       so each CTA runs length-N2 transforms of row blocks in shared memory and adds
//       the signed block outputs for the m sampled rows only.
// ------------------------------------------------------------------------------------
__global__ void srht_keys_kernel(int64_t N, uint64_t seed, uint32_t t, unsigned long long* __restrict__ keys,
                                 uint32_t* __restrict__ signbits, unsigned* __restrict__ hist) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool neg = false;
    if (i < N) {
      const uint4 k = philox_at(seed, (uint32_t)i, (uint32_t)(i >> 32), t, TAG_SAMPLE);
      const unsigned long long key = (((unsigned long long)k.x) << 32) | k.y;
      keys[i] = key;
      atomicAdd(&hist[key >> 48], 1u);
      neg = (philox_at(seed, (uint32_t)i, (uint32_t)(i >> 32), t, TAG_SIGN).x & 1u) != 0u;
    }
    const unsigned word = __ballot_sync(0xffffffffu, neg);
    if ((threadIdx.x & 31) == 0 && i < N) signbits[i >> 5] = word;
  }
}

// state: [0] prefix (digits found so far), [1] need (rank still to reach, 1-based),
//        [2] count of keys strictly below the current prefix bucket
__global__ void radix_hist_kernel(const unsigned long long* __restrict__ keys, int64_t N, int shift,
                                  const unsigned long long* __restrict__ state, unsigned* __restrict__ hist) {
  const unsigned long long prefix = state[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[i];
    if ((key >> (shift + 16)) == prefix) atomicAdd(&hist[(key >> shift) & 0xFFFFu], 1u);
  }
}

// one CTA of 1024 threads: finds the bucket holding rank `need`, clears the histogram.
// Thread t sums buckets [64 t, 64 t + 64) (16-byte loads), the CTA scans the 1024 partial
// counts (warp shuffles, then the 32 warp totals), and warp 0 scans the 64 buckets of the
// thread whose range holds rank `need`.
__global__ void __launch_bounds__(1024) radix_pick_kernel(unsigned* __restrict__ hist,
                                                          unsigned long long* __restrict__ state) {
  __shared__ unsigned long long wsum[32];
  __shared__ int owner;
  __shared__ unsigned long long owner_before;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint4* hp = reinterpret_cast<const uint4*>(hist) + tid * 16;
  unsigned long long local = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint4 q = hp[k];
    local += (unsigned long long)q.x + q.y + q.z + q.w;
  }
  // inclusive scan of the per-thread counts
  unsigned long long inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  if (tid == 0) owner = -1;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  const unsigned long long before = (w > 0 ? wsum[w - 1] : 0ull) + inc - local;
  const unsigned long long need = state[1], below = state[2];
  if (before < need && need <= before + local) {
    owner = tid;
    owner_before = before;
  }
  __syncthreads();
  if (w == 0 && owner >= 0) {
    // warp 0 walks the owner's 64 buckets: two per lane, one warp scan, first crossing by ballot
    const int t = owner;
    const unsigned h0 = hist[64 * t + 2 * lane], h1 = hist[64 * t + 2 * lane + 1];
    unsigned long long x = (unsigned long long)h0 + h1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned long long ex = owner_before + x - h0 - h1;  // before bucket 2 lane
    const bool hit0 = ex + h0 >= need, hit1 = ex + h0 + h1 >= need;
    const unsigned m0 = __ballot_sync(0xffffffffu, hit0), m1 = __ballot_sync(0xffffffffu, hit1);
    const int l0 = m0 ? __ffs(m0) - 1 : 32, l1 = m1 ? __ffs(m1) - 1 : 32;
    // the first bucket whose running count reaches `need`
    const int bkt = l0 <= l1 ? 2 * l0 : 2 * l1 + 1;
    if (lane == (bkt >> 1)) {
      const unsigned long long cum = (bkt & 1) ? ex + h0 : ex;
      state[0] = (state[0] << 16) | (unsigned long long)(64 * t + bkt);
      state[1] = need - cum;
      state[2] = below + cum;
    }
  }
  __syncthreads();
  uint4* hw = reinterpret_cast<uint4*>(hist);
  for (int k = tid; k < 65536 / 4; k += 1024) hw[k] = make_uint4(0u, 0u, 0u, 0u);
}

constexpr int SCAN_BLOCK = 1024;

// per block of 1024 rows: counts of keys < K and == K (K = state[0] after 4 rounds)
__global__ void select_count_kernel(const unsigned long long* __restrict__ keys, int64_t N,
                                    const unsigned long long* __restrict__ state, unsigned* __restrict__ cnt_lt,
                                    unsigned* __restrict__ cnt_eq) {
  __shared__ unsigned s_lt, s_eq;
  if (threadIdx.x == 0) { s_lt = 0; s_eq = 0; }
  __syncthreads();
  const unsigned long long K = state[0];
  const int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  if (i < N) {
    const unsigned long long key = keys[i];
    if (key < K) atomicAdd(&s_lt, 1u);
    else if (key == K) atomicAdd(&s_eq, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) { cnt_lt[blockIdx.x] = s_lt; cnt_eq[blockIdx.x] = s_eq; }
}

// exclusive prefix sums over the blocks (single CTA, sequential chunks)
__global__ void select_scan_kernel(unsigned* __restrict__ cnt_lt, unsigned* __restrict__ cnt_eq, int nb) {
  __shared__ unsigned long long carry_lt, carry_eq;
  __shared__ unsigned buf_lt[1024], buf_eq[1024];
  if (threadIdx.x == 0) { carry_lt = 0; carry_eq = 0; }
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int b = base + threadIdx.x;
    buf_lt[threadIdx.x] = b < nb ? cnt_lt[b] : 0u;
    buf_eq[threadIdx.x] = b < nb ? cnt_eq[b] : 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long a = carry_lt, e = carry_eq;
      for (int k = 0; k < 1024; ++k) {
        const unsigned vl = buf_lt[k], ve = buf_eq[k];
        buf_lt[k] = (unsigned)a;
        buf_eq[k] = (unsigned)e;
        a += vl;
        e += ve;
      }
      carry_lt = a;
      carry_eq = e;
    }
    __syncthreads();
    if (b < nb) { cnt_lt[b] = buf_lt[threadIdx.x]; cnt_eq[b] = buf_eq[threadIdx.x]; }
    __syncthreads();
  }
}

__global__ void select_write_kernel(const unsigned long long* __restrict__ keys, int64_t N,
                                    const unsigned long long* __restrict__ state, const unsigned* __restrict__ pre_lt,
                                    const unsigned* __restrict__ pre_eq, int64_t* __restrict__ rows, int m) {
  __shared__ unsigned warp_sel[32], warp_eq[32];
  const unsigned long long K = state[0];
  const unsigned need_eq = (unsigned)state[1];
  const int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long key = 0;
  if (i < N) key = keys[i];
  const bool lt = (i < N) && key < K;
  const bool eq = (i < N) && key == K;
  // rank of this row among the block's equal keys
  const unsigned eq_mask = __ballot_sync(0xffffffffu, eq);
  if (lane == 0) warp_eq[w] = __popc(eq_mask);
  __syncthreads();
  unsigned eq_before = pre_eq[blockIdx.x];
  for (int k = 0; k < w; ++k) eq_before += warp_eq[k];
  eq_before += __popc(eq_mask & ((1u << lane) - 1u));
  const bool sel = lt || (eq && eq_before < need_eq);
  const unsigned sel_mask = __ballot_sync(0xffffffffu, sel);
  if (lane == 0) warp_sel[w] = __popc(sel_mask);
  __syncthreads();
  // rows selected before this block: keys < K plus the equal keys admitted so far
  unsigned long long pos = (unsigned long long)pre_lt[blockIdx.x] + min(pre_eq[blockIdx.x], need_eq);
  for (int k = 0; k < w; ++k) pos += warp_sel[k];
  pos += __popc(sel_mask & ((1u << lane) - 1u));
  if (sel && pos < (unsigned long long)m) rows[pos] = i;
}

// Two-level transform.  A CTA owns a tile of DC columns and a range of row blocks of
// N2 = 2^logN2 rows.  Per block: the first (up to) 4 butterfly stages run in registers as
// the block is loaded (16 consecutive rows of one column per unit, signs applied), the
// remaining stages run as register radix-16 passes over a shared-memory copy, and the
// sampled second level adds +-Z[k2(s)] into the CTA's partial of SA[s] for every sampled
// row s.  Shared rows are DC elements (32 bytes) with 32 bytes of padding after every 16
// rows, which keeps all three access patterns free of bank conflicts.
constexpr int SRHT_THREADS = 512;

__host__ __device__ __forceinline__ int zphys(int row, int dc) { return (row + (row >> 4)) * dc; }

template <typename TC, int K>
__device__ __forceinline__ void butterflies(TC* v) {
#pragma unroll
  for (int h = 1; h < (1 << K); h <<= 1)
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
      if (!(j & h)) {
        const TC a = v[j], b = v[j + h];
        v[j] = a + b;
        v[j + h] = a - b;
      }
}

// stages over row bits [b, b + K) on the shared block
template <typename TC, int DC, int K>
__device__ __forceinline__ void radix_pass(TC* Z, int N2, int b) {
  const int units = (N2 >> K) * DC;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int c = u % DC, q = u / DC;
    const int base = ((q >> b) << (b + K)) | (q & ((1 << b) - 1));
    TC v[1 << K];
#pragma unroll
    for (int j = 0; j < (1 << K); ++j) v[j] = Z[zphys(base + (j << b), DC) + c];
    butterflies<TC, K>(v);
#pragma unroll
    for (int j = 0; j < (1 << K); ++j) Z[zphys(base + (j << b), DC) + c] = v[j];
  }
}

// load a block (signs applied, zero past n) with the stages over row bits [0, K); each
// thread issues the loads of two units before it uses any of them
template <typename TC, int DC, int K>
__device__ __forceinline__ void load_unit(TC* v, const void* A, int dtype, int64_t n, int d, int64_t ld, int c0,
                                          int64_t row0, const uint32_t* signbits, int u) {
  const int c = u % DC, q = u / DC;
  const int64_t r = row0 + ((int64_t)q << K);
  const bool col_ok = c0 + c < d;
  const uint32_t word = (r < n) ? __ldg(signbits + (r >> 5)) : 0u;
  const int sh = (int)(r & 31);
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) {
    const int64_t i = r + j;
    TC x = (TC)0;
    if (col_ok && i < n) {
      x = load_as<TC>(A, i * ld + c0 + c, dtype);
      if ((word >> (sh + j)) & 1u) x = -x;
    }
    v[j] = x;
  }
}

template <typename TC, int DC, int K>
__device__ __forceinline__ void store_unit(TC* Z, TC* v, int u) {
  const int c = u % DC, q = u / DC;
  butterflies<TC, K>(v);
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) Z[zphys((q << K) + j, DC) + c] = v[j];
}

template <typename TC, int DC, int K>
__device__ __forceinline__ void load_pass(TC* Z, const void* A, int dtype, int64_t n, int d, int64_t ld, int c0,
                                          int64_t row0, int N2, const uint32_t* signbits) {
  const int units = (N2 >> K) * DC;
  const int T = blockDim.x;
  for (int u = threadIdx.x; u < units; u += 2 * T) {
    TC v0[1 << K], v1[1 << K];
    const bool two = u + T < units;
    load_unit<TC, DC, K>(v0, A, dtype, n, d, ld, c0, row0, signbits, u);
    if (two) load_unit<TC, DC, K>(v1, A, dtype, n, d, ld, c0, row0, signbits, u + T);
    store_unit<TC, DC, K>(Z, v0, u);
    if (two) store_unit<TC, DC, K>(Z, v1, u + T);
  }
}

template <typename TC, int DC>
__global__ void __launch_bounds__(SRHT_THREADS, 1) srht_transform_kernel(
    const void* __restrict__ A, int dtype, int64_t n, int d, int64_t ld, int logN2, int64_t N1,
    int64_t blocks_per_group, const uint32_t* __restrict__ signbits, const int64_t* __restrict__ rows, int m,
    TC* __restrict__ part, uint32_t blk0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N2 = 1 << logN2;
  TC* Z = reinterpret_cast<TC*>(smem_raw);                   // padded [N2][DC]
  TC* Y = Z + (size_t)zphys(N2, DC);                         // [m][DC]
  uint32_t* k1s = reinterpret_cast<uint32_t*>(Y + (size_t)m * DC);  // [m]
  uint16_t* k2s = reinterpret_cast<uint16_t*>(k1s + m);             // [m]
  const int c0 = blockIdx.x * DC;
  const int64_t b_begin = (int64_t)blockIdx.y * blocks_per_group;
  const int64_t b_end = min(N1, b_begin + blocks_per_group);
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) Y[e] = (TC)0;
  for (int s = threadIdx.x; s < m; s += blockDim.x) {
    const int64_t k = rows[s];
    k1s[s] = (uint32_t)(k >> logN2);
    k2s[s] = (uint16_t)(k & (N2 - 1));
  }
  const int k0 = logN2 < 4 ? logN2 : 4;
  const int T = blockDim.x;
  const int units = (N2 >> k0) * DC;
  // Common case: 16-row units and at most two per thread.  The next block's loads are put
  // in flight as soon as the current block sits in shared memory, so they overlap the
  // remaining butterfly passes and the sampled second level.
  // (FP32 only: FP64 blocks are bound by the FP64 pipe and the registers are better spent)
  constexpr bool PIPE = sizeof(TC) == 4;
  constexpr int VB = PIPE ? 16 : 1;
  const bool pipelined = PIPE && k0 == 4 && units <= 2 * T;
  TC v0[VB], v1[VB];
  const bool has0 = threadIdx.x < units, has1 = threadIdx.x + T < units;
  if constexpr (PIPE) if (pipelined && b_begin < b_end) {
    if (has0) load_unit<TC, DC, 4>(v0, A, dtype, n, d, ld, c0, b_begin << logN2, signbits, threadIdx.x);
    if (has1) load_unit<TC, DC, 4>(v1, A, dtype, n, d, ld, c0, b_begin << logN2, signbits, threadIdx.x + T);
  }
  for (int64_t i1 = b_begin; i1 < b_end; ++i1) {
    __syncthreads();  // Z is free (previous block's second level is done)
    const int64_t row0 = i1 << logN2;
    if constexpr (PIPE) if (pipelined) {
      if (has0) store_unit<TC, DC, 4>(Z, v0, threadIdx.x);
      if (has1) store_unit<TC, DC, 4>(Z, v1, threadIdx.x + T);
      if (i1 + 1 < b_end) {
        const int64_t next0 = (i1 + 1) << logN2;
        if (has0) load_unit<TC, DC, 4>(v0, A, dtype, n, d, ld, c0, next0, signbits, threadIdx.x);
        if (has1) load_unit<TC, DC, 4>(v1, A, dtype, n, d, ld, c0, next0, signbits, threadIdx.x + T);
      }
    }
    if (!pipelined) {
      switch (k0) {
        case 4: load_pass<TC, DC, 4>(Z, A, dtype, n, d, ld, c0, row0, N2, signbits); break;
        case 3: load_pass<TC, DC, 3>(Z, A, dtype, n, d, ld, c0, row0, N2, signbits); break;
        case 2: load_pass<TC, DC, 2>(Z, A, dtype, n, d, ld, c0, row0, N2, signbits); break;
        case 1: load_pass<TC, DC, 1>(Z, A, dtype, n, d, ld, c0, row0, N2, signbits); break;
        default: load_pass<TC, DC, 0>(Z, A, dtype, n, d, ld, c0, row0, N2, signbits); break;
      }
    }
    for (int b = k0; b < logN2; b += 4) {
      __syncthreads();
      switch (logN2 - b < 4 ? logN2 - b : 4) {
        case 4: radix_pass<TC, DC, 4>(Z, N2, b); break;
        case 3: radix_pass<TC, DC, 3>(Z, N2, b); break;
        case 2: radix_pass<TC, DC, 2>(Z, N2, b); break;
        default: radix_pass<TC, DC, 1>(Z, N2, b); break;
      }
    }
    __syncthreads();
    const uint32_t i1w = (uint32_t)i1 + blk0;  // the block's index in the whole (zero-padded) matrix
    // one sampled row per thread: its k1/k2 and sign once, then the DC columns as 16-byte
    // vectors (a 32-byte row of the block and of the accumulator)
    for (int s = threadIdx.x; s < m; s += blockDim.x) {
      const bool neg = (__popc(k1s[s] & i1w) & 1) != 0;
      const TC* zr = Z + zphys(k2s[s], DC);
      TC* yr = Y + (size_t)s * DC;
      if constexpr (DC * sizeof(TC) % 16 == 0) {
#pragma unroll
        for (int c = 0; c < DC * (int)sizeof(TC) / 16; ++c) {
          uint4 zv = reinterpret_cast<const uint4*>(zr)[c];
          uint4 yv = reinterpret_cast<uint4*>(yr)[c];
          TC* zt = reinterpret_cast<TC*>(&zv);
          TC* yt = reinterpret_cast<TC*>(&yv);
#pragma unroll
          for (int q = 0; q < 16 / (int)sizeof(TC); ++q) yt[q] += neg ? -zt[q] : zt[q];
          reinterpret_cast<uint4*>(yr)[c] = yv;
        }
      } else {
#pragma unroll
        for (int c = 0; c < DC; ++c) yr[c] += neg ? -zr[c] : zr[c];
      }
    }
  }
  __syncthreads();
  TC* out = part + (int64_t)blockIdx.y * m * d;
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) {
    const int s = e / DC, c = e % DC;
    if (c0 + c < d) out[(int64_t)s * d + c0 + c] = Y[e];
  }
}

// The common case of the transform (FP32 arithmetic, 8-column tiles, 2048-row blocks) in a
// kernel of its own: a thread owns 16 consecutive rows x 2 adjacent columns of every block
// (512 units = 512 threads).  The next block's elements are loaded as raw 8- or 16-byte
// vectors and kept as loaded until the block is stored, so the loads stay in flight through
// the radix passes and the sampled second level; narrowing, signs and the first 4 butterfly
// stages happen at the store.  Same arithmetic, in the same order, as the general kernel.
template <typename TA>
__device__ __forceinline__ void srht_fast_load(TA (&r0)[16], TA (&r1)[16], uint32_t& sw, const TA* __restrict__ A,
                                               int64_t n, int64_t ld, int64_t row, int c, bool c_ok0, bool c_ok1,
                                               bool vec, const uint32_t* __restrict__ signbits) {
  using T2 = typename std::conditional<sizeof(TA) == 8, double2, float2>::type;
  sw = row < n ? (__ldg(signbits + (row >> 5)) >> (row & 31)) : 0u;
  const TA* src = A + (row < n ? row * ld + c : 0);
  if (vec && row + 15 < n) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const T2 x = __ldg(reinterpret_cast<const T2*>(src + j * ld));
      r0[j] = x.x;
      r1[j] = x.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const bool ok = row + j < n;
      r0[j] = (ok && c_ok0) ? __ldg(src + j * ld) : (TA)0;
      r1[j] = (ok && c_ok1) ? __ldg(src + j * ld + 1) : (TA)0;
    }
  }
}

template <typename TA>
__global__ void __launch_bounds__(SRHT_THREADS, 1) srht_fast_kernel(
    const TA* __restrict__ A, int64_t n, int d, int64_t ld, int64_t N1, int64_t blocks_per_group, int vec_ok,
    const uint32_t* __restrict__ signbits, const int64_t* __restrict__ rows, int m, float* __restrict__ part,
    uint32_t blk0) {
  constexpr int DC = 8, LOGN2 = 11, N2 = 1 << LOGN2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Z = reinterpret_cast<float*>(smem_raw);                        // padded [N2][DC]
  float* Y = Z + (size_t)zphys(N2, DC);                                 // [m][DC]
  uint32_t* k1s = reinterpret_cast<uint32_t*>(Y + (size_t)m * DC);      // [m]
  uint16_t* k2s = reinterpret_cast<uint16_t*>(k1s + m);                 // [m]
  const int c0 = blockIdx.x * DC;
  const int64_t b_begin = (int64_t)blockIdx.y * blocks_per_group;
  const int64_t b_end = min(N1, b_begin + blocks_per_group);
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) Y[e] = 0.f;
  for (int s = threadIdx.x; s < m; s += blockDim.x) {
    const int64_t k = rows[s];
    k1s[s] = (uint32_t)(k >> LOGN2);
    k2s[s] = (uint16_t)(k & (N2 - 1));
  }
  const int q = threadIdx.x >> 2, pc = threadIdx.x & 3;  // 16-row group, column pair
  const int c = c0 + 2 * pc;
  const bool c_ok0 = c < d, c_ok1 = c + 1 < d;
  const bool vec = vec_ok != 0 && c_ok1;
  TA r0[16], r1[16];
  uint32_t sw = 0;
  if (b_begin < b_end)
    srht_fast_load<TA>(r0, r1, sw, A, n, ld, (b_begin << LOGN2) + (q << 4), c, c_ok0, c_ok1, vec, signbits);
  for (int64_t i1 = b_begin; i1 < b_end; ++i1) {
    __syncthreads();  // Z is free (previous block's second level is done)
    {
      float v0[16], v1[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint32_t neg = ((sw >> j) & 1u) << 31;
        v0[j] = __uint_as_float(__float_as_uint(lsq_apass::narrow_f32(r0[j])) ^ neg);
        v1[j] = __uint_as_float(__float_as_uint(lsq_apass::narrow_f32(r1[j])) ^ neg);
      }
      butterflies<float, 4>(v0);
      butterflies<float, 4>(v1);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        *reinterpret_cast<float2*>(Z + zphys((q << 4) + j, DC) + 2 * pc) = make_float2(v0[j], v1[j]);
    }
    if (i1 + 1 < b_end)
      srht_fast_load<TA>(r0, r1, sw, A, n, ld, ((i1 + 1) << LOGN2) + (q << 4), c, c_ok0, c_ok1, vec, signbits);
    __syncthreads();
    radix_pass<float, DC, 4>(Z, N2, 4);
    __syncthreads();
    radix_pass<float, DC, 3>(Z, N2, 8);
    __syncthreads();
    const uint32_t i1w = (uint32_t)i1 + blk0;  // the block's index in the whole (zero-padded) matrix
    for (int s = threadIdx.x; s < m; s += blockDim.x) {
      const bool neg = (__popc(k1s[s] & i1w) & 1) != 0;
      const float4* zr = reinterpret_cast<const float4*>(Z + zphys(k2s[s], DC));
      float4* yr = reinterpret_cast<float4*>(Y + (size_t)s * DC);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 z = zr[h];
        float4 y = yr[h];
        y.x += neg ? -z.x : z.x;
        y.y += neg ? -z.y : z.y;
        y.z += neg ? -z.z : z.z;
        y.w += neg ? -z.w : z.w;
        yr[h] = y;
      }
    }
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.y * m * d;
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) {
    const int s = e / DC, cc = e % DC;
    if (c0 + cc < d) out[(int64_t)s * d + c0 + cc] = Y[e];
  }
}

// The common case once more, with the block staged by the tensor memory accelerator: per
// 2048-row block, eight 256-row x 8-column boxes of A land in shared memory as raw FP64 (or
// FP32) elements, completion counted in bytes on an mbarrier, while the previous block's
// radix passes and sampled second level run; the partial of SA lives in registers (thread t
// owns sampled rows t, t + 512, ...), so the second level reads only the block.  The register
// stage is over row bits 8..10 (a thread holds rows q, q + 256, ..., q + 1792 of a column
// quad), then radix passes over bits 0..3 and 4..7: the stages of a Walsh-Hadamard transform
// commute, so this is the same transform with its FP32 additions in another order.  The sign
// words of the next block are loaded one block ahead.  Every wait is bounded.
constexpr int SRHT_TMA_ROWS = 256;  // rows per box

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool srht_mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  uint32_t spins = 0;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (++spins > (1u << 26)) {
      atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      return false;
    }
  }
}

template <typename TA, int MY>
__global__ void __launch_bounds__(SRHT_THREADS, 1) srht_tma_kernel(
    const __grid_constant__ CUtensorMap tmap, int64_t n, int d, int64_t N1, int64_t blocks_per_group,
    const uint32_t* __restrict__ signbits, const int64_t* __restrict__ rows_all, int m_all,
    float* __restrict__ part, int* err, float* __restrict__ a32_all, int64_t ld32, int gy0, uint32_t blk0) {
  constexpr int DC = 8, LOGN2 = 11, N2 = 1 << LOGN2;
  const int64_t gy = (int64_t)blockIdx.y + gy0;  // row-block group (a launch may cover a range of them)
  // sampled rows [s0, s0 + m) of the m_all: up to 8 per thread, more in further grid.z slices
  // (each slice transforms the block again); the first slice writes the FP32 copy
  const int s0 = (int)blockIdx.z * 8 * SRHT_THREADS;
  const int m = min(m_all - s0, 8 * SRHT_THREADS);
  const int64_t* __restrict__ rows = rows_all + s0;
  float* __restrict__ a32 = blockIdx.z == 0 ? a32_all : nullptr;
  constexpr uint32_t STAGE_BYTES = N2 * DC * sizeof(TA);
  using T2 = typename std::conditional<sizeof(TA) == 8, double2, float2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the staged block starts on a 1024-byte boundary (tensor copies want 128-byte aligned
  // destinations); the launch adds 1 KB for the offset
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const TA* stage = reinterpret_cast<const TA*>(base);                    // [N2][DC] as the boxes land
  float* Z = reinterpret_cast<float*>(base + STAGE_BYTES);                // padded [N2][DC]
  uint32_t* k1s = reinterpret_cast<uint32_t*>(Z + (size_t)zphys(N2, DC));  // [m]
  uint16_t* k2s = reinterpret_cast<uint16_t*>(k1s + m);                   // [m]
  uint32_t* sgn = reinterpret_cast<uint32_t*>(k2s + ((m + 1) & ~1));      // [N2 / 32] signs of the block
  __shared__ __align__(8) uint64_t full;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * DC;
  const int64_t b_begin = gy * blocks_per_group;
  const int64_t b_end = min(N1, b_begin + blocks_per_group);
  for (int s = tid; s < m; s += SRHT_THREADS) {
    const int64_t k = rows[s];
    k1s[s] = (uint32_t)(k >> LOGN2);
    k2s[s] = (uint16_t)(k & (N2 - 1));
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0 starts the eight box copies of block `blk` (rows past n and columns past d read 0)
  auto issue = [&](int64_t blk) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&full)), "r"(STAGE_BYTES)
                 : "memory");
#pragma unroll
    for (int k = 0; k < N2 / SRHT_TMA_ROWS; ++k) {
      const int32_t x = c0, y = (int32_t)(blk * N2 + k * SRHT_TMA_ROWS);
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              smem_addr(stage + (size_t)k * SRHT_TMA_ROWS * DC)),
          "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x), "r"(y), "r"(smem_addr(&full))
          : "memory");
    }
  };
  if (tid == 0 && b_begin < b_end) issue(b_begin);

  float y[MY][DC];
#pragma unroll
  for (int i = 0; i < MY; ++i)
#pragma unroll
    for (int c = 0; c < DC; ++c) y[i][c] = 0.f;
  // load phase: thread t holds rows qq + 256 j (j < 8) of the column quad 4 p4 .. 4 p4 + 3
  // (qq = t / 2, p4 = t % 2), so a quarter-warp owns 256 contiguous bytes of each staged row
  // group; FP64 rows are read as two 16-byte halves, lanes 4..7 of a quarter taking the upper
  // half first, which puts the quarter's 8 reads on 8 distinct 16-byte bank groups
  const int qq = tid >> 1, p4 = tid & 1, hf = (tid >> 2) & 1;
  bool ok = true;
  int64_t issued = b_begin < b_end ? 1 : 0, waited = 0;
  // the sign words of the next block are loaded a block ahead (rows past n carry no data)
  uint32_t sgn_next = 0;
  if (tid < N2 / 32 && b_begin < b_end) {
    const int64_t r = b_begin * N2 + 32 * tid;
    sgn_next = r < n ? __ldg(signbits + (r >> 5)) : 0u;
  }
  for (int64_t i1 = b_begin; i1 < b_end; ++i1) {
    if (tid < N2 / 32) {
      sgn[tid] = sgn_next;
      const int64_t r = (i1 + 1) * N2 + 32 * tid;
      sgn_next = (i1 + 1 < b_end && r < n) ? __ldg(signbits + (r >> 5)) : 0u;
    }
    ok = ok && srht_mbar_wait(&full, (uint32_t)((i1 - b_begin) & 1), err);
    // Z is free (the previous second level is done) and the block has landed everywhere
    if (__syncthreads_or(!ok)) break;
    ++waited;
    {
      float v[4][8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = qq + 256 * j;
        float f[4];
        if constexpr (sizeof(TA) == 8) {
          const double2 x0 = *reinterpret_cast<const double2*>(stage + r * DC + 4 * p4 + 2 * hf);
          const double2 x1 = *reinterpret_cast<const double2*>(stage + r * DC + 4 * p4 + 2 * (hf ^ 1));
          const double2 xa = hf ? x1 : x0, xb = hf ? x0 : x1;
          f[0] = lsq_apass::narrow_f32(xa.x);
          f[1] = lsq_apass::narrow_f32(xa.y);
          f[2] = lsq_apass::narrow_f32(xb.x);
          f[3] = lsq_apass::narrow_f32(xb.y);
        } else {
          const float4 x = *reinterpret_cast<const float4*>(stage + r * DC + 4 * p4);
          f[0] = x.x;
          f[1] = x.y;
          f[2] = x.z;
          f[3] = x.w;
        }
        if (a32 != nullptr) {
          // the FP32 copy of A on the way (the narrowing of the solve's FP32 passes)
          const int64_t rg = i1 * N2 + r;
          const int cg = c0 + 4 * p4;
          if (rg < n) {
            float* o = a32 + rg * ld32 + cg;
            if (cg + 3 < d) {
              __stcs(reinterpret_cast<float4*>(o), make_float4(f[0], f[1], f[2], f[3]));
            } else {
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (cg + c < d) __stcs(o + c, f[c]);
            }
          }
        }
        const uint32_t neg = ((sgn[r >> 5] >> (r & 31)) & 1u) << 31;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c][j] = __uint_as_float(__float_as_uint(f[c]) ^ neg);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) butterflies<float, 3>(v[c]);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4*>(Z + zphys(qq + 256 * j, DC) + 4 * p4) = make_float4(v[0][j], v[1][j], v[2][j], v[3][j]);
    }
    __syncthreads();  // the staged block is consumed: the next one may land
    if (tid == 0 && i1 + 1 < b_end) {
      issue(i1 + 1);
      ++issued;
    }
    radix_pass<float, DC, 4>(Z, N2, 0);
    __syncthreads();
    radix_pass<float, DC, 4>(Z, N2, 4);
    __syncthreads();
    const uint32_t i1w = (uint32_t)i1 + blk0;  // the block's index in the whole (zero-padded) matrix
    // lanes 4..7 of each quarter-warp read the second half of their row first: rows fall on
    // even or odd 16-byte bank groups by half, so the two orders spread a quarter's reads
    const int hsw = (tid >> 2) & 1;
#pragma unroll
    for (int i = 0; i < MY; ++i) {
      const int s = tid + SRHT_THREADS * i;
      if (s < m) {
        const bool neg = (__popc(k1s[s] & i1w) & 1) != 0;
        const float4* zr = reinterpret_cast<const float4*>(Z + zphys(k2s[s], DC));
        const float4 z0 = zr[hsw], z1 = zr[hsw ^ 1];
        const float4 za = hsw ? z1 : z0, zb = hsw ? z0 : z1;
        y[i][0] += neg ? -za.x : za.x;
        y[i][1] += neg ? -za.y : za.y;
        y[i][2] += neg ? -za.z : za.z;
        y[i][3] += neg ? -za.w : za.w;
        y[i][4] += neg ? -zb.x : zb.x;
        y[i][5] += neg ? -zb.y : zb.y;
        y[i][6] += neg ? -zb.z : zb.z;
        y[i][7] += neg ? -zb.w : zb.w;
      }
    }
  }
  if (!ok && tid == 0 && issued > waited) {
    // a failed wait may leave a copy in flight: give it (bounded) time to land before exit
    (void)srht_mbar_wait(&full, (uint32_t)((issued - 1) & 1), err);
  }
  float* out = part + (gy * m_all + s0) * d;
#pragma unroll
  for (int i = 0; i < MY; ++i) {
    const int s = tid + SRHT_THREADS * i;
    if (s < m)
#pragma unroll
      for (int c = 0; c < DC; ++c)
        if (c0 + c < d) out[(int64_t)s * d + c0 + c] = ok ? y[i][c] : 0.f;
  }
}

// ------------------------------------------------------------------------------------
// SJLT: s distinct rows per column of S by Lemire's method on successive Philox words,
// then a shared-memory scatter of each data row into its s target rows.
// ------------------------------------------------------------------------------------
// The s target rows of data row i in SJLT instance t: Lemire's bounded integers in [0, m) from the
// successive words of Philox(i, draw, t, TAG_SJLT), duplicates skipped (at most 4096 draws).
template <int SMAX>
__device__ __forceinline__ void sjlt_targets(uint64_t seed, int64_t i, uint32_t t, int m, int s,
                                             int32_t (&picked)[SMAX]) {
  const uint32_t range = (uint32_t)m;
  const uint32_t threshold = (uint32_t)(0u - range) % range;
  int got = 0;
  for (uint32_t draw = 0; got < s && draw < 4096u; ++draw) {
    const uint4 w = philox_at(seed, (uint32_t)i, draw, t, TAG_SJLT);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (got >= s) break;
      const unsigned long long prod = (unsigned long long)words[k] * range;
      const uint32_t low = (uint32_t)prod;
      if (low < range && low < threshold) continue;
      const int32_t v = (int32_t)(prod >> 32);
      bool dup = false;
      for (int q = 0; q < got; ++q) dup |= (picked[q] == v);
      if (!dup) picked[got++] = v;
    }
  }
  for (int k = got; k < SMAX; ++k) picked[k] = 0;  // unreachable for s <= m; keeps every index in range
}

__global__ void sjlt_hash_kernel(int64_t n, int m, int s, uint64_t seed, uint32_t t, int32_t* __restrict__ h,
                                 uint32_t* __restrict__ signs, int64_t grow0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t picked[32];
    sjlt_targets<32>(seed, i + grow0, t, m, s, picked);  // column i + grow0 of S
    for (int k = 0; k < s; ++k) h[i * s + k] = picked[k];
    signs[i] = philox_at(seed, (uint32_t)(i + grow0), 0u, t, TAG_SJLT_SIGN).x;
  }
}

// The CTA owns a tile of DC columns (8 for FP32 arithmetic, 4 for FP64) and a range of
// rows; each thread takes whole rows of the tile: it loads
// the row's s positions, sign word and DC elements once and makes s * DC shared-memory
// additions.  Lane l visits the columns rotated by l, so the 32 lanes of an atomic spread
// over the banks instead of piling onto the DC banks of their targets.  The next row of
// each thread is loaded while the current one is scattered.
constexpr int SJLT_THREADS = 512;

template <typename TC, int DC>
__device__ __forceinline__ void rotate_by(TC (&a)[DC], int r) {
#pragma unroll
  for (int b = 1; b < DC; b <<= 1) {
    if (r & b) {
      TC t[DC];
#pragma unroll
      for (int c = 0; c < DC; ++c) t[c] = a[(c + b) & (DC - 1)];
#pragma unroll
      for (int c = 0; c < DC; ++c) a[c] = t[c];
    }
  }
}

// LSQ_SKETCH_BF16 for the SJLT: an element of A rounded to FP32, then to BF16 (nearest, ties to
// even); the +-1 signs are exact and the sums stay FP32
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <typename TC, int DC, int SMAX>
__device__ __forceinline__ void sjlt_load_row(const void* A, int dtype, int64_t ld, int c0, int d, int s,
                                              const int32_t* h, const uint32_t* signs, int64_t i, bool ok, TC (&a)[DC],
                                              int32_t (&tg)[SMAX], uint32_t& sw, bool bf16) {
#pragma unroll
  for (int c = 0; c < DC; ++c) a[c] = (ok && c0 + c < d) ? load_as<TC>(A, i * ld + c0 + c, dtype) : (TC)0;
  if constexpr (sizeof(TC) == 4) {
    if (bf16) {
#pragma unroll
      for (int c = 0; c < DC; ++c) a[c] = round_bf16(a[c]);
    }
  }
#pragma unroll
  for (int k = 0; k < SMAX; ++k) tg[k] = (ok && k < s) ? __ldg(h + i * s + k) : -1;
  sw = ok ? __ldg(signs + i) : 0u;
}

template <typename TC, int DC, int SMAX>
__global__ void __launch_bounds__(SJLT_THREADS, 1) sjlt_scatter_kernel(const void* __restrict__ A, int dtype,
                                                                      int64_t n, int d, int64_t ld, int m, int s,
                                                                      const int32_t* __restrict__ h,
                                                                      const uint32_t* __restrict__ signs,
                                                                      int64_t rows_per_group, TC* __restrict__ part,
                                                                      int bf16) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Y = reinterpret_cast<TC*>(smem_raw);  // [m][DC]
  const int c0 = blockIdx.x * DC;
  const int64_t i_begin = (int64_t)blockIdx.y * rows_per_group;
  const int64_t i_end = min(n, i_begin + rows_per_group);
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) Y[e] = (TC)0;
  __syncthreads();
  const int rot = (threadIdx.x & 31) & (DC - 1);
  TC a[DC], an[DC];
  int32_t tg[SMAX], tn[SMAX];
  uint32_t sw = 0, swn = 0;
  int64_t i = i_begin + threadIdx.x;
  sjlt_load_row<TC, DC, SMAX>(A, dtype, ld, c0, d, s, h, signs, i, i < i_end, a, tg, sw, bf16 != 0);
  for (; i < i_end; i += SJLT_THREADS) {
    const int64_t inext = i + SJLT_THREADS;
    sjlt_load_row<TC, DC, SMAX>(A, dtype, ld, c0, d, s, h, signs, inext, inext < i_end, an, tn, swn, bf16 != 0);
    rotate_by<TC, DC>(a, rot);
#pragma unroll
    for (int k = 0; k < SMAX; ++k) {
      if (k >= s) break;
      TC* yr = Y + (size_t)tg[k] * DC;
      const bool neg = (sw >> k) & 1u;
#pragma unroll
      for (int c = 0; c < DC; ++c) atomicAdd(yr + ((c + rot) & (DC - 1)), neg ? -a[c] : a[c]);
    }
#pragma unroll
    for (int c = 0; c < DC; ++c) a[c] = an[c];
#pragma unroll
    for (int k = 0; k < SMAX; ++k) tg[k] = tn[k];
    sw = swn;
  }
  __syncthreads();
  TC* out = part + (int64_t)blockIdx.y * m * d;
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) {
    const int row = e / DC, cc = e % DC;
    if (c0 + cc < d) out[(int64_t)row * d + c0 + cc] = Y[e];
  }
}

// Many SJLT sketches in one launch (FP32 arithmetic, 8-column tiles): work item (problem,
// column tile, row group) -> one CTA, which draws each row's targets and sign word itself
// (no hash pass: a problem with d columns redraws them d / 8 times, ~25 integer instructions
// an element), loads the row's 8 elements as two 16-byte vectors where A allows, and scatters
// them with shared-memory additions as sjlt_scatter_kernel does.
struct SjltJob {
  const void* A;
  int64_t n, ld, rpg;  // rows, row stride, rows per group
  float* part;         // [groups][m][d]
  int dtype, d, m, s, vec, bf16;
  uint32_t t;
};

template <int SMAX>
__global__ void __launch_bounds__(SJLT_THREADS, 1) sjlt_batched_kernel(const SjltJob* __restrict__ jobs,
                                                                      const int4* __restrict__ items,
                                                                      uint64_t seed) {
  constexpr int DC = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Y = reinterpret_cast<float*>(smem_raw);  // [m][DC]
  const int4 it = items[blockIdx.x];
  const SjltJob jb = jobs[it.x];
  const int c0 = it.y * DC, m = jb.m, s = jb.s, d = jb.d;
  const int64_t i_begin = (int64_t)it.z * jb.rpg;
  const int64_t i_end = min(jb.n, i_begin + jb.rpg);
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) Y[e] = 0.f;
  __syncthreads();
  const int rot = (threadIdx.x & 31) & (DC - 1);
  const bool vec = jb.vec != 0 && c0 + DC <= d;
  for (int64_t i = i_begin + threadIdx.x; i < i_end; i += SJLT_THREADS) {
    float a[DC];
    if (vec && jb.dtype == LSQ_F32) {
      const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(jb.A) + i * jb.ld + c0);
      const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
      a[0] = x0.x; a[1] = x0.y; a[2] = x0.z; a[3] = x0.w;
      a[4] = x1.x; a[5] = x1.y; a[6] = x1.z; a[7] = x1.w;
    } else {
#pragma unroll
      for (int c = 0; c < DC; ++c) a[c] = c0 + c < d ? load_as<float>(jb.A, i * jb.ld + c0 + c, jb.dtype) : 0.f;
    }
    if (jb.bf16) {
#pragma unroll
      for (int c = 0; c < DC; ++c) a[c] = round_bf16(a[c]);
    }
    int32_t tg[SMAX];
    sjlt_targets<SMAX>(seed, i, jb.t, m, s, tg);
    const uint32_t sw = philox_at(seed, (uint32_t)i, 0u, jb.t, TAG_SJLT_SIGN).x;
    rotate_by<float, DC>(a, rot);
#pragma unroll
    for (int k = 0; k < SMAX; ++k) {
      if (k >= s) break;
      float* yr = Y + (size_t)tg[k] * DC;
      const bool neg = (sw >> k) & 1u;
#pragma unroll
      for (int c = 0; c < DC; ++c) atomicAdd(yr + ((c + rot) & (DC - 1)), neg ? -a[c] : a[c]);
    }
  }
  __syncthreads();
  float* out = jb.part + (int64_t)it.z * m * d;
  for (int e = threadIdx.x; e < m * DC; e += blockDim.x) {
    const int row = e / DC, cc = e % DC;
    if (c0 + cc < d) out[(int64_t)row * d + c0 + cc] = Y[e];
  }
}

// SA_p = scale_p * sum over the groups of problem p's partials (double-FP32 sums), one launch;
// element e of the concatenation belongs to the problem whose prefix range holds it
__global__ void sjlt_batched_reduce_kernel(const SjltJob* __restrict__ jobs, const int64_t* __restrict__ prefix,
                                           const int* __restrict__ groups, double* const* __restrict__ SA, int nprob,
                                           int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const SjltJob& jb = jobs[lo];
    const int64_t md = (int64_t)jb.m * jb.d, k = e - prefix[lo];
    float h = 0.f, t = 0.f;
    for (int g = 0; g < groups[lo]; ++g) lsq_apass::df_add(h, t, jb.part[(int64_t)g * md + k], 0.f);
    SA[lo][k] = ((double)h + (double)t) / sqrt((double)jb.s);
  }
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
static int grid_for(int64_t work, int threads, int cap) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

static lsq_status validate_matrix(const lsq_matrix* A) {
  if (!A || !A->data) return LSQ_ERR_ARG;
  if (A->n < 1 || A->n >= (1ll << 31) || A->d < 1 || A->d > LSQ_MAX_D || A->ld < A->d) return LSQ_ERR_ARG;
  if (A->dtype != LSQ_F64 && A->dtype != LSQ_F32) return LSQ_ERR_ARG;
  const size_t es = A->dtype == LSQ_F64 ? 8 : 4;
  if (((uintptr_t)A->data) % es) return LSQ_ERR_ARG;
  return LSQ_OK;
}

template <typename TC>
static lsq_status gauss_run(lsq_ctx* ctx, const lsq_matrix* A, int m, uint64_t seed, uint32_t t, double* SA,
                            int64_t grow0) {
  const int d = (int)A->d;
  const int gx = lsq_ceil_div(m, GM), gy = lsq_ceil_div(d, GD);
  const int64_t ksteps = (A->n + GK - 1) / GK;
  int64_t splits = ((int64_t)2 * ctx->sm_count + gx * gy - 1) / (gx * gy);
  const int64_t cap = std::max<int64_t>(1, ((int64_t)256 << 20) / ((int64_t)m * d * (int64_t)sizeof(TC)));
  splits = std::max<int64_t>(1, std::min(std::min(splits, ksteps), cap));
  const int64_t rows_per_split = ((ksteps + splits - 1) / splits) * GK;
  splits = (A->n + rows_per_split - 1) / rows_per_split;
  lsq_status st = lsq_ensure_scratch(ctx, lsq_align256((size_t)splits * m * d * sizeof(TC)));
  if (st != LSQ_OK) return st;
  TC* part = reinterpret_cast<TC*>(ctx->scratch);
  dim3 grid(gx, gy, (unsigned)splits);
  gauss_sketch_kernel<TC><<<grid, 256, 0, ctx->stream>>>(A->data, A->dtype, A->n, d, A->ld, m, seed, t,
                                                          rows_per_split, part, grow0);
  LSQ_LAUNCH_CHECK();
  const int64_t md = (int64_t)m * d;
  reduce_splits_kernel<TC><<<grid_for(md, 256, 4 * ctx->sm_count), 256, 0, ctx->stream>>>(
      part, (int)splits, md, 1.0 / sqrt((double)m), SA);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

static size_t srht_smem_bytes(int logN2, int m, int dc, size_t es) {
  const size_t N2 = (size_t)1 << logN2;
  return (N2 + (N2 >> 4) + 1) * dc * es + (size_t)m * dc * es + (size_t)m * 6 + 64;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    (void)cudaGetLastError();
  }
  return fn;
}

// whether the TMA-staged kernel of the common case applies: A's layout allows tensor copies
// (16-byte aligned base and row stride), the sampled rows fit 8 register rows per thread and
// the staged block fits shared memory
template <typename TA>
static bool srht_tma_usable(const lsq_matrix* A, int m) {
  constexpr int DC = 8, N2 = 2048;
  const size_t es = sizeof(TA);
  if (((uintptr_t)A->data % 16) != 0 || ((size_t)A->ld * es) % 16 != 0) return false;
  const int ms = std::min(m, 8 * SRHT_THREADS);  // sampled rows per grid.z slice
  const size_t smem = 1024 + (size_t)N2 * DC * es + (size_t)zphys(N2, DC) * 4 + (size_t)ms * 4 +
                      (size_t)((ms + 1) & ~1) * 2 + (N2 / 32) * 4;
  return smem <= 232448 - 1024 && tensor_map_encoder() != nullptr;
}

// the TMA-staged kernel of the common case over row-block groups [gy0, gy0 + groups), when
// srht_tma_usable; returns false (nothing launched) otherwise
template <typename TA>
static bool srht_tma_launch(lsq_ctx* ctx, const lsq_matrix* A, int m, int64_t N1, const uint32_t* signbits,
                            const int64_t* rows, float* part, int groups, int64_t blocks_per_group, int* err,
                            float* a32, int64_t ld32, lsq_status* st, int gy0, uint32_t blk0) {
  constexpr int DC = 8, N2 = 2048;
  const size_t es = sizeof(TA);
  if (!srht_tma_usable<TA>(A, m)) return false;
  const int ms = std::min(m, 8 * SRHT_THREADS);
  const int slices = lsq_ceil_div(m, 8 * SRHT_THREADS);
  const size_t smem = 1024 + (size_t)N2 * DC * es + (size_t)zphys(N2, DC) * 4 + (size_t)ms * 4 +
                      (size_t)((ms + 1) & ~1) * 2 + (N2 / 32) * 4;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  CUtensorMap tm;
  const cuuint64_t dims[2] = {(cuuint64_t)A->d, (cuuint64_t)A->n};
  const cuuint64_t strides[1] = {(cuuint64_t)A->ld * es};
  const cuuint32_t box[2] = {(cuuint32_t)DC, (cuuint32_t)SRHT_TMA_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&tm, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(A->data),
          dims, strides,
          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const int d = (int)A->d;
  const dim3 grid(lsq_ceil_div(d, DC), groups, slices);
  auto launch = [&](auto kern) -> lsq_status {
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, SRHT_THREADS, smem, ctx->stream>>>(tm, A->n, d, N1, blocks_per_group, signbits, rows, m, part, err,
                                                     a32, ld32, gy0, blk0);
    LSQ_LAUNCH_CHECK();
    return LSQ_OK;
  };
  const int my = (ms + SRHT_THREADS - 1) / SRHT_THREADS;
  if (my <= 1) *st = launch(srht_tma_kernel<TA, 1>);
  else if (my <= 2) *st = launch(srht_tma_kernel<TA, 2>);
  else if (my <= 4) *st = launch(srht_tma_kernel<TA, 4>);
  else *st = launch(srht_tma_kernel<TA, 8>);
  return true;
}

template <typename TC, int DC>
static lsq_status srht_launch(lsq_ctx* ctx, const lsq_matrix* A, int m, int logN2, int64_t N1,
                              const uint32_t* signbits, const int64_t* rows, TC* part, int groups,
                              int64_t blocks_per_group, int* err, float* a32, int64_t ld32, bool& staged,
                              uint32_t blk0) {
  const int d = (int)A->d;
  const size_t smem = srht_smem_bytes(logN2, m, DC, sizeof(TC));
  dim3 grid(lsq_ceil_div(d, DC), groups);
  if constexpr (sizeof(TC) == 4 && DC == 8) {
    if (logN2 == 11) {
      lsq_status st = LSQ_OK;
      float* pf = reinterpret_cast<float*>(part);
      staged = A->dtype == LSQ_F64
                   ? srht_tma_launch<double>(ctx, A, m, N1, signbits, rows, pf, groups, blocks_per_group, err, a32,
                                             ld32, &st, 0, blk0)
                   : srht_tma_launch<float>(ctx, A, m, N1, signbits, rows, pf, groups, blocks_per_group, err, nullptr,
                                            0, &st, 0, blk0);
      if (staged) return st;
      const size_t es = A->dtype == LSQ_F64 ? 8 : 4;
      const size_t vb = 2 * es;  // bytes of one column pair
      const int vec_ok = (((uintptr_t)A->data % vb) == 0 && ((size_t)A->ld * es) % vb == 0) ? 1 : 0;
      if (A->dtype == LSQ_F64) {
        auto kf = srht_fast_kernel<double>;
        LSQ_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kf<<<grid, SRHT_THREADS, smem, ctx->stream>>>(reinterpret_cast<const double*>(A->data), A->n, d, A->ld, N1,
                                                      blocks_per_group, vec_ok, signbits, rows, m,
                                                      reinterpret_cast<float*>(part), blk0);
      } else {
        auto kf = srht_fast_kernel<float>;
        LSQ_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kf<<<grid, SRHT_THREADS, smem, ctx->stream>>>(reinterpret_cast<const float*>(A->data), A->n, d, A->ld, N1,
                                                      blocks_per_group, vec_ok, signbits, rows, m,
                                                      reinterpret_cast<float*>(part), blk0);
      }
      LSQ_LAUNCH_CHECK();
      return LSQ_OK;
    }
  }
  auto kern = srht_transform_kernel<TC, DC>;
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, SRHT_THREADS, smem, ctx->stream>>>(A->data, A->dtype, A->n, d, A->ld, logN2, N1, blocks_per_group,
                                                   signbits, rows, m, part, blk0);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

// lsq_upload_sketch: the host rows that become A (row stride host_ld elements)
struct SketchUpload {
  const void* host;
  int64_t host_ld;
};

// rows [r0, r1) of the host matrix into A's buffer, queued on `s`
static lsq_status upload_rows(const SketchUpload* up, const lsq_matrix* A, int64_t r0, int64_t r1, cudaStream_t s) {
  if (r1 <= r0) return LSQ_OK;
  const size_t es = A->dtype == LSQ_F64 ? 8 : 4;
  char* dst = static_cast<char*>(const_cast<void*>(A->data)) + (size_t)r0 * A->ld * es;
  const char* src = static_cast<const char*>(up->host) + (size_t)r0 * up->host_ld * es;
  if (A->ld == A->d && up->host_ld == A->d)
    LSQ_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)(r1 - r0) * A->d * es, cudaMemcpyHostToDevice, s));
  else
    LSQ_CUDA_TRY(cudaMemcpy2DAsync(dst, A->ld * es, src, up->host_ld * es, A->d * es, r1 - r0, cudaMemcpyHostToDevice,
                                   s));
  return LSQ_OK;
}

// the context's copy stream and event (created on first use)
static lsq_status ensure_copy_stream(lsq_ctx* ctx) {
  if (!ctx->copy) LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
  if (!ctx->ev_copy) LSQ_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_copy, cudaEventDisableTiming));
  return LSQ_OK;
}

template <typename TC>
static lsq_status srht_run(lsq_ctx* ctx, const lsq_matrix* A, int m, uint64_t seed, uint32_t t, double* SA,
                           float* a32, int64_t ld32, bool& a32_done, const SketchUpload* up, int64_t row0,
                           int64_t n_total) {
  const int d = (int)A->d;
  // the Hadamard transform spans the zero-padded rows of the whole matrix (n_total rows, of
  // which A holds [row0, row0 + n) as whole blocks of 2048 rows); signs and the sampled rows
  // are those of the whole matrix, and only the blocks that hold rows of A are transformed
  int64_t N = 1;
  int logN = 0;
  while (N < n_total) { N <<= 1; ++logN; }
  if (m > N) return LSQ_ERR_ARG;
  // shared memory: padded block + sampled accumulators + sample positions within the
  // 227 KB a CTA may opt into; 32-byte rows (DC * sizeof(TC) = 32) unless m forces narrower
  const size_t budget = 232448 - 1024;
  int DC = (int)(32 / sizeof(TC));
  int logN2 = std::min(logN, 11);
  auto fits = [&](int dc, int l2) { return srht_smem_bytes(l2, m, dc, sizeof(TC)) <= budget; };
  // the staged kernel keeps its sampled partials in registers (slices of 4096 rows), so the
  // shared-memory budget below, for the kernels that accumulate SA in shared memory, does not
  // apply to it
  const bool tma = sizeof(TC) == 4 && logN2 == 11 &&
                   (A->dtype == LSQ_F64 ? srht_tma_usable<double>(A, m) : srht_tma_usable<float>(A, m));
  if (!tma) {
    while (DC > 1 && !fits(DC, logN2)) DC >>= 1;
    while (logN2 > 0 && !fits(DC, logN2)) --logN2;
    if (!fits(DC, logN2) || logN2 > 16) return LSQ_ERR_ARG;
  }
  if (row0 % ((int64_t)1 << logN2) != 0) return LSQ_ERR_ARG;
  // blocks past the last row of A are all zero and add nothing
  const int64_t N1 = (A->n + ((int64_t)1 << logN2) - 1) >> logN2;
  const uint32_t blk0 = (uint32_t)(row0 >> logN2);
  const int tiles = lsq_ceil_div(d, DC);
  // about eight waves of one CTA per SM, so the last partial wave costs little
  int64_t groups = std::max<int64_t>(1, (8 * (int64_t)ctx->sm_count + tiles - 1) / tiles);
  groups = std::min(groups, N1);
  const int64_t cap = std::max<int64_t>(1, ((int64_t)256 << 20) / ((int64_t)m * d * (int64_t)sizeof(TC)));
  groups = std::min(groups, cap);
  const int64_t blocks_per_group = (N1 + groups - 1) / groups;
  groups = (N1 + blocks_per_group - 1) / blocks_per_group;

  const int64_t nscan = (N + SCAN_BLOCK - 1) / SCAN_BLOCK;
  size_t need = lsq_align256((size_t)N * 8) + lsq_align256((size_t)((N + 31) / 32) * 4) + lsq_align256(65536 * 4) +
                lsq_align256(4 * 8) + 2 * lsq_align256((size_t)nscan * 4) + lsq_align256((size_t)m * 8) +
                lsq_align256((size_t)groups * m * d * sizeof(TC)) + lsq_align256(4);
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  unsigned long long* keys = cv.take<unsigned long long>(N);
  uint32_t* signbits = cv.take<uint32_t>((N + 31) / 32);
  unsigned* hist = cv.take<unsigned>(65536);
  unsigned long long* state = cv.take<unsigned long long>(4);
  unsigned* cnt_lt = cv.take<unsigned>(nscan);
  unsigned* cnt_eq = cv.take<unsigned>(nscan);
  int64_t* rows = cv.take<int64_t>(m);
  TC* part = cv.take<TC>((size_t)groups * m * d);
  int* err = cv.take<int>(1);

  unsigned long long init_state[4] = {0ull, (unsigned long long)m, 0ull, 0ull};
  LSQ_CUDA_TRY(cudaMemsetAsync(hist, 0, 65536 * 4, ctx->stream));
  LSQ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  LSQ_CUDA_TRY(cudaMemcpyAsync(state, init_state, sizeof(init_state), cudaMemcpyHostToDevice, ctx->stream));
  srht_keys_kernel<<<grid_for(N, 256, 8 * ctx->sm_count), 256, 0, ctx->stream>>>(N, seed, t, keys, signbits, hist);
  LSQ_LAUNCH_CHECK();
  radix_pick_kernel<<<1, 1024, 0, ctx->stream>>>(hist, state);
  LSQ_LAUNCH_CHECK();
  for (int shift = 32; shift >= 0; shift -= 16) {
    radix_hist_kernel<<<grid_for(N, 256, 8 * ctx->sm_count), 256, 0, ctx->stream>>>(keys, N, shift, state, hist);
    LSQ_LAUNCH_CHECK();
    radix_pick_kernel<<<1, 1024, 0, ctx->stream>>>(hist, state);
    LSQ_LAUNCH_CHECK();
  }
  select_count_kernel<<<(unsigned)nscan, SCAN_BLOCK, 0, ctx->stream>>>(keys, N, state, cnt_lt, cnt_eq);
  LSQ_LAUNCH_CHECK();
  select_scan_kernel<<<1, 1024, 0, ctx->stream>>>(cnt_lt, cnt_eq, (int)nscan);
  LSQ_LAUNCH_CHECK();
  select_write_kernel<<<(unsigned)nscan, SCAN_BLOCK, 0, ctx->stream>>>(keys, N, state, cnt_lt, cnt_eq, rows, m);
  LSQ_LAUNCH_CHECK();

  // A's rows start at row0 of the whole matrix (a multiple of 32), and so do their sign bits
  const uint32_t* sb = signbits + (row0 >> 5);
  bool staged = false;
  bool launched = false;
  if (up) {
    const bool f64a = A->dtype == LSQ_F64;
    const bool chunked = sizeof(TC) == 4 && DC == 8 && logN2 == 11 &&
                         (f64a ? srht_tma_usable<double>(A, m) : srht_tma_usable<float>(A, m));
    if (!chunked) {
      st = upload_rows(up, A, 0, A->n, ctx->stream);  // the whole matrix first, in stream order
      if (st != LSQ_OK) return st;
    } else {
      // group g's rows go up on the copy stream (after the work already queued on the context
      // stream, which may still read A's buffer); its transform waits for them alone
      st = ensure_copy_stream(ctx);
      if (st != LSQ_OK) return st;
      LSQ_CUDA_TRY(cudaEventRecord(ctx->ev_copy, ctx->stream));
      LSQ_CUDA_TRY(cudaStreamWaitEvent(ctx->copy, ctx->ev_copy, 0));
      const int64_t rows_per_group = blocks_per_group * 2048;
      float* pf = reinterpret_cast<float*>(part);
      for (int64_t g = 0; g < groups; ++g) {
        const int64_t r0 = g * rows_per_group, r1 = std::min<int64_t>(A->n, r0 + rows_per_group);
        if (r1 > r0) {
          st = upload_rows(up, A, r0, r1, ctx->copy);
          if (st != LSQ_OK) return st;
          LSQ_CUDA_TRY(cudaEventRecord(ctx->ev_copy, ctx->copy));
          LSQ_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_copy, 0));
        }
        lsq_status lst = LSQ_OK;
        const bool ok = f64a ? srht_tma_launch<double>(ctx, A, m, N1, sb, rows, pf, 1, blocks_per_group, err, a32,
                                                       ld32, &lst, (int)g, blk0)
                             : srht_tma_launch<float>(ctx, A, m, N1, sb, rows, pf, 1, blocks_per_group, err,
                                                      nullptr, 0, &lst, (int)g, blk0);
        if (!ok) return LSQ_ERR_CUDA;  // srht_tma_usable said it would launch
        if (lst != LSQ_OK) return lst;
      }
      staged = launched = true;
    }
  }
  if (!launched) switch (DC) {
    case 8: st = srht_launch<TC, 8>(ctx, A, m, logN2, N1, sb, rows, part, (int)groups, blocks_per_group, err, a32,
                                  ld32, staged, blk0); break;
    case 4: st = srht_launch<TC, 4>(ctx, A, m, logN2, N1, sb, rows, part, (int)groups, blocks_per_group, err, a32,
                                  ld32, staged, blk0); break;
    case 2: st = srht_launch<TC, 2>(ctx, A, m, logN2, N1, sb, rows, part, (int)groups, blocks_per_group, err, a32,
                                  ld32, staged, blk0); break;
    default: st = srht_launch<TC, 1>(ctx, A, m, logN2, N1, sb, rows, part, (int)groups, blocks_per_group, err, a32,
                                  ld32, staged, blk0); break;
  }
  if (st != LSQ_OK) return st;
  const int64_t md = (int64_t)m * d;
  reduce_splits_kernel<TC><<<grid_for(md, 256, 4 * ctx->sm_count), 256, 0, ctx->stream>>>(
      part, (int)groups, md, 1.0 / sqrt((double)m), SA);
  LSQ_LAUNCH_CHECK();
  a32_done = staged && a32 != nullptr && A->dtype == LSQ_F64;
  if (staged) {
    // a timed-out wait on a staged block is reported here (or deferred)
    if (ctx->defer_checks) return lsq_defer_status(ctx, err, 0);
    LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 14, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LSQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->host_status[14]) return (lsq_status)ctx->host_status[14];
  }
  return LSQ_OK;
}

template <typename TC, int DC>
static lsq_status sjlt_launch(lsq_ctx* ctx, const lsq_matrix* A, int m, int s, const int32_t* h,
                              const uint32_t* signs, TC* part, int groups, int64_t rows_per_group, bool bf16) {
  const int d = (int)A->d;
  const size_t smem = (size_t)m * DC * sizeof(TC);
  dim3 grid(lsq_ceil_div(d, DC), groups);
  if (s <= 8) {
    auto kern = sjlt_scatter_kernel<TC, DC, 8>;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, SJLT_THREADS, smem, ctx->stream>>>(A->data, A->dtype, A->n, d, A->ld, m, s, h, signs,
                                                    rows_per_group, part, bf16 ? 1 : 0);
  } else {
    auto kern = sjlt_scatter_kernel<TC, DC, 32>;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, SJLT_THREADS, smem, ctx->stream>>>(A->data, A->dtype, A->n, d, A->ld, m, s, h, signs,
                                                    rows_per_group, part, bf16 ? 1 : 0);
  }
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

template <typename TC>
static lsq_status sjlt_run(lsq_ctx* ctx, const lsq_matrix* A, int m, int s, uint64_t seed, uint32_t t, double* SA,
                           bool bf16, int64_t grow0) {
  const int d = (int)A->d;
  const int64_t n = A->n;
  const size_t budget = 200 * 1024;
  int DC = (int)(sizeof(TC) == 8 ? 4 : 8);
  while (DC > 1 && (size_t)m * DC * sizeof(TC) > budget) DC >>= 1;
  if ((size_t)m * DC * sizeof(TC) > budget) return LSQ_ERR_ARG;
  const int tiles = lsq_ceil_div(d, DC);
  int64_t groups = std::max<int64_t>(1, (8 * (int64_t)ctx->sm_count + tiles - 1) / tiles);
  groups = std::min<int64_t>(groups, (n + 2047) / 2048);
  const int64_t cap = std::max<int64_t>(1, ((int64_t)256 << 20) / ((int64_t)m * d * (int64_t)sizeof(TC)));
  groups = std::max<int64_t>(1, std::min(groups, cap));
  const int64_t rows_per_group = (n + groups - 1) / groups;
  groups = (n + rows_per_group - 1) / rows_per_group;
  size_t need = lsq_align256((size_t)n * s * 4) + lsq_align256((size_t)n * 4) +
                lsq_align256((size_t)groups * m * d * sizeof(TC)) + lsq_align256(4);
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  int32_t* h = cv.take<int32_t>((size_t)n * s);
  uint32_t* signs = cv.take<uint32_t>(n);
  TC* part = cv.take<TC>((size_t)groups * m * d);
  sjlt_hash_kernel<<<grid_for(n, 256, 16 * ctx->sm_count), 256, 0, ctx->stream>>>(n, m, s, seed, t, h, signs, grow0);
  LSQ_LAUNCH_CHECK();
  switch (DC) {
    case 8: st = sjlt_launch<TC, 8>(ctx, A, m, s, h, signs, part, (int)groups, rows_per_group, bf16); break;
    case 4: st = sjlt_launch<TC, 4>(ctx, A, m, s, h, signs, part, (int)groups, rows_per_group, bf16); break;
    case 2: st = sjlt_launch<TC, 2>(ctx, A, m, s, h, signs, part, (int)groups, rows_per_group, bf16); break;
    default: st = sjlt_launch<TC, 1>(ctx, A, m, s, h, signs, part, (int)groups, rows_per_group, bf16); break;
  }
  if (st != LSQ_OK) return st;
  const int64_t md = (int64_t)m * d;
  reduce_splits_kernel<TC><<<grid_for(md, 256, 4 * ctx->sm_count), 256, 0, ctx->stream>>>(
      part, (int)groups, md, 1.0 / sqrt((double)s), SA);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

}  // namespace

lsq_status lsq_gauss_tc_run(lsq_ctx* ctx, const lsq_matrix* A, int m, uint64_t seed, uint32_t t, double* SA,
                            lsq_rows_hook rows_ready, void* hook_user, int64_t grow0);
lsq_status lsq_sjlt_tc_run(lsq_ctx* ctx, const lsq_matrix* A, int m, int s, uint64_t seed, uint32_t t, double* SA,
                           lsq_rows_hook rows_ready, void* hook_user, int64_t grow0);

// the hash pass of the SJLT (target rows in draw order and the sign word of every row of A)
lsq_status lsq_sjlt_hash_launch(lsq_ctx* ctx, int64_t n, int m, int s, uint64_t seed, uint32_t t, int64_t grow0,
                                int32_t* h, uint32_t* signs) {
  sjlt_hash_kernel<<<grid_for(n, 256, 16 * ctx->sm_count), 256, 0, ctx->stream>>>(n, m, s, seed, t, h, signs, grow0);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

// lsq_upload_sketch of the tensor-core Gaussian sketch: each chunk's rows go up on the copy stream
// (which first waits for the work already queued on the context stream, since it may still read
// A's buffer), and the context stream waits for them before the chunk is packed
struct ChunkUpload {
  lsq_ctx* ctx;
  const SketchUpload* up;
  const lsq_matrix* A;
  bool started;
};

static lsq_status chunk_upload(void* user, int64_t r0, int64_t r1, cudaStream_t consumer) {
  ChunkUpload* cu = static_cast<ChunkUpload*>(user);
  lsq_ctx* ctx = cu->ctx;
  if (!cu->started) {
    lsq_status st = ensure_copy_stream(ctx);
    if (st != LSQ_OK) return st;
    LSQ_CUDA_TRY(cudaEventRecord(ctx->ev_copy, ctx->stream));
    LSQ_CUDA_TRY(cudaStreamWaitEvent(ctx->copy, ctx->ev_copy, 0));
    cu->started = true;
  }
  lsq_status st = upload_rows(cu->up, cu->A, r0, r1, ctx->copy);
  if (st != LSQ_OK) return st;
  LSQ_CUDA_TRY(cudaEventRecord(ctx->ev_copy, ctx->copy));
  LSQ_CUDA_TRY(cudaStreamWaitEvent(consumer, ctx->ev_copy, 0));
  return LSQ_OK;
}

// the context stream waits for every copy queued on the copy stream, whatever path returned
static void join_copies(lsq_ctx* ctx) {
  if (!ctx->copy || !ctx->ev_copy) return;
  if (cudaEventRecord(ctx->ev_copy, ctx->copy) == cudaSuccess) cudaStreamWaitEvent(ctx->stream, ctx->ev_copy, 0);
}

static lsq_status sketch_impl(lsq_ctx* ctx, const lsq_matrix* A, int32_t type, int64_t m, uint64_t seed,
                              const lsq_sketch_opts* opts, double* SA, const SketchUpload* up) {
  if (!ctx || !SA) return LSQ_ERR_ARG;
  lsq_status st = validate_matrix(A);
  if (st != LSQ_OK) return st;
  if (m < 1 || m > 65536) return LSQ_ERR_ARG;
  const uint32_t t = opts ? opts->t : 0u;
  const int s = (opts && opts->s > 0) ? opts->s : 8;
  const int prec = opts ? opts->precision : LSQ_SKETCH_F64;
  if (prec != LSQ_SKETCH_F64 && prec != LSQ_SKETCH_F32 && prec != LSQ_SKETCH_BF16) return LSQ_ERR_ARG;
  if (prec == LSQ_SKETCH_BF16 && type != LSQ_SKETCH_GAUSS && type != LSQ_SKETCH_SJLT) return LSQ_ERR_ARG;
  const bool f64 = prec == LSQ_SKETCH_F64;
  float* a32 = (opts && A->dtype == LSQ_F64) ? opts->a32 : nullptr;
  const int64_t ld32 = a32 ? opts->ld32 : 0;
  if (a32 && (ld32 < A->d || ld32 % 4 != 0 || ((uintptr_t)a32 % 16) != 0)) return LSQ_ERR_ARG;
  bool a32_done = false;
  if (type != LSQ_SKETCH_GAUSS && type != LSQ_SKETCH_SRHT && type != LSQ_SKETCH_SJLT) return LSQ_ERR_ARG;
  // A as rows [row0, row0 + n) of a matrix of n_total rows: SA is that slab's share S[:, slab] A
  const int64_t row0 = opts ? opts->row0 : 0;
  const int64_t n_total = (opts && opts->n_total > 0) ? opts->n_total : A->n;
  if (row0 < 0 || row0 + A->n > n_total || n_total >= ((int64_t)1 << 31)) return LSQ_ERR_ARG;
  if (type == LSQ_SKETCH_SRHT && row0 % 2048 != 0) return LSQ_ERR_ARG;
  if (type == LSQ_SKETCH_SJLT && (s < 1 || s > 32 || s > m)) return LSQ_ERR_ARG;
  // the SRHT and the tensor-core Gaussian sketch consume the rows as they land; the other
  // sketches take the whole matrix first, in stream order
  const bool chunked_gauss = (type == LSQ_SKETCH_GAUSS || type == LSQ_SKETCH_SJLT) && prec == LSQ_SKETCH_BF16;
  if (up && type != LSQ_SKETCH_SRHT && !chunked_gauss) {
    st = upload_rows(up, A, 0, A->n, ctx->stream);
    if (st != LSQ_OK) return st;
  }
  ChunkUpload cu{ctx, up, A, false};
  switch (type) {
    case LSQ_SKETCH_GAUSS:
      if (prec == LSQ_SKETCH_BF16)
        st = lsq_gauss_tc_run(ctx, A, (int)m, seed, t, SA, up ? chunk_upload : nullptr, up ? &cu : nullptr, row0);
      else st = f64 ? gauss_run<double>(ctx, A, (int)m, seed, t, SA, row0)
                    : gauss_run<float>(ctx, A, (int)m, seed, t, SA, row0);
      break;
    case LSQ_SKETCH_SRHT:
      st = f64 ? srht_run<double>(ctx, A, (int)m, seed, t, SA, a32, ld32, a32_done, up, row0, n_total)
               : srht_run<float>(ctx, A, (int)m, seed, t, SA, a32, ld32, a32_done, up, row0, n_total);
      break;
    case LSQ_SKETCH_SJLT:
      if (s < 1 || s > 32 || s > m) return LSQ_ERR_ARG;
      if (prec == LSQ_SKETCH_BF16)  // on the tensor cores, in a fixed order
        st = lsq_sjlt_tc_run(ctx, A, (int)m, s, seed, t, SA, up ? chunk_upload : nullptr, up ? &cu : nullptr, row0);
      else
        st = f64 ? sjlt_run<double>(ctx, A, (int)m, s, seed, t, SA, false, row0)
                 : sjlt_run<float>(ctx, A, (int)m, s, seed, t, SA, false, row0);
      break;
    default:
      return LSQ_ERR_ARG;
  }
  // later work on the context stream sees all of A, also after an early error return
  if (up) join_copies(ctx);
  // the FP32 copy, where the sketch did not write it on the way
  if (st == LSQ_OK && a32 && !a32_done) st = lsq_narrow_copy(ctx, A, a32, ld32);
  return st;
}

extern "C" lsq_status lsq_sketch(lsq_ctx* ctx, const lsq_matrix* A, int32_t type, int64_t m, uint64_t seed,
                                 const lsq_sketch_opts* opts, double* SA) {
  return sketch_impl(ctx, A, type, m, seed, opts, SA, nullptr);
}

extern "C" lsq_status lsq_upload_sketch(lsq_ctx* ctx, const void* host_A, int64_t host_ld, const lsq_matrix* A,
                                        int32_t type, int64_t m, uint64_t seed, const lsq_sketch_opts* opts,
                                        double* SA) {
  if (!ctx || !host_A || !A || host_ld < A->d) return LSQ_ERR_ARG;
  const SketchUpload up{host_A, host_ld};
  return sketch_impl(ctx, A, type, m, seed, opts, SA, &up);
}

// Sketches of many problems in one launch (SJLT, FP32 arithmetic): problem p draws instance
// t = p of `seed` into SA[p] (m[p] x d FP64), exactly the embedding lsq_sketch would draw.
lsq_status lsq_sjlt_batched(lsq_ctx* ctx, int nprob, const lsq_matrix* A, const int* m, int s, uint64_t seed,
                            double* const* SA, int bf16) {
  if (nprob <= 0) return LSQ_OK;
  constexpr int DC = 8;
  std::vector<SjltJob> jobs(nprob);
  std::vector<int4> items;
  std::vector<int64_t> prefix(nprob);
  std::vector<int> groups(nprob);
  int64_t total = 0;
  size_t part_elems = 0;
  size_t smem_max = 0;
  for (int p = 0; p < nprob; ++p) {
    const lsq_matrix& a = A[p];
    const int d = (int)a.d, mp = m[p];
    const int sp = std::min(s, mp);
    if ((size_t)mp * DC * 4 > 200 * 1024 || sp < 1 || sp > 32) return LSQ_ERR_ARG;
    smem_max = std::max(smem_max, (size_t)mp * DC * 4);
    // about 16k rows per work item, at most 64 groups
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>(64, (a.n + 16383) / 16384));
    const int64_t rpg = (a.n + g - 1) / g;
    const int gp = (int)((a.n + rpg - 1) / rpg);
    const size_t es = a.dtype == LSQ_F64 ? 8 : 4;
    SjltJob& jb = jobs[p];
    jb.A = a.data;
    jb.n = a.n;
    jb.ld = a.ld;
    jb.rpg = rpg;
    jb.part = nullptr;
    jb.dtype = a.dtype;
    jb.d = d;
    jb.m = mp;
    jb.s = sp;
    jb.vec = (((uintptr_t)a.data % 16) == 0 && ((size_t)a.ld * es) % 16 == 0) ? 1 : 0;
    jb.bf16 = bf16 ? 1 : 0;
    jb.t = (uint32_t)p;
    groups[p] = gp;
    prefix[p] = total;
    total += (int64_t)mp * d;
    part_elems += (size_t)gp * mp * d;
    for (int ct = 0; ct < (d + DC - 1) / DC; ++ct)
      for (int gg = 0; gg < gp; ++gg) items.push_back(make_int4(p, ct, gg, 0));
  }
  // the costliest items first (rows of the group x sampled rows)
  std::stable_sort(items.begin(), items.end(), [&](const int4& x, const int4& y) {
    const double cx = (double)std::min<int64_t>(jobs[x.x].rpg, jobs[x.x].n) * jobs[x.x].m;
    const double cy = (double)std::min<int64_t>(jobs[y.x].rpg, jobs[y.x].n) * jobs[y.x].m;
    return cx > cy;
  });
  const size_t need = lsq_align256(part_elems * 4) + lsq_align256(nprob * sizeof(SjltJob)) +
                      lsq_align256(items.size() * sizeof(int4)) + lsq_align256(nprob * 8) +
                      lsq_align256(nprob * 4) + lsq_align256(nprob * sizeof(double*));
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  float* part = cv.take<float>(part_elems);
  SjltJob* d_jobs = cv.take<SjltJob>(nprob);
  int4* d_items = cv.take<int4>(items.size());
  int64_t* d_prefix = cv.take<int64_t>(nprob);
  int* d_groups = cv.take<int>(nprob);
  double** d_sa = cv.take<double*>(nprob);
  size_t off = 0;
  for (int p = 0; p < nprob; ++p) {
    jobs[p].part = part + off;
    off += (size_t)groups[p] * jobs[p].m * jobs[p].d;
  }
  cudaStream_t str = ctx->stream;
  LSQ_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), nprob * sizeof(SjltJob), cudaMemcpyHostToDevice, str));
  LSQ_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, str));
  LSQ_CUDA_TRY(cudaMemcpyAsync(d_prefix, prefix.data(), nprob * 8, cudaMemcpyHostToDevice, str));
  LSQ_CUDA_TRY(cudaMemcpyAsync(d_groups, groups.data(), nprob * 4, cudaMemcpyHostToDevice, str));
  LSQ_CUDA_TRY(cudaMemcpyAsync(d_sa, SA, nprob * sizeof(double*), cudaMemcpyHostToDevice, str));
  const int smax = s <= 8 ? 8 : 32;
  if (smax == 8) {
    auto kern = sjlt_batched_kernel<8>;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    kern<<<(unsigned)items.size(), SJLT_THREADS, smem_max, str>>>(d_jobs, d_items, seed);
  } else {
    auto kern = sjlt_batched_kernel<32>;
    LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    kern<<<(unsigned)items.size(), SJLT_THREADS, smem_max, str>>>(d_jobs, d_items, seed);
  }
  LSQ_LAUNCH_CHECK();
  sjlt_batched_reduce_kernel<<<grid_for(total, 256, 8 * ctx->sm_count), 256, 0, str>>>(d_jobs, d_prefix, d_groups,
                                                                                          d_sa, nprob, total);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}
