// common.cuh -- internal helpers of the GB300 least-squares library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsq.h"

#define LSQ_WARPS 8
#define LSQ_THREADS (LSQ_WARPS * 32)
#define LSQ_MAX_D 1024

// Philox stream tags (counter word 3); must stay equal to the documented ABI values.
#define TAG_GAUSS 1u
#define TAG_SIGN 2u
#define TAG_SAMPLE 3u
#define TAG_SJLT 4u
#define TAG_SJLT_SIGN 5u

struct lsq_ctx {
  int device;
  int sm_count;
  cudaStream_t stream;
  void* scratch;           // device arena of sketch / factor / single passes, grown on demand
  size_t scratch_bytes;
  void* state;             // device arena of the solver's iteration state (separate, so that a
  size_t state_bytes;      // refreshed solve can call the sketch and the factor between steps)
  void* a32;               // FP32 copy of an FP64 A that a mixed-precision solve streams
  size_t a32_bytes;
  int* host_status;        // pinned host words for status read-back (32 ints; 16, 17: deferred)
  int* dev_pending;        // device words: first deferred sketch / factor error (0 = none)
  int32_t defer_checks;    // lsq_set_deferred_checks
  int32_t pending;         // deferred statuses may be set on the device
  cudaStream_t capture;    // non-blocking stream on which CUDA graphs are captured (lazily)
  cudaStream_t copy;       // non-blocking stream of lsq_upload_sketch's row copies (lazily)
  cudaEvent_t ev_copy;     // hand-over between the copy stream and the context stream
  cudaStream_t aux;        // non-blocking stream of the tensor-core sketch's packing (lazily)
  cudaEvent_t ev_aux[5];   // packed chunk ready (2), chunk's MMAs done (2), start (1)
  cudaEvent_t ev0, ev1;
};

#define LSQ_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t e__ = (expr);                      \
    if (e__ != cudaSuccess) {                      \
      (void)cudaGetLastError();                    \
      return LSQ_ERR_CUDA;                         \
    }                                              \
  } while (0)

// Deferred checks: keep the first nonzero *err of kind `slot` (0 sketch, 1 factor) on the
// device without waiting; lsq_pending_enqueue queues their read-back before a stream sync,
// lsq_pending_take reports (and clears) them after it.
lsq_status lsq_defer_status(lsq_ctx* c, const int* err, int slot);
lsq_status lsq_pending_enqueue(lsq_ctx* c);
lsq_status lsq_pending_take(lsq_ctx* c);

// Called by a sketch before work on stream `consumer` reads rows [r0, r1) of A
// (lsq_upload_sketch queues their copy and makes `consumer` wait for it).
typedef lsq_status (*lsq_rows_hook)(void* user, int64_t r0, int64_t r1, cudaStream_t consumer);

// Number of kernels this library has launched in the process (lsq_launch_count).
void lsq_count_launch();

#define LSQ_LAUNCH_CHECK()                         \
  do {                                             \
    lsq_count_launch();                            \
    cudaError_t e__ = cudaGetLastError();          \
    if (e__ != cudaSuccess) return LSQ_ERR_CUDA;   \
  } while (0)

// Ensures the context arena holds at least `bytes` (256-byte aligned carving is the caller's).
lsq_status lsq_ensure_scratch(lsq_ctx* ctx, size_t bytes);
lsq_status lsq_ensure_state(lsq_ctx* ctx, size_t bytes);
lsq_status lsq_ensure_a32(lsq_ctx* ctx, size_t bytes);
// SJLT sketches of nprob problems in one launch (FP32 arithmetic, over BF16-rounded A when bf16;
// instance t = p) (sketch.cu)
lsq_status lsq_sjlt_batched(lsq_ctx* ctx, int nprob, const lsq_matrix* A, const int* m, int s, uint64_t seed,
                            double* const* SA, int bf16);
// a32[i * ld32 + c] = FP32 narrowing of A[i][c] (FP64 A), on the context's stream (solve.cu)
lsq_status lsq_narrow_copy(lsq_ctx* ctx, const lsq_matrix* A, float* a32, int64_t ld32);

// Factorisations of many sketches (batched solves): W_p = R_p^{-1} and W_p^T; status_out[p]
// (host) = LSQ_OK or LSQ_ERR_RANK; the Gram matrices in double-FP32 when df_gram.
lsq_status lsq_factor_batched(lsq_ctx* ctx, int nprob, const double* const* SA, const int* m, const int* d,
                              double* const* W, double* const* WT, bool df_gram, int* status_out);

// LSQ_FCG behind lsq_solve (arguments already checked; W_fixed = NULL refreshes)
lsq_status lsq_fcg_solve(lsq_ctx* ctx, const lsq_matrix* A, const double* b, const double* W_fixed, double* x,
                         double tol, int maxit, const lsq_solve_opts& o, double lam1, lsq_solve_info* info);

static inline size_t lsq_align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves consecutive 256-byte aligned regions out of a base pointer.
struct Carver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += lsq_align256(count * sizeof(T));
    return p;
  }
};

// ----------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, multipliers
// 0xD2511F53 / 0xCD9E8D57, key increments 0x9E3779B9 / 0xBB67AE85.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_at(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t t, uint32_t tag) {
  return philox4x32_10(make_uint4(c0, c1, t, tag), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ----------------------------------------------------------------------------------
// Warp reductions (fixed butterfly order: every lane ends with the same value).
// ----------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ----------------------------------------------------------------------------------
// Grid-wide barrier for cooperatively launched kernels, with a bounded wait.
// `bar[0]` counts arrivals, `bar[1]` is the generation.  A CTA that waits more than
// `LSQ_SPIN_LIMIT` polls sets *err = LSQ_ERR_TIMEOUT and leaves the barrier; callers
// test the flag after every barrier and return, so the kernel always terminates.
// ----------------------------------------------------------------------------------
#define LSQ_SPIN_LIMIT (1u << 24)
#define LSQ_WAIT_NS 4000000000ull

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int grid_barrier_bounded(unsigned* bar, unsigned nblocks, int* err, unsigned spin_limit,
                                                    uint64_t wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(bar + 1) == gen) {
        if (*(volatile int*)err != 0) break;  // another CTA already gave up
        if (++spins > spin_limit || global_ns() - t0 > wait_ns) {
          atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err;
}

__device__ __forceinline__ int grid_barrier(unsigned* bar, unsigned nblocks, int* err) {
  return grid_barrier_bounded(bar, nblocks, err, LSQ_SPIN_LIMIT, LSQ_WAIT_NS);
}

// Grid-wide barrier over an arrival count that only grows within a launch (zeroed before
// it): every CTA passes the same sequence of barriers, so the k-th one of each CTA waits for
// the count to reach k * nblocks (`target` is the CTA's running k * nblocks).  Nothing is
// reset, so the last arrival costs one add and each waiter one acquire load per poll.  The
// CTA barrier orders its threads' writes before thread 0's release-add, the release is
// cumulative, and the acquire load that sees the count orders the reads after the closing
// CTA barrier, so no separate fence is needed.  The wait is bounded like grid_barrier's.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int grid_sync_count_bounded(unsigned long long* cnt, unsigned long long& target,
                                                       unsigned nblocks, int* err, unsigned spin_limit,
                                                       uint64_t wait_ns) {
  __syncthreads();
  target += nblocks;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
    const uint64_t t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire_u64(cnt) < target) {
      if (*(volatile int*)err != 0) break;  // another CTA already gave up
      if (++spins > spin_limit || global_ns() - t0 > wait_ns) {
        atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
  return *(volatile int*)err;
}

__device__ __forceinline__ int grid_sync_count(unsigned long long* cnt, unsigned long long& target, unsigned nblocks,
                                               int* err) {
  return grid_sync_count_bounded(cnt, target, nblocks, err, LSQ_SPIN_LIMIT, LSQ_WAIT_NS);
}

static inline int lsq_ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
