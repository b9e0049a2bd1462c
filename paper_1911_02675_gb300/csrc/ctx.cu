// ctx.cu -- context, scratch arena and status strings of the C ABI.
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "common.cuh"

extern "C" lsq_status lsq_create(lsq_ctx** out, void* stream) {
  if (!out) return LSQ_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  LSQ_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  LSQ_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  if (!prop.cooperativeLaunch) return LSQ_ERR_CUDA;
  lsq_ctx* c = (lsq_ctx*)calloc(1, sizeof(lsq_ctx));
  if (!c) return LSQ_ERR_ALLOC;
  c->device = dev;
  c->sm_count = prop.multiProcessorCount;
  c->stream = (cudaStream_t)stream;
  if (cudaMallocHost((void**)&c->host_status, 128) != cudaSuccess || cudaMalloc((void**)&c->dev_pending, 8) != cudaSuccess ||
      cudaMemset(c->dev_pending, 0, 8) != cudaSuccess || cudaEventCreate(&c->ev0) != cudaSuccess ||
      cudaEventCreate(&c->ev1) != cudaSuccess) {
    (void)cudaGetLastError();
    if (c->host_status) cudaFreeHost(c->host_status);
    if (c->dev_pending) cudaFree(c->dev_pending);
    free(c);
    return LSQ_ERR_CUDA;
  }
  memset(c->host_status, 0, 128);
  *out = c;
  return LSQ_OK;
}

extern "C" lsq_status lsq_destroy(lsq_ctx* c) {
  if (!c) return LSQ_OK;
  cudaStreamSynchronize(c->stream);
  if (c->scratch) cudaFree(c->scratch);
  if (c->state) cudaFree(c->state);
  if (c->a32) cudaFree(c->a32);
  if (c->capture) cudaStreamDestroy(c->capture);
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
  }
  if (c->ev_copy) cudaEventDestroy(c->ev_copy);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
  }
  for (cudaEvent_t e : c->ev_aux)
    if (e) cudaEventDestroy(e);
  cudaFreeHost(c->host_status);
  cudaFree(c->dev_pending);
  cudaEventDestroy(c->ev0);
  cudaEventDestroy(c->ev1);
  (void)cudaGetLastError();
  free(c);
  return LSQ_OK;
}

extern "C" lsq_status lsq_set_stream(lsq_ctx* c, void* stream) {
  if (!c) return LSQ_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return LSQ_OK;
}

extern "C" lsq_status lsq_set_deferred_checks(lsq_ctx* c, int32_t on) {
  if (!c) return LSQ_ERR_ARG;
  c->defer_checks = on ? 1 : 0;
  return LSQ_OK;
}

namespace {
__global__ void keep_first_status_kernel(const int* err, int* slot) {
  if (*slot == 0) *slot = *err;
}
}  // namespace

lsq_status lsq_defer_status(lsq_ctx* c, const int* err, int slot) {
  keep_first_status_kernel<<<1, 1, 0, c->stream>>>(err, c->dev_pending + slot);
  LSQ_LAUNCH_CHECK();
  c->pending = 1;
  return LSQ_OK;
}

lsq_status lsq_pending_enqueue(lsq_ctx* c) {
  if (c->pending)
    LSQ_CUDA_TRY(cudaMemcpyAsync(c->host_status + 16, c->dev_pending, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
  return LSQ_OK;
}

lsq_status lsq_pending_take(lsq_ctx* c) {
  if (!c->pending) return LSQ_OK;
  c->pending = 0;
  const int e = c->host_status[16] ? c->host_status[16] : c->host_status[17];
  if (e) {
    c->host_status[16] = c->host_status[17] = 0;
    LSQ_CUDA_TRY(cudaMemsetAsync(c->dev_pending, 0, 2 * sizeof(int), c->stream));
  }
  return (lsq_status)e;
}

extern "C" lsq_status lsq_sync(lsq_ctx* c) {
  if (!c) return LSQ_ERR_ARG;
  lsq_status st = lsq_pending_enqueue(c);
  if (st != LSQ_OK) return st;
  LSQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return lsq_pending_take(c);
}

static lsq_status grow(lsq_ctx* c, void** buf, size_t* have, size_t bytes) {
  if (bytes <= *have) return LSQ_OK;
  // the old buffer may still be in use by work queued on the stream
  LSQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (*buf) {
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  size_t want = lsq_align256(bytes + (bytes >> 3));
  if (cudaMalloc(buf, want) != cudaSuccess) {
    (void)cudaGetLastError();
    *buf = nullptr;
    return LSQ_ERR_ALLOC;
  }
  *have = want;
  return LSQ_OK;
}

lsq_status lsq_ensure_scratch(lsq_ctx* c, size_t bytes) { return grow(c, &c->scratch, &c->scratch_bytes, bytes); }

lsq_status lsq_ensure_state(lsq_ctx* c, size_t bytes) { return grow(c, &c->state, &c->state_bytes, bytes); }

lsq_status lsq_ensure_a32(lsq_ctx* c, size_t bytes) { return grow(c, &c->a32, &c->a32_bytes, bytes); }

extern "C" const char* lsq_status_str(int32_t s) {
  switch (s) {
    case LSQ_OK: return "ok";
    case LSQ_ERR_ARG: return "invalid argument";
    case LSQ_ERR_RANK: return "sketched Hessian not positive definite (rank deficient)";
    case LSQ_ERR_BREAKDOWN: return "iteration breakdown (non-positive curvature or non-finite value)";
    case LSQ_ERR_MAXIT: return "tolerance not reached within maxit iterations";
    case LSQ_ERR_TIMEOUT: return "bounded device-side wait timed out";
    case LSQ_ERR_CUDA: return "CUDA runtime error";
    case LSQ_ERR_ALLOC: return "device allocation failed";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------------
// lsq_selftest_wait: one cooperative launch of the grid barriers every cooperative kernel of
// the library uses, waiting for `missing` arrivals more than the grid has.  With missing > 0
// no CTA can pass, so each waiter gives up at the limit and the launch ends with
// LSQ_ERR_TIMEOUT, the path every bounded wait takes.
// ---------------------------------------------------------------------------------
namespace {
__global__ void selftest_wait_kernel(int kind, unsigned missing, uint64_t wait_ns, void* bar, int* err) {
  const unsigned nblocks = gridDim.x + missing;
  if (kind == 0) {
    unsigned long long target = 0;
    grid_sync_count_bounded(static_cast<unsigned long long*>(bar), target, nblocks, err, LSQ_SPIN_LIMIT, wait_ns);
  } else {
    grid_barrier_bounded(static_cast<unsigned*>(bar), nblocks, err, LSQ_SPIN_LIMIT, wait_ns);
  }
}
}  // namespace

extern "C" lsq_status lsq_selftest_wait(lsq_ctx* c, int32_t kind, int32_t missing, int64_t wait_ns) {
  if (!c || (kind != 0 && kind != 1) || missing < 0 || missing > 1024) return LSQ_ERR_ARG;
  const uint64_t limit = wait_ns > 0 ? (uint64_t)wait_ns : LSQ_WAIT_NS;
  if (limit > LSQ_WAIT_NS) return LSQ_ERR_ARG;
  lsq_status st = lsq_ensure_scratch(c, 256);
  if (st != LSQ_OK) return st;
  int* err = reinterpret_cast<int*>(c->scratch);
  void* bar = reinterpret_cast<char*>(c->scratch) + 64;
  LSQ_CUDA_TRY(cudaMemsetAsync(c->scratch, 0, 128, c->stream));
  int k = kind;
  unsigned miss = (unsigned)missing;
  uint64_t ns = limit;
  void* args[] = {&k, &miss, &ns, &bar, &err};
  LSQ_CUDA_TRY(cudaLaunchCooperativeKernel((void*)selftest_wait_kernel, dim3(c->sm_count), dim3(128), args, 0,
                                           c->stream));
  lsq_count_launch();
  LSQ_CUDA_TRY(cudaMemcpyAsync(c->host_status + 15, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LSQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return (lsq_status)c->host_status[15];
}

static std::atomic<unsigned long long> g_launches{0};

void lsq_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" uint64_t lsq_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char* lsq_version(void) { return "lsq-gb300 0.1 (sm_103a)"; }
