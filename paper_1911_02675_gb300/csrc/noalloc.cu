// noalloc.cu -- lsq_hmatvec_noalloc: the fused pass over A (v = A^T (A p), q = ||A p||^2)
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that must hand every byte of device memory to
// its own pool allocator (and treats any other allocation as a leak or a failure), and
// latency-bound loops that cannot afford the implicit device synchronisation an allocation
// may bring.  This entry point needs no context and allocates nothing: its only scratch,
// the per-CTA partial sums of the pass, lives in a fixed array in this file.
#include <algorithm>
#include <mutex>

#include "apass.cuh"
#include "common.cuh"

using namespace lsq_apass;

// Per-CTA partials of the pass: (dp + 1) doubles per CTA, dp = d rounded up to a power of
// two times 32 (at most 1024).  160 x 1025 doubles = 1.25 MiB, held by every GPU that loads
// the library until the process exits.  Enough for 160 CTAs at d = 1024 (more at smaller d).
#define LSQ_NOALLOC_SCRATCH_DOUBLES (160 * 1025)
static __device__ __align__(256) double g_noalloc_scratch[LSQ_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_sm_count[kMaxDevices];

// Once per device, with that device current: the device address of the array.  In host
// code `g_noalloc_scratch` names a host-side stand-in, never a device address.
lsq_status setup_device(int dev, double** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return LSQ_ERR_CUDA;
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n < 1) {
      (void)cudaGetLastError();
      return LSQ_ERR_CUDA;
    }
    g_sm_count[dev] = n;
    g_scratch_ptr[dev] = reinterpret_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  *sms = g_sm_count[dev];
  return LSQ_OK;
}

}  // namespace

extern "C" lsq_status lsq_hmatvec_noalloc(const lsq_matrix* A, const double* p, double* v, double* q,
                                          void* cuda_stream) {
  if (!A || !A->data || !p || !v || !q) return LSQ_ERR_ARG;
  if (A->n < 1 || A->n >= (1ll << 31) || A->d < 1 || A->d > LSQ_MAX_D || A->ld < A->d) return LSQ_ERR_ARG;
  if (A->dtype != LSQ_F64 && A->dtype != LSQ_F32) return LSQ_ERR_ARG;
  if (((uintptr_t)A->data) % (A->dtype == LSQ_F64 ? 8 : 4)) return LSQ_ERR_ARG;
  int dev = 0;
  LSQ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return LSQ_ERR_ARG;
  double* part = nullptr;
  int sms = 0;
  lsq_status st = setup_device(dev, &part, &sms);
  if (st != LSQ_OK) return st;

  const int d = (int)A->d, epl = epl_for(d), dp = 32 * epl;
  void* kern = A->dtype == LSQ_F64 ? pick_hmv<double>(epl) : pick_hmv<float>(epl);
  const size_t smem = hmatvec_smem_bytes(dp);
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LSQ_THREADS, smem));
  int64_t P = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  P = std::min<int64_t>(P, (A->n + 31) / 32);
  P = std::min<int64_t>(P, LSQ_NOALLOC_SCRATCH_DOUBLES / (dp + 1));
  if (P < 1) return LSQ_ERR_ARG;
  const int64_t rows_per_cta = (A->n + P - 1) / P;
  P = (A->n + rows_per_cta - 1) / rows_per_cta;
  if ((P * (dp + 1)) > LSQ_NOALLOC_SCRATCH_DOUBLES) return LSQ_ERR_ARG;  // beyond the fixed scratch

  // Every partial the reduction reads is written by the pass first, so the array's
  // contents from an earlier call need no clearing.
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const void* Ad = A->data;
  int64_t n = A->n, ld = A->ld;
  int di = d, dpi = dp;
  void* args[] = {(void*)&Ad, &n, &di, &dpi, &ld, (void*)&rows_per_cta, (void*)&p, &part};
  LSQ_CUDA_TRY(cudaLaunchKernel(kern, dim3((unsigned)P), dim3(LSQ_THREADS), args, smem, s));
  lsq_count_launch();
  reduce_part_kernel<<<std::max(1, (d + 1 + 7) / 8), 256, 0, s>>>(part, (int)P, d, dp, v, q);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}
