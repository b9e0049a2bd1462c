// dist.cu -- the O(d^2) tail of a PCG iteration (Section 1, eq. (PCG)) as a call of its own,
// for solves whose passes over A are split by rows across GPUs.
//
// With A partitioned into row slabs A_p, H p = sum_p A_p^T (A_p p) and p^T H p = sum_p ||A_p p||^2,
// so one iteration is: every GPU runs the fused pass over its slab (lsq_hmatvec), the (d + 1)
// partial sums are added across GPUs (the only exchange per iteration), and every GPU applies
// this tail to the same sums, so that all of them hold the same x, r, z, p.
//
// One CTA of 1024 threads (d <= 1024): the vector updates, t = W^T r (thread j forms t_j from
// column j of W, coalesced over j), z = W t (a warp per row of W, lanes over its columns) and the
// block reductions run in order inside the kernel, so one launch is one tail.
#include <string.h>

#include "common.cuh"

namespace {

constexpr int TAIL_THREADS = 1024;

// state layout (caller-owned, (4d + 8) doubles): x, r, z, p (d each), then scalars
enum { S_RZ = 0, S_BX = 1, S_ALPHA = 2, S_BETA = 3, S_FLAG = 4, S_STATUS = 5, S_ITERS = 6 };

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  // every thread adds the warp sums in the same order, so all see the same total
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

__global__ void __launch_bounds__(TAIL_THREADS) pcg_tail_kernel(int d, const double* __restrict__ W,
                                                               const double* __restrict__ b,
                                                               const double* __restrict__ vq, int phase,
                                                               double tol, double rho, double* __restrict__ state) {
  __shared__ double t[1024];
  __shared__ double red[32];
  double* x = state;
  double* r = state + d;
  double* z = state + 2 * d;
  double* p = state + 3 * d;
  double* sc = state + 4 * d;
  const int tid = threadIdx.x;
  // the previous r^T z, read by every thread before thread 0 overwrites it at the end
  const double rz_old = sc[S_RZ];
  if (phase == 0) {
    // r = b - H x0 (vq = H x0 summed over the slabs; x is the caller's x0)
    for (int i = tid; i < d; i += blockDim.x) r[i] = b[i] - vq[i];
  } else {
    if (sc[S_FLAG] != 0.0) return;  // converged or failed: nothing changes
    const double q = vq[d];
    const double alpha = rz_old / q;
    if (!(q > 0.0) || !isfinite(alpha)) {
      if (tid == 0) {
        sc[S_FLAG] = 2.0;
        sc[S_STATUS] = (double)LSQ_ERR_BREAKDOWN;
      }
      return;
    }
    for (int i = tid; i < d; i += blockDim.x) {
      x[i] += alpha * p[i];
      r[i] -= alpha * vq[i];
    }
    if (tid == 0) sc[S_ALPHA] = alpha;
  }
  __syncthreads();
  // t = W^T r (W = R^{-1} upper triangular: t_j = sum_{i <= j} W[i][j] r_i)
  for (int j = tid; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i <= j; ++i) s = fma(W[(int64_t)i * d + j], r[i], s);
    t[j] = s;
  }
  __syncthreads();
  // z = W t (z_i = sum_{j >= i} W[i][j] t_j), a warp per row
  const int lane = tid & 31, warp = tid >> 5, warps = blockDim.x >> 5;
  for (int i = warp; i < d; i += warps) {
    double s = 0.0;
    for (int j = i + lane; j < d; j += 32) s = fma(W[(int64_t)i * d + j], t[j], s);
    s = warp_sum(s);
    if (lane == 0) z[i] = s;
  }
  __syncthreads();
  double rz = 0.0, bx = 0.0;
  for (int i = tid; i < d; i += blockDim.x) {
    rz = fma(r[i], z[i], rz);
    bx = fma(b[i], x[i], bx);
  }
  rz = block_sum(rz, red);
  bx = block_sum(bx, red);
  const double beta = phase == 0 ? 0.0 : rz / rz_old;
  for (int i = tid; i < d; i += blockDim.x) p[i] = phase == 0 ? z[i] : fma(beta, p[i], z[i]);
  if (tid == 0) {
    sc[S_RZ] = rz;
    sc[S_BX] = bx;
    sc[S_BETA] = beta;
    if (phase != 0) sc[S_ITERS] += 1.0;
    // the stopping rule of lsq_solve: (1 + sqrt(rho))^2 r^T H_S^{-1} r <= tol^2 <b, x>
    const double lam1 = (1.0 + sqrt(rho)) * (1.0 + sqrt(rho));
    if (!isfinite(rz)) {
      sc[S_FLAG] = 2.0;
      sc[S_STATUS] = (double)LSQ_ERR_BREAKDOWN;
    } else if (rz == 0.0 || lam1 * rz <= tol * tol * bx) {
      sc[S_FLAG] = 1.0;
    }
  }
}

}  // namespace

extern "C" lsq_status lsq_pcg_tail(lsq_ctx* ctx, int64_t d, const double* W, const double* b, const double* vq,
                                   int32_t phase, double tol, double rho, double* state, int32_t* flag_out) {
  if (!ctx || !W || !b || !vq || !state || d < 1 || d > 1024 || (phase != 0 && phase != 1) || !(rho > 0.0) ||
      !(rho < 1.0) || !(tol >= 0.0))
    return LSQ_ERR_ARG;
  if (phase == 0) {
    // fresh scalars; x (the caller's x0) is kept
    LSQ_CUDA_TRY(cudaMemsetAsync(state + 4 * d, 0, 8 * sizeof(double), ctx->stream));
  }
  pcg_tail_kernel<<<1, TAIL_THREADS, 0, ctx->stream>>>((int)d, W, b, vq, phase, tol, rho, state);
  LSQ_LAUNCH_CHECK();
  if (flag_out) {
    LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 20, state + 4 * d + S_FLAG, 2 * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    LSQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    double fs[2];
    memcpy(fs, ctx->host_status + 20, sizeof(fs));
    *flag_out = (int32_t)fs[0];
    if (fs[0] == 2.0) return (lsq_status)(int)fs[1];
  }
  return LSQ_OK;
}
