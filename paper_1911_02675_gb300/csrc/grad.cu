// grad.cu -- the data-matrix gradient of x* = H^{-1} b (differentiation through the solve).
//
// For a loss L(x*) with g = dL/dx*: lambda = H^{-1} g (a second solve with the forward's
// preconditioner), dL/db = lambda and
//     dL/dA = -(A x*) lambda^T - (A lambda) x*^T,
// obtained from dx* = H^{-1} (db - (dA^T A + A^T dA) x*) with H = A^T A (Section 1, problem
// statement).  This file computes dL/dA in one pass over A: per row, u_i = a_i . x* and
// w_i = a_i . lambda (FP64 arithmetic), then the row -(u_i lambda + w_i x*) is written.
#include <algorithm>

#include "common.cuh"

namespace {

template <typename TA, int EPL>
__global__ void __launch_bounds__(256) grad_a_kernel(const TA* __restrict__ A, int64_t n, int d, int64_t ld,
                                                     const double* __restrict__ x, const double* __restrict__ lam,
                                                     TA* __restrict__ gA, int64_t ldg) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double xv[EPL], lv[EPL];
#pragma unroll
  for (int k = 0; k < EPL; ++k) {
    const int c = lane + 32 * k;
    xv[k] = c < d ? x[c] : 0.0;
    lv[k] = c < d ? lam[c] : 0.0;
  }
  for (int64_t i = warp; i < n; i += nwarps) {
    const TA* a = A + i * ld;
    double av[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      const int c = lane + 32 * k;
      av[k] = c < d ? (double)__ldg(a + c) : 0.0;
    }
    double u = 0.0, w = 0.0;
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      u = fma(av[k], xv[k], u);
      w = fma(av[k], lv[k], w);
    }
    u = warp_sum(u);
    w = warp_sum(w);
    TA* out = gA + i * ldg;
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      const int c = lane + 32 * k;
      if (c < d) out[c] = (TA)(-(u * lv[k] + w * xv[k]));
    }
  }
}

template <typename TA>
lsq_status launch(lsq_ctx* ctx, const lsq_matrix* A, const double* x, const double* lam, void* gA, int64_t ldg) {
  const int d = (int)A->d;
  int epl = 1;
  while (32 * epl < d) epl <<= 1;
  const int64_t warps_needed = A->n;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((warps_needed + 7) / 8, 8 * (int64_t)ctx->sm_count));
  const TA* Ad = reinterpret_cast<const TA*>(A->data);
  TA* g = reinterpret_cast<TA*>(gA);
  switch (epl) {
    case 1: grad_a_kernel<TA, 1><<<grid, 256, 0, ctx->stream>>>(Ad, A->n, d, A->ld, x, lam, g, ldg); break;
    case 2: grad_a_kernel<TA, 2><<<grid, 256, 0, ctx->stream>>>(Ad, A->n, d, A->ld, x, lam, g, ldg); break;
    case 4: grad_a_kernel<TA, 4><<<grid, 256, 0, ctx->stream>>>(Ad, A->n, d, A->ld, x, lam, g, ldg); break;
    case 8: grad_a_kernel<TA, 8><<<grid, 256, 0, ctx->stream>>>(Ad, A->n, d, A->ld, x, lam, g, ldg); break;
    case 16: grad_a_kernel<TA, 16><<<grid, 256, 0, ctx->stream>>>(Ad, A->n, d, A->ld, x, lam, g, ldg); break;
    default: grad_a_kernel<TA, 32><<<grid, 256, 0, ctx->stream>>>(Ad, A->n, d, A->ld, x, lam, g, ldg); break;
  }
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}

}  // namespace

extern "C" lsq_status lsq_grad_a(lsq_ctx* ctx, const lsq_matrix* A, const double* x, const double* lam, void* gA,
                                 int64_t ldg) {
  if (!ctx || !A || !A->data || !x || !lam || !gA) return LSQ_ERR_ARG;
  if (A->n < 1 || A->n >= (1ll << 31) || A->d < 1 || A->d > LSQ_MAX_D || A->ld < A->d || ldg < A->d)
    return LSQ_ERR_ARG;
  if (A->dtype == LSQ_F64) return launch<double>(ctx, A, x, lam, gA, ldg);
  if (A->dtype == LSQ_F32) return launch<float>(ctx, A, x, lam, gA, ldg);
  return LSQ_ERR_ARG;
}
