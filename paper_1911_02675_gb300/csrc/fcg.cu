// fcg.cu -- flexible conjugate gradients with refreshed embeddings: GCC (full
// orthogonalisation), FCG(k) and IPCG (k = 1) (Section 1, eqs.
// eqnconjugatedirectionsrefreshed and eqnflexiblecg; Section 4).  Iteration t:
//   v_t = H_{S_t}^{-1} r_t  (W_t W_t^T r_t with W_t = R_t^{-1} of the fresh sketch t),
//   p_t = v_t - sum_{j = t - k_t}^{t-1} <v_t, H p_j> / <p_j, H p_j> p_j,
//   alpha_t = <p_t, r_t> / <p_t, H p_t>,  x += alpha_t p_t,  r -= alpha_t H p_t.
// The host draws sketch t and factors it; one cooperative launch per iteration does the rest
// (bounded grid barriers).  H p_t comes from an exact pass (FP64, or double-FP32 in mixed
// mode) because the orthogonalisation relies on it; the stored p_j, H p_j stay FP64.
#include <algorithm>
#include <math.h>

#include "apass.cuh"
#include "common.cuh"

using namespace lsq_apass;

namespace {

struct FcgArgs {
  const void* A;
  int64_t n;
  int d, dp;
  int64_t ld, rows_per_cta;
  const double* b;
  const double* W;
  const double* WT;
  double* x;
  double* r;      // dp
  double* v;      // dp
  double* z;      // dp
  double* P;      // [maxit][dp] earlier directions
  double* HP;     // [maxit][dp] H times them
  double* qs;     // [maxit] <p_j, H p_j>
  double* coef;   // [maxit]
  double* part;   // [(dp+1)][P]
  double* red;    // [4][P]
  int t, kt;      // iteration index and window length
  double tol2;
  unsigned* bar;
  int* err;
  double* out;    // [0] converged flag, [1] est (r^T v / <b,x>), [2] status
};

__device__ __forceinline__ double row_dot(const double* __restrict__ row, const double* vec_s, int k_lo, int k_hi) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = k_lo + lane; k < k_hi; k += 32) s = fma(__ldg(row + k), vec_s[k], s);
  return warp_sum(s);
}

template <typename TA, int EPL, bool MIXED>
__global__ void __launch_bounds__(LSQ_THREADS, (EPL <= 16 ? 2 : 1)) fcg_step_kernel(FcgArgs a) {
  extern __shared__ __align__(16) double smem[];
  const int dp = a.dp, d = a.d;
  double* vec = smem;                     // dp: p
  double* wred = vec + dp;                // LSQ_WARPS * dp
  double* qred = wred + LSQ_WARPS * dp;   // LSQ_WARPS
  double* stage = qred + LSQ_WARPS;       // dp
  double* scal = stage + dp;              // 8
  const int P = gridDim.x, cta = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = cta * LSQ_WARPS + warp, nw = P * LSQ_WARPS;
  const int64_t r0 = (int64_t)cta * a.rows_per_cta, r1 = min(a.n, r0 + a.rows_per_cta);
  const TA* A = reinterpret_cast<const TA*>(a.A);
  double* red0 = a.red;
  double* red1 = a.red + P;

  auto cta_sum_to = [&](double mine, double* dst) {
    if (lane == 0) qred[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < LSQ_WARPS; ++w) s += qred[w];
      dst[cta] = s;
    }
    __syncthreads();
  };
  auto total = [&](const double* red) -> double {
    if (warp == 0) {
      const double s = warp_sum_strip(red, P);
      if (lane == 0) scal[7] = s;
    }
    __syncthreads();
    const double s = scal[7];
    __syncthreads();
    return s;
  };

  // v = W (W^T r), <r, v>; <b, x>
  for (int c = threadIdx.x; c < dp; c += blockDim.x) stage[c] = c < d ? a.r[c] : 0.0;
  __syncthreads();
  double bxp = 0.0;
  for (int i = gw; i < d; i += nw) {
    const double zi = row_dot(a.WT + (int64_t)i * d, stage, 0, i + 1);
    if (lane == 0) {
      a.z[i] = zi;
      bxp += a.b[i] * a.x[i];
    }
  }
  cta_sum_to(bxp, red1);
  if (grid_barrier(a.bar, P, a.err)) return;
  for (int c = threadIdx.x; c < dp; c += blockDim.x) stage[c] = c < d ? a.z[c] : 0.0;
  __syncthreads();
  double rvp = 0.0;
  for (int j = gw; j < d; j += nw) {
    const double vj = row_dot(a.W + (int64_t)j * d, stage, j, d);
    if (lane == 0) {
      a.v[j] = vj;
      rvp += vj * a.r[j];
    }
  }
  cta_sum_to(rvp, red0);
  if (grid_barrier(a.bar, P, a.err)) return;
  const double rv = total(red0), bx = total(red1);
  if (cta == 0 && threadIdx.x == 0) a.out[1] = bx > 0.0 ? rv / bx : 0.0;
  if (!isfinite(rv)) {
    if (cta == 0 && threadIdx.x == 0) a.out[2] = LSQ_ERR_BREAKDOWN;
    return;
  }
  if (rv == 0.0 || rv <= a.tol2 * bx) {
    if (cta == 0 && threadIdx.x == 0) a.out[0] = 1.0;
    return;
  }
  // coefficients against the window of earlier directions (one warp per direction)
  const int j0 = a.t - a.kt;
  for (int c = threadIdx.x; c < dp; c += blockDim.x) stage[c] = c < d ? a.v[c] : 0.0;
  __syncthreads();
  for (int jj = gw; jj < a.kt; jj += nw) {
    const int j = j0 + jj;
    const double s = row_dot(a.HP + (int64_t)j * dp, stage, 0, d);
    if (lane == 0) a.coef[jj] = s / a.qs[j];
  }
  if (grid_barrier(a.bar, P, a.err)) return;
  // p = v - sum coef_j p_j, whole in every CTA
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    double pc = c < d ? stage[c] : 0.0;
    for (int jj = 0; jj < a.kt; ++jj) pc -= a.coef[jj] * a.P[(int64_t)(j0 + jj) * dp + c];
    vec[c] = c < d ? pc : 0.0;
  }
  __syncthreads();
  if (cta == 0)
    for (int c = threadIdx.x; c < dp; c += blockDim.x) a.P[(int64_t)a.t * dp + c] = vec[c];
  if (MIXED) fused_pass_df<TA, EPL>(A, a.ld, d, dp, r0, r1, vec, wred, qred, a.part, P, cta);
  else fused_pass<TA, EPL, (EPL <= 4)>(A, a.ld, d, dp, r0, r1, vec, wred, qred, a.part, P, cta);
  if (grid_barrier(a.bar, P, a.err)) return;
  // H p per column; q = <p, H p>, <p, r>
  double qp = 0.0, prp = 0.0;
  for (int c = gw; c < d; c += nw) {
    const double hp = warp_sum_strip(a.part + (int64_t)c * P, P);
    if (lane == 0) {
      a.HP[(int64_t)a.t * dp + c] = hp;
      qp += vec[c] * hp;
      prp += vec[c] * a.r[c];
    }
  }
  cta_sum_to(qp, red0);
  cta_sum_to(prp, red1);
  if (grid_barrier(a.bar, P, a.err)) return;
  const double q = total(red0), pr = total(red1);
  if (!(q > 0.0) || !isfinite(q)) {
    if (cta == 0 && threadIdx.x == 0) a.out[2] = LSQ_ERR_BREAKDOWN;
    return;
  }
  const double alpha = pr / q;
  for (int c = gw; c < d; c += nw) {
    if (lane == 0) {
      a.x[c] += alpha * vec[c];
      a.r[c] -= alpha * a.HP[(int64_t)a.t * dp + c];
    }
  }
  if (cta == 0 && threadIdx.x == 0) a.qs[a.t] = q;
}

template <typename TA, bool MIXED>
void* pick(int epl) {
  switch (epl) {
    case 1: return (void*)fcg_step_kernel<TA, 1, MIXED>;
    case 2: return (void*)fcg_step_kernel<TA, 2, MIXED>;
    case 4: return (void*)fcg_step_kernel<TA, 4, MIXED>;
    case 8: return (void*)fcg_step_kernel<TA, 8, MIXED>;
    case 16: return (void*)fcg_step_kernel<TA, 16, MIXED>;
    default: return (void*)fcg_step_kernel<TA, 32, MIXED>;
  }
}

__global__ void transpose_into(const double* __restrict__ W, int d, double* __restrict__ WT) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = by + k, c = bx + threadIdx.x;
    tile[k][threadIdx.x] = (r < d && c < d) ? W[(int64_t)r * d + c] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = bx + k, c = by + threadIdx.x;
    if (r < d && c < d) WT[(int64_t)r * d + c] = tile[threadIdx.x][k];
  }
}

// r = b - H x0 from the partials of one FP64 pass
__global__ void residual_finish(const double* part, int P, int d, const double* b, double* r) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < d; c += nw) {
    const double s = warp_sum_strip(part + (int64_t)c * P, P);
    if (lane == 0) r[c] = b[c] - s;
  }
}

}  // namespace

// called by lsq_solve for LSQ_FCG; W = NULL draws a fresh embedding per iteration
lsq_status lsq_fcg_solve(lsq_ctx* ctx, const lsq_matrix* A, const double* b, const double* W_fixed, double* x,
                         double tol, int maxit, const lsq_solve_opts& o, double lam1, lsq_solve_info* info) {
  const int d = (int)A->d, epl = epl_for(d), dp = 32 * epl;
  const bool mixed = o.precision == LSQ_PREC_MIXED;
  void* kern = A->dtype == LSQ_F64 ? (mixed ? pick<double, true>(epl) : pick<double, false>(epl))
                                   : (mixed ? pick<float, true>(epl) : pick<float, false>(epl));
  const size_t smem = (size_t)(dp + LSQ_WARPS * dp + LSQ_WARPS + dp + 8) * 8;
  LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LSQ_THREADS, smem));
  if (per_sm < 1) return LSQ_ERR_CUDA;
  int P = per_sm * ctx->sm_count;
  if (o.grid_blocks > 0) P = std::min(P, o.grid_blocks);
  P = (int)std::min<int64_t>(P, std::max<int64_t>(1, (A->n + 31) / 32));
  const int64_t rows_per_cta = (A->n + P - 1) / P;
  P = (int)((A->n + rows_per_cta - 1) / rows_per_cta);
  const int hist = std::max(1, maxit);
  const size_t mat = (size_t)d * d;
  const size_t need = lsq_align256((size_t)(dp + 1) * P * 8) + lsq_align256((size_t)4 * P * 8) +
                      3 * lsq_align256((size_t)dp * 8) + 2 * lsq_align256((size_t)hist * dp * 8) +
                      2 * lsq_align256((size_t)hist * 8) + lsq_align256(mat * 8) + lsq_align256(64) +
                      lsq_align256(64) + lsq_align256((size_t)o.m * d * 8) + 2 * lsq_align256(mat * 8);
  lsq_status st = lsq_ensure_state(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->state), 0};
  FcgArgs a;
  a.part = cv.take<double>((size_t)(dp + 1) * P);
  a.red = cv.take<double>((size_t)4 * P);
  a.r = cv.take<double>(dp);
  a.v = cv.take<double>(dp);
  a.z = cv.take<double>(dp);
  a.P = cv.take<double>((size_t)hist * dp);
  a.HP = cv.take<double>((size_t)hist * dp);
  a.qs = cv.take<double>(hist);
  a.coef = cv.take<double>(hist);
  double* WT = cv.take<double>(mat);
  a.bar = cv.take<unsigned>(16);
  a.err = reinterpret_cast<int*>(a.bar + 8);
  a.out = cv.take<double>(8);
  double* SA = cv.take<double>((size_t)o.m * d);
  double* Rr = cv.take<double>(mat);
  double* Wr = cv.take<double>(mat);
  a.A = A->data;
  a.n = A->n;
  a.d = d;
  a.dp = dp;
  a.ld = A->ld;
  a.rows_per_cta = rows_per_cta;
  a.b = b;
  a.x = x;
  a.WT = WT;
  a.W = W_fixed ? W_fixed : Wr;
  a.tol2 = tol * tol / lam1;
  cudaStream_t s = ctx->stream;
  LSQ_CUDA_TRY(cudaEventRecord(ctx->ev0, s));
  int passes = 0;
  if (o.x0_zero) {
    LSQ_CUDA_TRY(cudaMemcpyAsync(a.r, b, (size_t)d * 8, cudaMemcpyDeviceToDevice, s));
  } else {  // r0 = b - H x0
    void* rk = A->dtype == LSQ_F64 ? pick_hmv<double>(epl) : pick_hmv<float>(epl);
    const size_t rs = hmatvec_smem_bytes(dp);
    LSQ_CUDA_TRY(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs));
    const void* Ad = A->data;
    int64_t n = A->n, ld = A->ld;
    int di = d, dpi = dp;
    int64_t rpc = rows_per_cta;
    const double* xp = x;
    double* pp = a.part;
    void* args[] = {(void*)&Ad, &n, &di, &dpi, &ld, &rpc, (void*)&xp, &pp};
    LSQ_CUDA_TRY(cudaLaunchKernel(rk, dim3(P), dim3(LSQ_THREADS), args, rs, s));
    lsq_count_launch();
    residual_finish<<<std::max(1, (d + 7) / 8), 256, 0, s>>>(a.part, P, d, b, a.r);
    LSQ_LAUNCH_CHECK();
    passes = 1;
  }
  if (W_fixed) {
    transpose_into<<<dim3((d + 31) / 32, (d + 31) / 32), dim3(32, 8), 0, s>>>(W_fixed, d, WT);
    LSQ_LAUNCH_CHECK();
  }
  lsq_sketch_opts so = {};
  so.s = o.s > 0 ? o.s : 8;
  so.precision = mixed ? LSQ_SKETCH_F32 : LSQ_SKETCH_F64;
  so.a32 = nullptr;
  so.ld32 = 0;
  int status = LSQ_ERR_MAXIT, t = 0;
  double est = 0.0, ms_sketch = 0.0;
  cudaEvent_t e_a, e_b;
  LSQ_CUDA_TRY(cudaEventCreate(&e_a));
  LSQ_CUDA_TRY(cudaEventCreate(&e_b));
  for (t = 0; t < maxit; ++t) {
    if (!W_fixed) {
      so.t = (uint32_t)t;
      cudaEventRecord(e_a, s);
      st = lsq_sketch(ctx, A, o.sketch_type, o.m, o.seed, &so, SA);
      if (st == LSQ_OK) st = lsq_factor(ctx, SA, o.m, d, Rr, Wr);
      cudaEventRecord(e_b, s);
      if (st != LSQ_OK) {
        status = st;
        break;
      }
      transpose_into<<<dim3((d + 31) / 32, (d + 31) / 32), dim3(32, 8), 0, s>>>(Wr, d, WT);
      LSQ_LAUNCH_CHECK();
    }
    a.t = t;
    a.kt = (o.fcg_k < 0 || o.fcg_k > t) ? t : o.fcg_k;
    LSQ_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(a.out, 0, 64, s));
    void* args[] = {&a};
    LSQ_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(P), dim3(LSQ_THREADS), args, smem, s));
    lsq_count_launch();
    LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status, a.out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 12, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    if (!W_fixed) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e_a, e_b);
      ms_sketch += ms;
    }
    const double* o3 = reinterpret_cast<const double*>(ctx->host_status);
    const int errc = ctx->host_status[12];
    est = sqrt(lam1 * fmax(o3[1], 0.0));
    if (errc) {
      status = errc;
      break;
    }
    if ((int)o3[2] != 0) {
      status = (int)o3[2];
      break;
    }
    if (o3[0] != 0.0) {
      status = LSQ_OK;
      break;
    }
    ++passes;
  }
  cudaEventRecord(ctx->ev1, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e_a);
  cudaEventDestroy(e_b);
  float ms_total = 0.f;
  cudaEventElapsedTime(&ms_total, ctx->ev0, ctx->ev1);
  (void)cudaGetLastError();
  if (info) {
    info->iters = t;
    info->status = status;
    info->passes = passes;
    info->exact_passes = passes;
    info->est_err = est;
    info->ms_total = ms_total;
    info->ms_sketch = ms_sketch;
    info->a32_copy = 0;
    info->reserved = 0;
  }
  return (lsq_status)status;
}
