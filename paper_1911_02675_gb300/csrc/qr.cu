// qr.cu -- the preconditioner factor by Householder QR with column pivoting of SA (Section 1,
// PCG paragraph: the factor of H_S may come from a pivoted QR of SA instead of a Cholesky
// factor of (SA)^T (SA)); SA[:, perm] = Q R, so H_S = P R^T R P^T and H_S^{-1} = W W^T with
// W = P R^{-1} (rows of R^{-1} permuted: dense as stored, which lsq_solve takes with
// lsq_solve_opts.w_dense = 1).  Working on SA itself, the factor's error grows with cond(SA),
// not with cond(SA)^2 as the Gram route does.
//
// qrp_kernel (cooperative, FP64): T = SA^T, so a column of SA is a contiguous row of T.  Step
// k: every CTA takes the pivot -- the active column of largest remaining norm (rows k..m-1),
// ties to the lower position -- from the norms the previous step left, and swaps it into
// position k of its own copy of the permutation (shared memory; the same in every CTA, so no
// data moves); the reflector v = x - alpha e_k of the pivot column x (alpha = -sign(x_k) |x|)
// needs |x|^2 and sum_{r>k} x_r^2, which the previous step also left; then a warp per other
// active column applies I - 2 v v^T / v^T v, writes its entry of row k of R and the two norms
// the next step needs (rows >= k + 1 and >= k + 2); one bounded grid barrier ends the step.
// The numerical rank is the number of steps before the largest remaining norm falls to
// tol times the first pivot's norm.  Rows of R are kept by original column index and put in
// pivot order (with positive diagonal) afterwards.
#include "common.cuh"

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;

struct QrArgs {
  double* T;        // d x m, T[c][r] = SA[r][c] (overwritten)
  int64_t m;
  int d;
  double tol;
  double* n1;       // d: sum of squares of rows >= k of each column (the pivot norm at step k)
  double* n2;       // d: the same over rows >= k + 1
  double* Ro;       // d x d, rows of R by original column index (zeroed before)
  int32_t* perm;    // d (out)
  int* rank;        // (out)
  double* alpha;    // d: R[k][k] before the sign fix
  unsigned long long* bar;
  int* err;
};

__global__ void transpose_sa_kernel(const double* __restrict__ SA, int64_t m, int d, double* __restrict__ T) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k;
    const int c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < m && c < d) ? SA[r * d + c] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k;
    const int64_t r = r0 + threadIdx.x;
    if (c < d && r < m) T[(int64_t)c * m + r] = tile[threadIdx.x][k];
  }
}

// n1, n2 of every column at step 0 (a warp per column)
__global__ void qrp_norms_kernel(const double* __restrict__ T, int64_t m, int d, double* n1, double* n2) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= d) return;
  const double* x = T + (int64_t)w * m;
  double s = 0.0;
  for (int64_t r = 1 + lane; r < m; r += 32) s = fma(x[r], x[r], s);
  s = warp_sum(s);
  if (lane == 0) {
    n2[w] = s;
    n1[w] = s + x[0] * x[0];
  }
}

__global__ void __launch_bounds__(QR_THREADS) qrp_kernel(QrArgs a) {
  __shared__ int32_t perm[1024];
  __shared__ double red_v[QR_WARPS];
  __shared__ int red_i[QR_WARPS];
  const int d = a.d;
  const int64_t m = a.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = gridDim.x;
  const int gw = blockIdx.x * QR_WARPS + warp, nw = P * QR_WARPS;  // warps of the grid
  unsigned long long bar_target = 0;
  for (int c = threadIdx.x; c < d; c += blockDim.x) perm[c] = c;
  __syncthreads();
  double first = 0.0;
  int k = 0;
  for (; k < d; ++k) {
    // ---- pivot: largest n1 over positions k..d-1, the lower position on ties (every CTA alike)
    double best = -1.0;
    int bpos = d;
    for (int j = k + threadIdx.x; j < d; j += blockDim.x) {
      const double v = a.n1[perm[j]];
      if (v > best) {
        best = v;
        bpos = j;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, bpos, o);
      if (ov > best || (ov == best && op < bpos)) {
        best = ov;
        bpos = op;
      }
    }
    if (lane == 0) {
      red_v[warp] = best;
      red_i[warp] = bpos;
    }
    __syncthreads();
    best = red_v[0];
    bpos = red_i[0];
    for (int w = 1; w < QR_WARPS; ++w)
      if (red_v[w] > best || (red_v[w] == best && red_i[w] < bpos)) {
        best = red_v[w];
        bpos = red_i[w];
      }
    const double norm = sqrt(best);
    if (k == 0) first = norm;
    if (!(norm > 0.0) || !(norm > a.tol * first)) break;  // the same decision in every CTA
    __syncthreads();  // every thread has read red_v / red_i and perm[j] before they change
    if (threadIdx.x == 0 && bpos != k) {
      const int32_t t = perm[k];
      perm[k] = perm[bpos];
      perm[bpos] = t;
    }
    __syncthreads();
    // ---- the reflector of the pivot column q: v = x - alpha e_k, v^T v = tail + (x_k - alpha)^2
    const int q = perm[k];
    const double* x = a.T + (int64_t)q * m;
    const double xk = x[k];
    const double alpha = xk > 0.0 ? -norm : norm;
    const double vk = xk - alpha;
    const double vtv = a.n2[q] + vk * vk;
    const double tau = vtv > 0.0 ? 2.0 / vtv : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.alpha[k] = alpha;
    // ---- apply to every other active column, a warp per column
    for (int t = gw; t < d - k - 1; t += nw) {
      const int c = perm[k + 1 + t];
      double* y = a.T + (int64_t)c * m;
      double s = lane == 0 ? vk * y[k] : 0.0;
      for (int64_t r = k + 1 + lane; r < m; r += 32) s = fma(x[r], y[r], s);
      s = warp_sum(s);
      const double f = tau * s;
      double s1 = 0.0, s2 = 0.0;
      if (lane == 0) {
        const double yk = y[k] - f * vk;
        a.Ro[(int64_t)k * d + c] = yk;  // R[k][c], c the original column index
      }
      for (int64_t r = k + 1 + lane; r < m; r += 32) {
        const double yr = fma(-f, x[r], y[r]);
        y[r] = yr;
        s1 = fma(yr, yr, s1);
        if (r >= k + 2) s2 = fma(yr, yr, s2);
      }
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
      if (lane == 0) {
        a.n1[c] = s1;
        a.n2[c] = s2;
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.Ro[(int64_t)k * d + q] = alpha;
    if (grid_sync_count(a.bar, bar_target, (unsigned)P, a.err)) return;
  }
  if (blockIdx.x == 0) {
    for (int c = threadIdx.x; c < d; c += blockDim.x) a.perm[c] = perm[c];
    if (threadIdx.x == 0) *a.rank = k;
  }
}

// R[i][j] = sign_i * Ro[i][perm[j]] for j >= i (upper, positive diagonal), 0 below
__global__ void qrp_gather_kernel(const double* __restrict__ Ro, const int32_t* __restrict__ perm,
                                  const double* __restrict__ alpha, const int* __restrict__ rank, int d,
                                  double* __restrict__ R) {
  const int rk = *rank;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)d * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    double v = 0.0;
    if (i < rk && j >= i) v = (alpha[i] < 0.0 ? -1.0 : 1.0) * Ro[(int64_t)i * d + perm[j]];
    R[e] = v;
  }
}

// W[perm[i]][j] = (R^{-1})[i][j]: a warp per column j of R^{-1}, back substitution from row j up,
// the column held in shared memory
__global__ void __launch_bounds__(QR_THREADS) qrp_inverse_kernel(const double* __restrict__ R,
                                                                 const int32_t* __restrict__ perm, int d,
                                                                 double* __restrict__ W) {
  extern __shared__ double col_s[];  // QR_WARPS x d
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * QR_WARPS + warp;
  if (j >= d) return;
  double* xcol = col_s + (size_t)warp * d;
  for (int i = lane; i < d; i += 32) xcol[i] = 0.0;
  __syncwarp();
  for (int i = j; i >= 0; --i) {
    double s = 0.0;
    for (int kk = i + 1 + lane; kk <= j; kk += 32) s = fma(R[(int64_t)i * d + kk], xcol[kk], s);
    s = warp_sum(s);
    if (lane == 0) xcol[i] = ((i == j ? 1.0 : 0.0) - s) / R[(int64_t)i * d + i];
    __syncwarp();
  }
  for (int i = lane; i < d; i += 32) W[(int64_t)perm[i] * d + j] = xcol[i];
}

}  // namespace

extern "C" lsq_status lsq_factor_qr(lsq_ctx* ctx, const double* SA, int64_t m, int64_t d, double tol, double* R,
                                    double* W, int32_t* perm, int64_t* rank_out) {
  if (!ctx || !SA || !R || !W || !perm || d < 1 || d > 1024 || m < d || m > 65536 || !(tol >= 0.0) || !(tol < 1.0))
    return LSQ_ERR_ARG;
  const int di = (int)d;
  const size_t Tb = lsq_align256((size_t)d * m * 8), Rb = lsq_align256((size_t)d * d * 8);
  const size_t need = Tb + Rb + 3 * lsq_align256((size_t)d * 8) + 256 + 256;
  lsq_status st = lsq_ensure_scratch(ctx, need);
  if (st != LSQ_OK) return st;
  Carver cv{reinterpret_cast<char*>(ctx->scratch), 0};
  QrArgs a;
  a.T = cv.take<double>((size_t)d * m);
  a.Ro = cv.take<double>((size_t)d * d);
  a.n1 = cv.take<double>(d);
  a.n2 = cv.take<double>(d);
  a.alpha = cv.take<double>(d);
  a.bar = cv.take<unsigned long long>(4);
  a.err = cv.take<int>(4);
  a.rank = a.err + 1;
  a.m = m;
  a.d = di;
  a.tol = tol;
  a.perm = perm;
  LSQ_CUDA_TRY(cudaMemsetAsync(a.Ro, 0, (size_t)d * d * 8, ctx->stream));
  LSQ_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned long long), ctx->stream));
  LSQ_CUDA_TRY(cudaMemsetAsync(a.err, 0, 4 * sizeof(int), ctx->stream));
  dim3 tg((unsigned)((m + 31) / 32), (unsigned)((d + 31) / 32));
  transpose_sa_kernel<<<tg, dim3(32, 8), 0, ctx->stream>>>(SA, m, di, a.T);
  LSQ_LAUNCH_CHECK();
  qrp_norms_kernel<<<(unsigned)((d * 32 + 255) / 256), 256, 0, ctx->stream>>>(a.T, m, di, a.n1, a.n2);
  LSQ_LAUNCH_CHECK();
  int per_sm = 0;
  LSQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrp_kernel, QR_THREADS, 0));
  // enough warps for every column in the first steps, at most what is co-resident
  const int want = (di + QR_WARPS - 1) / QR_WARPS;
  const int P = std::max(1, std::min(want, std::max(1, per_sm) * ctx->sm_count));
  void* args[] = {&a};
  LSQ_CUDA_TRY(cudaLaunchCooperativeKernel((void*)qrp_kernel, dim3(P), dim3(QR_THREADS), args, 0, ctx->stream));
  lsq_count_launch();
  qrp_gather_kernel<<<std::max(1, std::min(4 * ctx->sm_count, (int)((d * d + 255) / 256))), 256, 0, ctx->stream>>>(
      a.Ro, perm, a.alpha, a.rank, di, R);
  LSQ_LAUNCH_CHECK();
  // the rank (and a timed-out barrier) decide whether W exists
  LSQ_CUDA_TRY(cudaMemcpyAsync(ctx->host_status + 24, a.err, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LSQ_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const int err = ctx->host_status[24], rank = ctx->host_status[25];
  if (rank_out) *rank_out = rank;
  if (err) return (lsq_status)err;
  if (rank < d) return LSQ_ERR_RANK;
  const size_t smem = (size_t)QR_WARPS * d * 8;
  LSQ_CUDA_TRY(cudaFuncSetAttribute(qrp_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  qrp_inverse_kernel<<<(unsigned)((d + QR_WARPS - 1) / QR_WARPS), QR_THREADS, smem, ctx->stream>>>(R, perm, di, W);
  LSQ_LAUNCH_CHECK();
  return LSQ_OK;
}
