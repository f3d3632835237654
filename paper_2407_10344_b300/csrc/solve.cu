// solve.cu -- Gauss-Newton step of a quadratic factor, xi = -H^-1 b, by Cholesky in FP64.
// One thread per system; the systems are at most 12 x 12.
#include "common.cuh"

namespace {

constexpr int MAXD = 12;

__global__ void k_cholesky_solve(const double* __restrict__ H, int ldh, int64_t stride_H,
                                 const double* __restrict__ b, int64_t stride_b, int dim, int64_t count,
                                 double* __restrict__ xi, int32_t* __restrict__ status, int* __restrict__ n_bad) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const double* A = H + s * stride_H;
  const double* r = b + s * stride_b;
  double L[MAXD][MAXD];
  bool ok = true;
  for (int j = 0; j < dim && ok; ++j) {
    double d = A[j * ldh + j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !isfinite(d)) {
      ok = false;
      break;
    }
    const double ljj = sqrt(d);
    L[j][j] = ljj;
    for (int i = j + 1; i < dim; ++i) {
      double v = A[i * ldh + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / ljj;
    }
  }
  double* x = xi + s * dim;
  if (!ok) {
    for (int i = 0; i < dim; ++i) x[i] = 0.0;
    if (status) status[s] = GLIM_ENOTPD;
    atomicAdd(n_bad, 1);
    return;
  }
  double y[MAXD];
  for (int i = 0; i < dim; ++i) {  // L y = -b
    double v = -r[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
  for (int i = dim - 1; i >= 0; --i) {  // L^T x = y
    double v = y[i];
    for (int k = i + 1; k < dim; ++k) v -= L[k][i] * x[k];
    x[i] = v / L[i][i];
  }
  if (status) status[s] = GLIM_OK;
}

}  // namespace

extern "C" glim_status glim_gn_solve(glim_ctx* ctx, const double* H, int32_t ldh, int64_t stride_H, const double* b,
                                     int64_t stride_b, int32_t dim, int64_t count, double* xi_out,
                                     int32_t* status_out) {
  GLIM_RANGE("glim_gn_solve");
  if (!ctx) return GLIM_EINVAL;
  if (dim < 1 || dim > MAXD || count < 0 || ldh < dim || (count > 0 && (!H || !b || !xi_out)))
    return set_error(ctx, GLIM_EINVAL, "gn_solve: bad arguments (dim=%d ldh=%d)", dim, ldh);
  if (count == 0) return GLIM_OK;
  DevBuf<int> bad;
  GLIM_CUDA(ctx, bad.alloc(1, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(bad.p, 0, sizeof(int), ctx->stream));
  k_cholesky_solve<<<ceil_div_i(count, 64), 64, 0, ctx->stream>>>(H, ldh, stride_H, b, stride_b, dim, count, xi_out,
                                                                  status_out, bad.p);
  GLIM_LAUNCHED(ctx);
  int nb = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&nb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (nb > 0) return set_error(ctx, GLIM_ENOTPD, "gn_solve: %d system(s) not positive definite", nb);
  ctx->err.clear();
  return GLIM_OK;
}
