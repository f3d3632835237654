// graph.cu -- Gauss-Newton / Levenberg-Marquardt step of a small factor graph on the device:
// the per-pair quadratic factors (H 12 x 12 over [xi_s; xi_t], b 12) of a batch are summed
// into the global system of all frame poses, one frame is held fixed (the gauge of the
// relative-pose factors), the remaining system is damped and solved by a dense Cholesky in
// FP64.  This is the step of the all-to-all submap optimisation of local mapping (Sec. V-A),
// whose linearization is the batched kernel of this library.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int MAX_FRAMES = 128;

// H_glob (6n x 6n, row-major) and b_glob (6n): entry by entry, summing the pairs in order.
__global__ void k_assemble(const int32_t* __restrict__ pf, int npairs, int n, const double* __restrict__ H,
                           const double* __restrict__ b, double* __restrict__ Hg, double* __restrict__ bg) {
  const int N = 6 * n;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < int64_t(N) * N) {
    const int r = int(e / N), c = int(e % N);
    const int fr = r / 6, a = r % 6, fc = c / 6, bb = c % 6;
    double s = 0.0;
    for (int p = 0; p < npairs; ++p) {
      const int sp = pf[2 * p], tp = pf[2 * p + 1];
      const int ro = fr == sp ? 0 : (fr == tp ? 6 : -1);
      const int co = fc == sp ? 0 : (fc == tp ? 6 : -1);
      if (ro >= 0 && co >= 0) s += H[int64_t(p) * 144 + (ro + a) * 12 + (co + bb)];
    }
    Hg[e] = s;
  }
  if (e < N) {
    const int fr = int(e) / 6, a = int(e) % 6;
    double s = 0.0;
    for (int p = 0; p < npairs; ++p) {
      const int sp = pf[2 * p], tp = pf[2 * p + 1];
      const int ro = fr == sp ? 0 : (fr == tp ? 6 : -1);
      if (ro >= 0) s += b[int64_t(p) * 12 + ro + a];
    }
    bg[e] = s;
  }
}

// Reduced, damped system A = H_ff + lambda diag(H_ff), rhs = -b_f (variables of the free
// frames in frame order), then a right-looking Cholesky and the two triangular solves, all
// in one block.  *bad = 1 if A is not positive definite.
__global__ void __launch_bounds__(1024) k_reduce_solve(const double* __restrict__ Hg, const double* __restrict__ bg,
                                                       int n, int fixed, double lambda, double* __restrict__ A,
                                                       double* __restrict__ y, double* __restrict__ xi,
                                                       int* __restrict__ bad) {
  const int Nf = 6 * n;
  const int N = fixed >= 0 ? Nf - 6 : Nf;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto gv = [&](int i) { return (fixed >= 0 && i >= 6 * fixed) ? i + 6 : i; };  // reduced -> full index
  for (int64_t e = tid; e < int64_t(N) * N; e += nt) {
    const int i = int(e / N), j = int(e % N);
    double v = Hg[int64_t(gv(i)) * Nf + gv(j)];
    if (i == j) v += lambda * v;
    A[e] = v;
  }
  for (int i = tid; i < N; i += nt) y[i] = -bg[gv(i)];
  __shared__ double s_piv;
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      const double d = A[int64_t(k) * N + k];
      if (!(d > 0.0) || !isfinite(d)) s_bad = 1;
      s_piv = sqrt(fmax(d, 0.0));
      A[int64_t(k) * N + k] = s_piv;
    }
    __syncthreads();
    if (s_bad) break;
    for (int i = k + 1 + tid; i < N; i += nt) A[int64_t(i) * N + k] /= s_piv;
    __syncthreads();
    const int m = N - k - 1;
    for (int64_t e = tid; e < int64_t(m) * m; e += nt) {
      const int i = k + 1 + int(e / m), j = k + 1 + int(e % m);
      if (j <= i) A[int64_t(i) * N + j] -= A[int64_t(i) * N + k] * A[int64_t(j) * N + k];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) *bad = 1;
    for (int i = tid; i < Nf; i += nt) xi[i] = 0.0;
    return;
  }
  // L z = y (column sweep), then L^T x = z
  for (int k = 0; k < N; ++k) {
    if (tid == 0) y[k] /= A[int64_t(k) * N + k];
    __syncthreads();
    for (int i = k + 1 + tid; i < N; i += nt) y[i] -= A[int64_t(i) * N + k] * y[k];
    __syncthreads();
  }
  for (int k = N - 1; k >= 0; --k) {
    if (tid == 0) y[k] /= A[int64_t(k) * N + k];
    __syncthreads();
    for (int i = tid; i < k; i += nt) y[i] -= A[int64_t(k) * N + i] * y[k];
    __syncthreads();
  }
  for (int i = tid; i < Nf; i += nt) {
    const bool fx = fixed >= 0 && i >= 6 * fixed && i < 6 * fixed + 6;
    xi[i] = fx ? 0.0 : y[(fixed >= 0 && i >= 6 * fixed + 6) ? i - 6 : i];
  }
}

}  // namespace

extern "C" glim_status glim_graph_step(glim_ctx* ctx, const int32_t* pair_frames, int32_t npairs, int32_t nframes,
                                       const double* H, const double* b, int32_t fixed_frame, double lambda,
                                       double* xi_out, double* H_out, double* b_out) {
  GLIM_RANGE("glim_graph_step");
  if (!ctx) return GLIM_EINVAL;
  if (nframes < 1 || nframes > MAX_FRAMES || npairs < 0 || (npairs > 0 && (!pair_frames || !H || !b)) || !xi_out ||
      fixed_frame < -1 || fixed_frame >= nframes || !(lambda >= 0.0) || !std::isfinite(lambda))
    return set_error(ctx, GLIM_EINVAL, "graph_step: bad arguments (nframes=%d, at most %d)", nframes, MAX_FRAMES);
  std::vector<int32_t> pf(pair_frames, pair_frames + 2 * npairs);
  for (int p = 0; p < npairs; ++p)
    if (pf[2 * p] < 0 || pf[2 * p] >= nframes || pf[2 * p + 1] < 0 || pf[2 * p + 1] >= nframes ||
        pf[2 * p] == pf[2 * p + 1])
      return set_error(ctx, GLIM_EINVAL, "graph_step: pair %d has bad frames", p);
  const int N = 6 * nframes;
  DevBuf<int32_t> dpf;
  DevBuf<double> Hg, bg, A, y;
  GLIM_CUDA(ctx, dpf.alloc(std::max<int64_t>(2 * npairs, 1), ctx->stream));
  GLIM_CUDA(ctx, Hg.alloc(size_t(N) * N, ctx->stream));
  GLIM_CUDA(ctx, bg.alloc(N, ctx->stream));
  GLIM_CUDA(ctx, A.alloc(size_t(N) * N, ctx->stream));
  GLIM_CUDA(ctx, y.alloc(N, ctx->stream));
  DevBuf<int> bad;
  GLIM_CUDA(ctx, bad.alloc(1, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(bad.p, 0, sizeof(int), ctx->stream));
  if (npairs > 0)
    GLIM_CUDA(ctx, cudaMemcpyAsync(dpf.p, pf.data(), 2 * npairs * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  k_assemble<<<ceil_div_i(int64_t(N) * N, 256), 256, 0, ctx->stream>>>(dpf.p, npairs, nframes, H, b, Hg.p, bg.p);
  GLIM_LAUNCHED(ctx);
  k_reduce_solve<<<1, 1024, 0, ctx->stream>>>(Hg.p, bg.p, nframes, fixed_frame, lambda, A.p, y.p, xi_out, bad.p);
  GLIM_LAUNCHED(ctx);
  if (H_out)
    GLIM_CUDA(ctx, cudaMemcpyAsync(H_out, Hg.p, size_t(N) * N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (b_out) GLIM_CUDA(ctx, cudaMemcpyAsync(b_out, bg.p, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  int nb = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&nb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (nb) return set_error(ctx, GLIM_ENOTPD, "graph_step: the reduced system is not positive definite");
  ctx->err.clear();
  return GLIM_OK;
}
