// measure.cu -- FP32 and FP64 FMA throughput of the device.  The FP32 figure is the
// denominator of the FP32 roofline of the linearization kernel (whose arithmetic is FP32
// multiply-adds on the CUDA cores, not a dense contraction); the FP64 figure is what an
// all-FP64 kernel would be bounded by, recorded to show why only the cross-block sums are
// FP64.  Every thread runs eight independent register-resident FMA chains; with eight
// 256-thread blocks per SM there are enough independent FMAs in flight to keep every pipe
// busy, so the time measures issue throughput, not latency.
#include "common.cuh"

namespace {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_UNROLL = 16;

__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }
__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ sink, int iters, T a, T b) {
  T x[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) x[c] = T(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < FMA_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fma_rn(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
  if (s == T(-1)) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

template <typename T>
glim_status fma_peak(glim_ctx* ctx, int32_t iters, double* tflops_out, const char* what) {
  if (!ctx || !tflops_out || iters < 1) return GLIM_EINVAL;
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  const int blocks = 8 * ctx->num_sms, threads = 256;
  DevBuf<T> sink;
  GLIM_CUDA(ctx, sink.alloc(blocks, ctx->stream));
  cudaEvent_t e0, e1;
  GLIM_CUDA(ctx, cudaEventCreate(&e0));
  GLIM_CUDA(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  glim_status st = GLIM_OK;
  for (int rep = 0; rep < 4 && st == GLIM_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, ctx->stream);
    k_fma_chains<T><<<blocks, threads, 0, ctx->stream>>>(sink.p, iters, T(0.99999), T(1e-6));
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
      st = cuda_check(ctx, le, what);
      break;
    }
    ctx->launches++;
    cudaEventRecord(e1, ctx->stream);
    const cudaError_t se = cudaEventSynchronize(e1);
    if (se != cudaSuccess) {
      st = cuda_check(ctx, se, what);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GLIM_OK) return st;
  const double fmas = double(blocks) * threads * double(iters) * FMA_UNROLL * FMA_CHAINS;
  *tflops_out = 2.0 * fmas / (double(best) * 1e-3) / 1e12;
  ctx->err.clear();
  return GLIM_OK;
}

}  // namespace

extern "C" glim_status glim_fp32_fma_peak(glim_ctx* ctx, int32_t iters, double* tflops_out) {
  return fma_peak<float>(ctx, iters, tflops_out, "fp32 fma peak");
}

extern "C" glim_status glim_fp64_fma_peak(glim_ctx* ctx, int32_t iters, double* tflops_out) {
  return fma_peak<double>(ctx, iters, tflops_out, "fp64 fma peak");
}
