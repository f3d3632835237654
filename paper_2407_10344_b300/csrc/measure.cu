// measure.cu -- FP32 FMA throughput of the device, the denominator of the FP32 roofline of the
// linearization kernel (whose arithmetic is FP32 multiply-adds on the CUDA cores, not a dense
// contraction).  Every thread runs eight independent register-resident FMA chains; with
// eight 256-thread blocks per SM there are enough independent FMAs in flight to keep every
// FP32 pipe busy, so the time measures issue throughput, not latency.
#include "common.cuh"

namespace {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_UNROLL = 16;

__global__ void __launch_bounds__(256) k_fma_chains(float* __restrict__ sink, int iters, float a, float b) {
  float x[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) x[c] = float(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < FMA_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < FMA_CHAINS; ++c) x[c] = __fmaf_rn(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" glim_status glim_fp32_fma_peak(glim_ctx* ctx, int32_t iters, double* tflops_out) {
  if (!ctx || !tflops_out || iters < 1) return GLIM_EINVAL;
  GLIM_CUDA(ctx, cudaSetDevice(ctx->device));
  const int blocks = 8 * ctx->num_sms, threads = 256;
  DevBuf<float> sink;
  GLIM_CUDA(ctx, sink.alloc(blocks, ctx->stream));
  cudaEvent_t e0, e1;
  GLIM_CUDA(ctx, cudaEventCreate(&e0));
  GLIM_CUDA(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  glim_status st = GLIM_OK;
  for (int rep = 0; rep < 4 && st == GLIM_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, ctx->stream);
    k_fma_chains<<<blocks, threads, 0, ctx->stream>>>(sink.p, iters, 0.99999f, 1e-6f);
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
      st = cuda_check(ctx, le, "fma peak launch");
      break;
    }
    ctx->launches++;
    cudaEventRecord(e1, ctx->stream);
    const cudaError_t se = cudaEventSynchronize(e1);
    if (se != cudaSuccess) {
      st = cuda_check(ctx, se, "fma peak sync");
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
