// api.cu -- context lifetime, error reporting and pose helpers of the C ABI.
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <cmath>
#include <cstring>

#include "common.cuh"

// Allocation-failure injection for tests: the countdown is the number of allocations that
// still succeed before one fails; negative disables it.  Process-wide, shared by all threads.
static std::atomic<long long> g_fail_countdown{-1};

bool alloc_should_fail() {
  long long c = g_fail_countdown.load(std::memory_order_relaxed);
  while (c >= 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1, std::memory_order_relaxed)) return c == 0;
  }
  return false;
}

extern "C" void glim_debug_fail_allocation(int64_t n) { g_fail_countdown.store(n < 0 ? -1 : n); }

glim_status set_error(glim_ctx* ctx, glim_status st, const char* fmt, ...) {
  if (!ctx) return st;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  ctx->err = buf;
  return st;
}

glim_status cuda_check(glim_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(ctx, GLIM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  }
  return set_error(ctx, GLIM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

glim_status take_device_status(glim_ctx* ctx, const char* where) {
  unsigned int s = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&s, ctx->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (s & GLIM_DS_NONFINITE) return set_error(ctx, GLIM_EINVAL, "%s: non-finite input", where);
  if (s & GLIM_DS_RANGE) return set_error(ctx, GLIM_ERANGE, "%s: voxel key outside [-2^20, 2^20)", where);
  if (s & GLIM_DS_HASHFULL) return set_error(ctx, GLIM_EHASHFULL, "%s: hash table full", where);
  if (s & GLIM_DS_TIMEOUT) return set_error(ctx, GLIM_ETIMEOUT, "%s: bounded wait gave up", where);
  return GLIM_OK;
}

// T_rel = T_t^-1 T_s:  R = R_t^T R_s,  t = R_t^T (t_s - t_t), in FP64.
RelPose relative_pose(const double* s, const double* t) {
  RelPose r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v += t[4 * k + i] * s[4 * k + j];
      r.R[3 * i + j] = v;
    }
  const double dt[3] = {s[3] - t[3], s[7] - t[7], s[11] - t[11]};
  for (int i = 0; i < 3; ++i) r.t[i] = t[i] * dt[0] + t[4 + i] * dt[1] + t[8 + i] * dt[2];
  return r;
}

// FP32 rounding of T_rel and the target viewpoint in the source frame, v = -R^T t (FP64,
// then rounded).
PoseF pose_to_f32(const RelPose& T) {
  PoseF p;
  for (int i = 0; i < 9; ++i) p.R[i] = float(T.R[i]);
  for (int i = 0; i < 3; ++i) {
    p.t[i] = float(T.t[i]);
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v += T.R[3 * k + i] * T.t[k];
    p.v[i] = float(-v);
  }
  p.pad = 0.f;
  return p;
}

namespace {
std::mutex g_vmap_mu;
std::unordered_map<const glim_vmap*, uint64_t> g_vmaps;  // live map -> serial
uint64_t g_vmap_serial = 0;
std::atomic<uint64_t> g_vmap_epoch{0};
}  // namespace

void vmap_register(glim_vmap* vm) {
  std::lock_guard<std::mutex> lk(g_vmap_mu);
  vm->serial = ++g_vmap_serial;
  g_vmaps[vm] = vm->serial;
}

void vmap_unregister(glim_vmap* vm) {
  {
    std::lock_guard<std::mutex> lk(g_vmap_mu);
    g_vmaps.erase(vm);
  }
  vmap_bump_epoch();
}

bool vmap_alive(const glim_vmap* vm, uint64_t serial) {
  std::lock_guard<std::mutex> lk(g_vmap_mu);
  const auto it = g_vmaps.find(vm);
  return it != g_vmaps.end() && it->second == serial;
}

uint64_t vmap_epoch() { return g_vmap_epoch.load(std::memory_order_acquire); }
void vmap_bump_epoch() { g_vmap_epoch.fetch_add(1, std::memory_order_acq_rel); }

extern "C" glim_status glim_create(glim_ctx** out, int device, void* cuda_stream) {
  if (!out) return GLIM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GLIM_EINVAL;
  }
  DeviceGuard device_guard;
  if (device_guard.set(device) != cudaSuccess) return GLIM_ECUDA;
  glim_ctx* ctx = new glim_ctx;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return GLIM_ECUDA;
    }
    ctx->own_stream = true;
  }
  if (dmalloc(&ctx->d_status, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(unsigned int)) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return GLIM_ENOMEM;
  }
  *out = ctx;
  return GLIM_OK;
}

extern "C" void glim_destroy(glim_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard device_guard;
  device_guard.set(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_status);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

extern "C" const char* glim_last_error(const glim_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int32_t glim_num_sms(const glim_ctx* ctx) { return ctx ? ctx->num_sms : 0; }

extern "C" int64_t glim_kernel_launches(const glim_ctx* ctx) { return ctx ? ctx->launches : 0; }
