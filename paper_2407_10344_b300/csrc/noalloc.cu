// noalloc.cu -- a linearization entry point that allocates no memory.
//
// Some callers cannot allocate device memory when they linearize: processes whose device
// memory is reserved up front by another allocator (a cudaMalloc may then fail or wait), and
// real-time loops that must not block in the driver (cudaFree synchronizes the device).  For
// them, glim_linearize_factors_noalloc keeps every piece of scratch it needs (descriptors, the
// work list, the queue head and the per-item partial sums) in one statically sized device array
// defined in this file, and writes its results to device arrays the caller passes in.
#include <cstring>

#include "lin_kernel.cuh"

namespace {

constexpr int NA_MAX_FRAMES = 256;
constexpr int NA_MAX_PAIRS = 256;
constexpr int NA_MAX_ITEMS = 16384;  // work items (tiles of block * pts_per_thread points)
constexpr int NA_MAX_DEVICES = 64;

// Everything the host fills in, then the device-only part (queue head, partial sums).
struct NoAllocHostPart {
  FrameDev frames[NA_MAX_FRAMES];
  MapDev maps[NA_MAX_PAIRS];
  DenseMapDev dmaps[NA_MAX_PAIRS];  // per pair, when every target level is a dense grid
  HashMapDev hmaps[NA_MAX_PAIRS];   // per pair, when every target level is a hash table
  PairDev pairs[NA_MAX_PAIRS];
  PoseF pose32[NA_MAX_PAIRS];
  double pose64[NA_MAX_PAIRS * 12];
  Item items[NA_MAX_ITEMS];
  int32_t item_begin[NA_MAX_PAIRS + 1];
};

struct NoAllocScratch {
  NoAllocHostPart host;
  alignas(256) VoxSlot empty16[16];  // all-empty table for the levels a hash map lacks
  alignas(256) int32_t head[64];
  alignas(256) double part[size_t(NA_MAX_ITEMS) * PSTRIDE];
};

// The scratch array: about 4.5 MB on every device that loads this library, held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Host staging of the descriptor block (calls must not overlap, see the header).  It is
// page-locked once per process (cudaHostRegister pins this existing array; nothing is
// allocated), so that its upload is an asynchronous copy that does not wait for the
// stream's earlier work.
static NoAllocHostPart g_stage;
static bool g_stage_pinned = false;
static bool g_stage_register_tried = false;

// Per device, set up on the first call on that device: the device address of
// g_noalloc_scratch, and an event recorded after each upload of g_stage, so that the next
// call rewrites g_stage only once that upload has been read.
static void* g_scratch_addr[NA_MAX_DEVICES] = {nullptr};
static cudaEvent_t g_stage_read[NA_MAX_DEVICES] = {nullptr};
static int g_last_device = -1;  // device of the last upload of g_stage (-1: none yet)

// First call on a device (that device current): look up the scratch array's device address,
// fill the all-empty hash table, wait for that fill, create the upload event.  The address is
// stored last, so that a failure leaves the device to be set up again by the next call.
glim_status noalloc_setup(glim_ctx* ctx) {
  void* ptr = nullptr;
  GLIM_CUDA(ctx, cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
  NoAllocScratch* d0 = static_cast<NoAllocScratch*>(ptr);
  GLIM_CUDA(ctx, cudaMemsetAsync(d0->empty16, 0x80, sizeof(d0->empty16), ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (!g_stage_read[ctx->device])
    GLIM_CUDA(ctx, cudaEventCreateWithFlags(&g_stage_read[ctx->device], cudaEventDisableTiming));
  if (!g_stage_register_tried) {
    g_stage_register_tried = true;
    g_stage_pinned = cudaHostRegister(&g_stage, sizeof(g_stage), cudaHostRegisterDefault) == cudaSuccess;
    if (!g_stage_pinned) cudaGetLastError();  // the uploads then stay correct, only synchronous
  }
  g_scratch_addr[ctx->device] = ptr;
  return GLIM_OK;
}

}  // namespace

extern "C" glim_status glim_linearize_factors_noalloc(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                                      const glim_pair* pairs, int32_t npairs, const double* poses12,
                                                      const glim_lin_opts* opts, double* e_out, double* H_out,
                                                      double* b_out, int64_t* inliers_out) {
  if (!ctx) return GLIM_EINVAL;
  if (nframes < 0 || npairs < 0 || (nframes > 0 && (!frames || !poses12)) || (npairs > 0 && !pairs))
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: bad batch arguments");
  if (nframes > NA_MAX_FRAMES || npairs > NA_MAX_PAIRS)
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: %d frames / %d pairs exceed the limits (%d frames, %d pairs)",
                     nframes, npairs, NA_MAX_FRAMES, NA_MAX_PAIRS);
  if (npairs > 0 && (!e_out || !H_out || !b_out))
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: null output");
  if (ctx->device < 0 || ctx->device >= NA_MAX_DEVICES)
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: device %d out of range", ctx->device);
  glim_lin_opts o{};
  if (opts) o = *opts;
  if (o.block == 0) o.block = 256;
  if (o.pts_per_thread == 0) o.pts_per_thread = 16;
  if (!(o.block == 128 || o.block == 256) || o.pts_per_thread < 1 || o.pts_per_thread > 256 ||
      o.accum_mode < 0 || o.accum_mode > 2)
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: invalid options");
  for (int f = 0; f < nframes; ++f) {
    const glim_frame& F = frames[f];
    if (F.n < 0 || F.n > 0x7FFFFFFFll || (F.n > 0 && (!F.pts4 || !F.cov6)) ||
        (reinterpret_cast<uintptr_t>(F.pts4) & 15) || (reinterpret_cast<uintptr_t>(F.cov6) & 7))
      return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: frame %d is invalid", f);
  }
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  // The descriptors travel through g_stage, which every call rewrites: a captured call would
  // replay whatever the latest call left there, so capture is refused.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GLIM_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: the context's stream is capturing a graph");
  // set-up, once per device, with that device current
  if (!g_scratch_addr[ctx->device]) {
    const glim_status st = noalloc_setup(ctx);
    if (st != GLIM_OK) return st;
  }
  NoAllocScratch* dev = static_cast<NoAllocScratch*>(g_scratch_addr[ctx->device]);
  // the previous upload of g_stage (on whichever device) must have been read before it is
  // rewritten; this waits for no work enqueued after that upload
  if (g_last_device >= 0) GLIM_CUDA(ctx, cudaEventSynchronize(g_stage_read[g_last_device]));

  // descriptors, poses and work list, staged on the host
  NoAllocHostPart& h = g_stage;
  int lmax = 1;
  for (int f = 0; f < nframes; ++f) {
    h.frames[f].pts = reinterpret_cast<const float4*>(frames[f].pts4);
    h.frames[f].cov = reinterpret_cast<const float2*>(frames[f].cov6);
    h.frames[f].nrm = frames[f].normal3;
    h.frames[f].n = frames[f].n;
  }
  const int tile = o.block * o.pts_per_thread;
  int nitems = 0;
  bool all_dense = npairs > 0, all_hash = npairs > 0;
  for (int q = 0; q < npairs; ++q)
    if (pairs[q].tgt) {
      all_dense = all_dense && map_all_dense(pairs[q].tgt);
      all_hash = all_hash && map_all_hash(pairs[q].tgt);
    }
  for (int f = 0; f < nframes; ++f)
    if (frames[f].n > 0x7FFFFFFFll - (1 << 17)) all_dense = all_hash = false;
  if ((o.kernel == 2 && !all_dense) || (o.kernel == 3 && !all_hash) || o.kernel < 0 || o.kernel > 3)
    return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: the requested kernel does not fit the maps' layout");
  const int lane = o.kernel == 1 ? 0 : (all_dense ? 1 : (all_hash ? 2 : 0));
  for (int q = 0; q < npairs; ++q) {
    const glim_pair& P = pairs[q];
    if (P.src_frame < 0 || P.src_frame >= nframes || P.tgt_frame < 0 || P.tgt_frame >= nframes || !P.tgt ||
        P.tgt->device != ctx->device)
      return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: pair %d is invalid", q);
    std::memset(&h.maps[q], 0, sizeof(MapDev));
    h.maps[q].levels = P.tgt->levels;
    for (int l = 0; l < P.tgt->levels; ++l) h.maps[q].lv[l] = P.tgt->dev(l);
    lmax = P.tgt->levels > lmax ? P.tgt->levels : lmax;
    if (lane == 1) fill_dense_map(P.tgt, h.dmaps[q]);
    if (lane == 2) fill_hash_map(P.tgt, dev->empty16, h.hmaps[q]);
    h.pairs[q].src = P.src_frame;
    h.pairs[q].map = q;
    const RelPose T = relative_pose(poses12 + 12 * P.src_frame, poses12 + 12 * P.tgt_frame);
    h.pose32[q] = pose_to_f32(T);
    std::memcpy(h.pose64 + 12 * q, T.R, 9 * sizeof(double));
    std::memcpy(h.pose64 + 12 * q + 9, T.t, 3 * sizeof(double));
    h.item_begin[q] = nitems;
    const int64_t n = frames[P.src_frame].n;
    for (int64_t s = 0; s < n; s += tile) {
      if (nitems >= NA_MAX_ITEMS)
        return set_error(ctx, GLIM_EINVAL,
                         "linearize_noalloc: more than %d work items of %d points; raise pts_per_thread or split the batch",
                         NA_MAX_ITEMS, tile);
      h.items[nitems++] = Item{q, int32_t(s)};
    }
  }
  h.item_begin[npairs] = nitems;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&dev->host, &h, sizeof(NoAllocHostPart), cudaMemcpyHostToDevice, ctx->stream));
  GLIM_CUDA(ctx, cudaEventRecord(g_stage_read[ctx->device], ctx->stream));
  g_last_device = ctx->device;

  if (nitems > 0) {
    const LinKernelInfo ki = pick_lin_kernel(o.block, o.accum_mode, lmax, lane);
    if (!ki.fn) return set_error(ctx, GLIM_EINVAL, "linearize_noalloc: no kernel for these options");
    GLIM_CUDA(ctx, cudaFuncSetAttribute(reinterpret_cast<const void*>(ki.fn),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, int(ki.smem)));
    int per_sm = 1;
    GLIM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, o.block, ki.smem));
    const int grid = std::max(1, std::min(std::max(per_sm, 1) * ctx->num_sms, nitems));
    // the queue head must start at zero on every call
    GLIM_CUDA(ctx, cudaMemsetAsync(dev->head, 0, sizeof(int32_t), ctx->stream));
    LinArgs a;
    a.items = dev->host.items;
    a.nitems = nitems;
    a.item_base = 0;
    a.pairs = dev->host.pairs;
    a.frames = dev->host.frames;
    a.maps = dev->host.maps;
    a.dmaps = lane == 1 ? dev->host.dmaps : nullptr;
    a.hmaps = lane == 2 ? dev->host.hmaps : nullptr;
    a.pose = dev->host.pose32;
    a.head = dev->head;
    a.part = dev->part;
    a.tile = tile;
    a.ppt = o.pts_per_thread;
    a.validate = o.validate_surface;
    ki.fn<<<grid, o.block, ki.smem, ctx->stream>>>(a);
    GLIM_LAUNCHED(ctx);
  }
  return enqueue_reduce_expand(ctx, dev->part, dev->host.item_begin, dev->host.pose64, npairs,
                               o.accum_mode == GLIM_ACC_FP32 ? 1 : 0, e_out, H_out, b_out,
                               reinterpret_cast<long long*>(inliers_out));
}
