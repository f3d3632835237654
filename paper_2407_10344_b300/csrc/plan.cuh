// plan.cuh -- device descriptions of a factor batch (frames, voxelmaps, pairs, work items)
// and the plan object that owns them; shared by the forward and backward kernels.
#pragma once
#include <utility>
#include <vector>

#include "lookup.cuh"

namespace glim_detail {

constexpr int NACC = 28;    // accumulators per point (forward)
constexpr int PSTRIDE = 32; // doubles per partial slot: 28 sums, inliers, 3 spare

struct FrameDev {
  const float4* pts;
  const float2* cov;  // 3 float2 per point
  const float* nrm;   // 3 floats per point or null
  int64_t n;
};

struct MapDev {
  LevelDev lv[GLIM_MAX_LEVELS];
  int32_t levels;
  int32_t pow2;  // 1: inv_r of level l is exactly inv_r of level 0 times 2^-l
  int32_t pad[2];
};

// One dense level as the dense-grid kernel sees it: the record of key (kx, ky, kz) is
// cells[((kx - ox) * ny + (ky - oy)) * nz + (kz - oz)] inside the box, and cells[-1] (an empty
// record) is read for every key outside it.  A level that a map does not have is a box of
// size 0 whose cells[-1] is some map's empty record.
// 32 bytes, read by the kernel as two 16-byte words (offsets checked where it is read).
struct DenseLevelDev {
  const VoxSlot* cells;
  int32_t ox, oy, oz;
  uint32_t nx, ny, nz;
};

struct DenseMapDev {
  DenseLevelDev lv[GLIM_MAX_LEVELS];
  float inv_r[GLIM_MAX_LEVELS];
};

// One hashed level as the per-lane hash kernel sees it (32 bytes, two 16-byte words):
// {cell records, block table} {mask, log2cap, max_probe, pad}.
struct HashLevelDev {
  const VoxSlot* slots;
  const int4* btab;
  uint32_t mask;
  int32_t log2cap;
  int32_t max_probe;
  int32_t pad;
};

struct HashMapDev {
  HashLevelDev lv[GLIM_MAX_LEVELS];
  float inv_r[GLIM_MAX_LEVELS];
};

struct PairDev {
  int32_t src;
  int32_t map;
};

struct Item {
  int32_t pair;
  int32_t start;
};

struct LinArgs {
  const Item* items;
  int32_t nitems;
  int32_t item_base;   // first item (non-persistent launches)
  const PairDev* pairs;
  const FrameDev* frames;
  const MapDev* maps;
  const DenseMapDev* dmaps = nullptr;  // per map, when every target level is a dense grid
  const HashMapDev* hmaps = nullptr;   // per map, when every target level is a hash table
  const PoseF* pose;   // per pair
  int* head;           // work-queue head (persistent)
  double* part;        // nitems x PSTRIDE
  int32_t tile;      // points per item = blockDim.x * ppt
  int32_t ppt;       // rounds per item (points per thread)
  int32_t validate;
  // Read only by the id-recording instantiations (*_ids kernels): the canonical voxel id (or
  // -1) that the kernel resolved for point k of pair p at level l goes to
  // ids[ids_off[p] + k * ids_lv[p] + l], ids_lv[p] being the levels of the pair's map.
  int32_t* ids = nullptr;
  const int64_t* ids_off = nullptr;
  const int32_t* ids_lv = nullptr;
};

struct PairView {
  float R[9], t[3], v[3];
  FrameDev F;
  MapDev M;
};

// Scratch of the gradient pass of a plan (defined with the gradient kernels); freed by
// bwd_scratch_free.
struct BwdScratch;
void bwd_scratch_free(BwdScratch* sc);
// The captured device Gauss-Newton loop of a plan (one frame, a number of iterations) and
// its buffers; freed by gn_graph_free.
struct GnGraph;
void gn_graph_free(GnGraph* g);

using LinKernel = void (*)(const LinArgs);
struct LinKernelInfo {
  LinKernel fn = nullptr;
  size_t smem = 0;  // dynamic shared memory per block
};

}  // namespace glim_detail

using namespace glim_detail;

struct glim_plan {
  glim_ctx* ctx = nullptr;
  int nframes = 0, npairs = 0;
  glim_lin_opts opts{};
  std::vector<glim_frame> frames;
  std::vector<glim_pair> pairs;
  // static device data
  FrameDev* d_frames = nullptr;
  MapDev* d_maps = nullptr;
  PairDev* d_pairs = nullptr;
  int nmaps = 0;
  DenseMapDev* d_dmaps = nullptr;  // set when every level of every target map is a dense grid
  HashMapDev* d_hmaps = nullptr;   // set when every level of every target map is a hash table
  VoxSlot* d_empty_slots = nullptr;  // an all-empty table for the levels a hash map lacks
  // target maps as the plan saw them (address, registry serial, table version), and the map
  // registry's epoch at the last check that found them all unchanged
  struct MapSeen {
    const glim_vmap* m;
    uint64_t serial, version;
  };
  std::vector<MapSeen> map_versions;
  uint64_t maps_checked_epoch = ~0ull;
  int lmax = 1;  // most levels of any target map (kernel template parameter)
  // work list (depends on the tile size)
  Item* d_items = nullptr;
  int32_t* d_item_begin = nullptr;
  int nitems = 0;
  int tile = 0;
  double* d_part = nullptr;
  int* d_head = nullptr;
  int grid = 0;
  LinKernel kernel = nullptr;
  int lane_kernel = 0;  // 0: general kernel; 1: per-lane dense-grid kernel; 2: per-lane hash kernel
  size_t kernel_smem = 0;
  // pose block on the device: PoseF[npairs] then double[npairs * 12], formed by k_pack_poses
  // from the frame poses, which are the only pose data that travel: pinned staging h_fposes ->
  // d_fposes (nframes * 12 doubles)
  size_t in_bytes = 0;
  void* d_in = nullptr;
  double* d_fposes = nullptr;
  double* h_fposes = nullptr;
  bool fposes_on_device = false;  // d_fposes and the pose block hold h_fposes (set after an upload)
  int2* d_pair_frames = nullptr;  // (source frame, target frame) per pair
  // serialized output block: e[npairs], H[npairs*144], b[npairs*12], inliers[npairs]
  size_t out_bytes = 0;
  void* d_out = nullptr;
  void* h_out = nullptr;
  double* d_rec = nullptr;  // per pair its factor record (GLIM_RECORD_DOUBLES doubles), for exchange

  std::vector<cudaEvent_t> ev;       // timing slots: ev[2 s], ev[2 s + 1]
  bool use_graph = true;
  cudaGraphExec_t g_full = nullptr;  // upload + kernels + download
  cudaGraphExec_t g_dev = nullptr;   // kernels only
  GnGraph* gn = nullptr;             // glim_plan_gauss_newton's captured loop
  BwdScratch* bwd = nullptr;         // gradient pass scratch (glim_plan_backward)

  PoseF* in_pose32() const { return reinterpret_cast<PoseF*>(d_in); }
  double* in_pose64() const { return reinterpret_cast<double*>(reinterpret_cast<char*>(d_in) + sizeof(PoseF) * npairs); }
  double* out_e() const { return reinterpret_cast<double*>(d_out); }
  double* out_H() const { return out_e() + npairs; }
  double* out_b() const { return out_H() + size_t(npairs) * 144; }
  long long* out_inl() const { return reinterpret_cast<long long*>(out_b() + size_t(npairs) * 12); }
};


// shared host helpers (linearize.cu)
// Stage the frame poses (host, into the pinned block), then enqueue their upload and the
// pose-packing kernel on the context stream (also inside a graph capture).
void plan_stage_poses(glim_plan* p, const double* poses12);
glim_status plan_enqueue_poses(glim_plan* p);
inline glim_status plan_upload_poses(glim_plan* p, const double* poses12) {
  plan_stage_poses(p, poses12);
  const glim_status st = plan_enqueue_poses(p);
  p->fposes_on_device = st == GLIM_OK;
  return st;
}
// false once a target map was freed or had its tables replaced since the plan was created
bool plan_maps_current(glim_plan* p);
bool map_all_dense(const glim_vmap* m);     // every level a dense grid, resolutions doubling per level
bool map_all_hash(const glim_vmap* m);      // every level a hash table, resolutions doubling per level
void fill_dense_map(const glim_vmap* m, DenseMapDev& d);
void fill_hash_map(const glim_vmap* m, const VoxSlot* empty16, HashMapDev& d);  // empty16: 16 empty slots
// the kernel for an options' accumulation mode and block size, the deepest map's levels and
// lane (0: general, 1: per-lane dense grid, 2: per-lane hash)
LinKernelInfo pick_lin_kernel(int block, int acc, int lmax, int lane);
glim_status plan_configure(glim_plan* p, const glim_lin_opts& o);
glim_status enqueue_reduce_expand(glim_ctx* ctx, const double* part, const int32_t* item_begin,
                                  const double* pose64, int32_t npairs, int32_t fp32_sum, double* e, double* H,
                                  double* b, long long* inl);
