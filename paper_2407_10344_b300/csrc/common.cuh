// common.cuh -- shared internals of the linearization library (context, status words,
// voxel keys, hash slots).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/glim_lin.h"

// An NVTX range for the lifetime of a scope, named after the entry point: a profiler
// (ncu --nvtx, Nsight Systems) attributes the call's launches to it; with no tool attached
// a push and a pop cost a few nanoseconds.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};
#define GLIM_RANGE(name) NvtxScope glim_nvtx_scope_(name)

// Makes a device current for the lifetime of a scope and restores the caller's current
// device afterwards, so that an entry point leaves the calling thread's device as it found it.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() = default;
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  cudaError_t set(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      cur = -1;
    }
    if (cur == dev) return cudaSuccess;
    const cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) prev = cur;
    return e;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// ------------------------------------------------------------------ context
struct glim_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int64_t launches = 0;
  unsigned int* d_status = nullptr;  // device status word (bit flags below)
};

// device status bits (set with atomicOr; read by the host after a synchronize)
#define GLIM_DS_RANGE 1u      // a build key was outside [-2^20, 2^20)
#define GLIM_DS_NONFINITE 2u  // a non-finite input value
#define GLIM_DS_HASHFULL 4u   // the hash insert exhausted its probe bound
#define GLIM_DS_TIMEOUT 8u    // a bounded wait gave up

glim_status set_error(glim_ctx* ctx, glim_status st, const char* fmt, ...);
glim_status cuda_check(glim_ctx* ctx, cudaError_t e, const char* what);
#define GLIM_CUDA(ctx, call)                                   \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return cuda_check((ctx), _e, #call); \
  } while (0)
// after a kernel launch: count it and check the launch
#define GLIM_LAUNCHED(ctx)                                                   \
  do {                                                                       \
    (ctx)->launches++;                                                       \
    cudaError_t _e = cudaGetLastError();                                     \
    if (_e != cudaSuccess) return cuda_check((ctx), _e, "kernel launch");    \
  } while (0)

// read and clear the device status word; map to a status code
glim_status take_device_status(glim_ctx* ctx, const char* where);

// ------------------------------------------------------------------ allocations
// Every device and pinned host allocation of the library goes through these wrappers, so
// that a test can make one chosen allocation fail (glim_debug_fail_allocation) and reach each
// error path on the host; a failed wrapper leaves *p null and allocates nothing.
bool alloc_should_fail();
template <class T>
inline cudaError_t dmalloc(T** p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t dmalloc_async(T** p, size_t bytes, cudaStream_t s) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
}
template <class T>
inline cudaError_t hmalloc(T** p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}

// stream-ordered temporary device buffer
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  cudaError_t alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count == 0) return cudaSuccess;
    return dmalloc_async(&p, count * sizeof(T), stream);
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
};

// ------------------------------------------------------------------ voxel keys
// A voxel key (kx, ky, kz) with every component in [-2^20, 2^20) packs into 63 bits as
// ((kx + 2^20) << 42) | ((ky + 2^20) << 21) | (kz + 2^20); unsigned order of packed keys
// equals lexicographic (x, y, z) order of the keys.
#define GLIM_KEY_BIAS (1 << 20)
#define GLIM_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

__host__ __device__ inline unsigned long long pack_key(int kx, int ky, int kz) {
  return ((unsigned long long)(kx + GLIM_KEY_BIAS) << 42) |
         ((unsigned long long)(ky + GLIM_KEY_BIAS) << 21) | (unsigned long long)(kz + GLIM_KEY_BIAS);
}
__host__ __device__ inline int unpack_x(unsigned long long k) { return int((k >> 42) & 0x1FFFFF) - GLIM_KEY_BIAS; }
__host__ __device__ inline int unpack_y(unsigned long long k) { return int((k >> 21) & 0x1FFFFF) - GLIM_KEY_BIAS; }
__host__ __device__ inline int unpack_z(unsigned long long k) { return int(k & 0x1FFFFF) - GLIM_KEY_BIAS; }

// Fibonacci hashing of a packed key into a power-of-two table (grid cells of the kNN search).
__host__ __device__ inline uint32_t hash_slot(unsigned long long key, int log2cap) {
  return uint32_t((key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap));
}

// Voxel-table hash of an integer block key: a linear hash, the top log2cap bits of
// kx a + ky b + kz c (mod 2^32), with odd multipliers (each the Fibonacci multiplier 2654435761
// times a 32-bit mixing constant).  Blocks next to each other land in slots a fixed stride
// apart, so the handful of blocks that the lanes of a warp touch rarely share or crowd a slot:
// on the urban submaps the share of hits not found in their home slot fell from 8-21 % with
// the XOR-of-products spatial hash of Teschner et al. (2003) to under 1 % at load <= 1/16.
// A lattice hash can still line up with a particular key set (longer probe chains, bounded by
// the table's longest probe sequence); that costs time, never correctness.
__host__ __device__ inline uint32_t hash3(int kx, int ky, int kz, int log2cap) {
  const uint32_t h = uint32_t(kx) * 0xFFE6CC61u + uint32_t(ky) * 0xFC4A3B47u + uint32_t(kz) * 0x27004D2Du;
  return h >> (32 - log2cap);
}

// Coordinate value marking an empty slot (every byte 0x80, outside [-2^20, 2^20)).
#define GLIM_EMPTY_COORD int(0x80808080)
#define GLIM_EMPTY_XY 0x8080808080808080ull

// floor(c * inv_r) as an int in [-2^20, 2^20), or false.  One FP32 multiply, rounded to
// nearest (explicit so that the compiler cannot fuse it with anything).
__device__ __forceinline__ bool voxel_coord(float c, float inv_r, int& k) {
  float f = floorf(__fmul_rn(c, inv_r));
  if (!(f >= -1048576.0f && f < 1048576.0f)) return false;  // also rejects NaN
  k = __float2int_rz(f);
  return true;
}

// ------------------------------------------------------------------ voxel record (48 bytes)
// The record of one voxel cell: w0 = {canonical id (int bits), c22, kx (int bits), c22},
// w1 = {mean x, mean y, mean z, c00}, w2 = {c01, c02, c11, c12}.  An empty cell has every byte
// 0x80, so its id reads negative.  c22 sits next to the id (one 8-byte read gives both) and
// again at w0.w.
struct __align__(16) VoxSlot {
  float4 w0, w1, w2;
};

// Voxel blocks of the hashed layout: 2 x 2 x 2 cells.  Block key (kx >> 1, ky >> 1, kz >> 1)
// (arithmetic shifts, i.e. floor division), cell kx & 1, ky & 1, kz & 1 inside it.
#define GLIM_BLOCK_SHIFT 1
#define GLIM_BLOCK_CELLS 8

__host__ __device__ inline int block_local(int kx, int ky, int kz) {
  return ((kx & 1) << 2) | ((ky & 1) << 1) | (kz & 1);
}

// One resolution level of a voxelmap as the kernels see it: the voxel records live in cells
// (empty cells all 0x80, and one empty record just before cell 0 that a miss reads), either
//   dense: a grid over the bounding box of the occupied keys, cell ((kx - ox) ny + ky - oy)
//          nz + kz - oz; or
//   hashed: voxel blocks (spatial hashing of voxel blocks, as in voxel hashing): an
//          open-addressing table (linear probing) of entries {bx, by, bz, block} maps a block
//          key to its block, whose 8 cells hold the records, cell block * 8 + local.
struct LevelDev {
  const VoxSlot* slots;    // cell records: grid cells (dense) or block cells (hashed)
  const int4* btab;        // hashed: block table {bx, by, bz, block index}, empty = 0x80 bytes
  const int32_t* unused;   // null (keeps the descriptor's layout)
  uint32_t mask;           // hashed: block-table capacity - 1
  int32_t log2cap;
  int32_t max_probe;       // hashed: longest probe sequence of any block in the table
  float inv_r;
  int32_t dense;
  int32_t ox, oy, oz;      // dense: key of grid cell (0, 0, 0)
  uint32_t nx, ny, nz;     // dense: grid dimensions
};

// host-side voxelmap
struct glim_vmap {
  int device = 0;
  int levels = 0;
  double res[GLIM_MAX_LEVELS] = {0};
  float inv_r[GLIM_MAX_LEVELS] = {0};
  int64_t n_vox[GLIM_MAX_LEVELS] = {0};
  int64_t cap[GLIM_MAX_LEVELS] = {0};
  int32_t log2cap[GLIM_MAX_LEVELS] = {0};
  int32_t max_probe[GLIM_MAX_LEVELS] = {0};
  VoxSlot* slots[GLIM_MAX_LEVELS] = {nullptr};       // cell 0 (grid or block cells)
  VoxSlot* slots_alloc[GLIM_MAX_LEVELS] = {nullptr}; // allocation: an empty record at slots - 1
  int4* btab[GLIM_MAX_LEVELS] = {nullptr};           // hashed: block table (cap entries)
  int64_t nblk[GLIM_MAX_LEVELS] = {0};               // hashed: number of blocks
  int32_t dense[GLIM_MAX_LEVELS] = {0};
  int32_t org[GLIM_MAX_LEVELS][3] = {};
  uint32_t dim[GLIM_MAX_LEVELS][3] = {};
  unsigned long long* vkey[GLIM_MAX_LEVELS] = {nullptr};  // canonical order
  float* vmean[GLIM_MAX_LEVELS] = {nullptr};              // n_vox x 3
  float* vcov[GLIM_MAX_LEVELS] = {nullptr};               // n_vox x 6
  int32_t* vcount[GLIM_MAX_LEVELS] = {nullptr};
  double* vsum[GLIM_MAX_LEVELS] = {nullptr};              // n_vox x 9 FP64 sums (mean 3, cov 6)
  uint64_t version = 0;  // incremented whenever the tables are replaced (insertion)
  uint64_t serial = 0;   // unique per map of the process (registry of live maps)
  LevelDev dev(int l) const {
    LevelDev d;
    d.slots = slots[l];
    d.btab = btab[l];
    d.unused = nullptr;
    d.mask = uint32_t(cap[l] - 1);
    d.log2cap = log2cap[l];
    d.max_probe = max_probe[l];
    d.inv_r = inv_r[l];
    d.dense = dense[l];
    d.ox = org[l][0];
    d.oy = org[l][1];
    d.oz = org[l][2];
    d.nx = dim[l][0];
    d.ny = dim[l][1];
    d.nz = dim[l][2];
    return d;
  }
};

// Registry of the live voxelmaps of the process, so that a plan can tell, without touching a
// freed map, whether its target maps still exist unchanged: every map gets a unique serial
// when it is registered; freeing a map unregisters it.  The epoch changes whenever a map is
// freed or its tables are replaced, so a plan re-checks its maps only after such a change.
void vmap_register(glim_vmap* vm);
void vmap_unregister(glim_vmap* vm);
bool vmap_alive(const glim_vmap* vm, uint64_t serial);  // registered under that serial
uint64_t vmap_epoch();
void vmap_bump_epoch();

// per-pair relative pose in FP32 as used by the point loop
struct __align__(16) PoseF {
  float R[9];
  float t[3];
  float v[3];  // target viewpoint in the source frame, -R^T t
  float pad;
};

// host helpers shared by the linearize / backward / correspondence paths
struct RelPose {
  double R[9], t[3];
};
RelPose relative_pose(const double* pose_s12, const double* pose_t12);
PoseF pose_to_f32(const RelPose& T);

// ------------------------------------------------------------------ primitives (sort.cu)
// Exclusive prefix sum of n uint32 values (in may equal out).  tmp is managed internally.
glim_status scan_exclusive_u32(glim_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n);
// Stable LSD radix sort of (key, value) pairs by the key bits in `varying` (bits that are
// not set in `varying` are equal in all keys).  Results in keys_out / vals_out.
glim_status radix_sort_pairs(glim_ctx* ctx, const unsigned long long* keys_in, const uint32_t* vals_in,
                             unsigned long long* keys_out, uint32_t* vals_out, int64_t n,
                             unsigned long long varying);
// OR over (k ^ k[0]) of all keys: the bits that vary.
glim_status key_varying_bits(glim_ctx* ctx, const unsigned long long* keys, int64_t n,
                             unsigned long long* varying_host);

// builds a sorted grid (keys of points at inv_r, their sorted order, unique cells)
struct SortedCells {
  DevBuf<unsigned long long> key_sorted;  // n
  DevBuf<uint32_t> idx_sorted;            // n
  DevBuf<uint32_t> cell_start;            // m + 1
  DevBuf<unsigned long long> cell_key;    // m
  int64_t m = 0;
};
glim_status sort_into_cells(glim_ctx* ctx, const float* pts4, int64_t n, float inv_r, SortedCells& out,
                            bool range_is_error);
// Segments (unique keys and their first positions) of an already sorted key array; fills
// out.cell_start (m + 1), out.cell_key (m) and out.m.  EMPTY keys (sorted last) are excluded.
glim_status segment_sorted(glim_ctx* ctx, const unsigned long long* key_sorted, int64_t n, SortedCells& out);

inline int ceil_div_i(int64_t a, int64_t b) { return int((a + b - 1) / b); }
