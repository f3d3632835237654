// voxelmap.cu -- multi-resolution voxelmap build (Sec. III-C "Preprocessing"), export,
// per-point correspondences and the overlap rate (Sec. IV-B).
//
// Build of one level:
//   1. voxel key of every point (FP32 floor(x * inv_r)), sorted with its point index by a
//      stable radix sort, so the members of a voxel are contiguous and in point order;
//   2. one thread per voxel sums its members' means and covariances in FP64 in that order
//      and stores the averages (canonical id = rank of the key = position in sorted order);
//   3. the voxel records (48 bytes) are written into a dense grid over their key box when it
//      is small enough, else into voxel blocks (2 x 2 x 2 cells) found through an
//      open-addressing table of block keys (linear probing, load <= 1/16): spatial hashing of
//      voxel blocks, as voxel hashing does.
#include <climits>

#include "lookup.cuh"

namespace {

__global__ void k_voxel_stats(const float4* __restrict__ pts, const float* __restrict__ cov6,
                              const uint32_t* __restrict__ idx_sorted, const uint32_t* __restrict__ cell_start,
                              const unsigned long long* __restrict__ cell_key, int64_t m,
                              unsigned long long* __restrict__ vkey, float* __restrict__ vmean,
                              float* __restrict__ vcov, int32_t* __restrict__ vcount, double* __restrict__ vsum,
                              unsigned int* __restrict__ status) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= m) return;
  const uint32_t b = cell_start[v], e = cell_start[v + 1];
  double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (uint32_t j = b; j < e; ++j) {
    const uint32_t i = idx_sorted[j];
    const float4 p = pts[i];
    s[0] += p.x;
    s[1] += p.y;
    s[2] += p.z;
    const float2* c = reinterpret_cast<const float2*>(cov6 + 6 * int64_t(i));
    const float2 c0 = c[0], c1 = c[1], c2 = c[2];
    if (!(isfinite(c0.x) && isfinite(c0.y) && isfinite(c1.x) && isfinite(c1.y) && isfinite(c2.x) && isfinite(c2.y)))
      atomicOr(status, GLIM_DS_NONFINITE);
    s[3] += c0.x;
    s[4] += c0.y;
    s[5] += c1.x;
    s[6] += c1.y;
    s[7] += c2.x;
    s[8] += c2.y;
  }
  const double inv = 1.0 / double(e - b);
  for (int c = 0; c < 9; ++c) vsum[9 * v + c] = s[c];
  vkey[v] = cell_key[v];
  for (int c = 0; c < 3; ++c) vmean[3 * v + c] = float(s[c] * inv);
  for (int c = 0; c < 6; ++c) vcov[6 * v + c] = float(s[3 + c] * inv);
  vcount[v] = int32_t(e - b);
}

// Block key of every voxel (its key >> 1 per axis, packed), with the voxel's index.
__global__ void k_block_keys(const unsigned long long* __restrict__ vkey, int64_t m, unsigned long long* __restrict__ bkey,
                             uint32_t* __restrict__ idx) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= m) return;
  const unsigned long long k = vkey[v];
  bkey[v] = pack_key(unpack_x(k) >> GLIM_BLOCK_SHIFT, unpack_y(k) >> GLIM_BLOCK_SHIFT, unpack_z(k) >> GLIM_BLOCK_SHIFT);
  idx[v] = uint32_t(v);
}

// One thread per block (blocks in sorted block-key order; the block index is the rank): its
// entry {bx, by, bz, block} goes into the table by linear probing, claimed through its first
// 8 bytes (bx, by); block keys are unique, so a claimed slot is never claimed again.
__global__ void k_block_table(const unsigned long long* __restrict__ bkey_unique, int64_t nblk, int4* __restrict__ btab,
                              int log2cap, uint32_t mask, int* __restrict__ max_probe,
                              unsigned int* __restrict__ status) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  const unsigned long long key = bkey_unique[b];
  const int bx = unpack_x(key), by = unpack_y(key), bz = unpack_z(key);
  const unsigned long long xy = (unsigned long long)(uint32_t)bx | ((unsigned long long)(uint32_t)by << 32);
  uint32_t h = hash3(bx, by, bz, log2cap);
  for (uint32_t p = 0; p <= mask; ++p) {
    unsigned long long* kp = reinterpret_cast<unsigned long long*>(&btab[h]);
    if (atomicCAS(kp, GLIM_EMPTY_XY, xy) == GLIM_EMPTY_XY) {
      int* e = reinterpret_cast<int*>(&btab[h]);
      e[2] = bz;
      e[3] = int(b);
      atomicMax(max_probe, int(p + 1));
      return;
    }
    h = (h + 1u) & mask;
  }
  atomicOr(status, GLIM_DS_HASHFULL);
}

// The voxel record {id, C~22, kx, C~22} {mean, C~00} {C~01, C~02, C~11, C~12} of voxel v.
__device__ __forceinline__ VoxSlot voxel_record(const unsigned long long* __restrict__ vkey, const float* __restrict__ vmean,
                                                const float* __restrict__ vcov, int64_t v) {
  const int kx = unpack_x(vkey[v]);
  VoxSlot r;
  r.w0 = make_float4(__int_as_float(int(v)), vcov[6 * v + 5], __int_as_float(kx), vcov[6 * v + 5]);
  r.w1 = make_float4(vmean[3 * v], vmean[3 * v + 1], vmean[3 * v + 2], vcov[6 * v + 0]);
  r.w2 = make_float4(vcov[6 * v + 1], vcov[6 * v + 2], vcov[6 * v + 3], vcov[6 * v + 4]);
  return r;
}

// One thread per block: the records of its voxels (sorted positions start[b] .. start[b+1]-1,
// at most 8) into its cells.
__global__ void k_block_scatter(const uint32_t* __restrict__ start, const uint32_t* __restrict__ idx_sorted, int64_t nblk,
                                const unsigned long long* __restrict__ vkey, const float* __restrict__ vmean,
                                const float* __restrict__ vcov, VoxSlot* __restrict__ cells) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  for (uint32_t j = start[b]; j < start[b + 1]; ++j) {
    const int64_t v = idx_sorted[j];
    const unsigned long long k = vkey[v];
    cells[b * GLIM_BLOCK_CELLS + block_local(unpack_x(k), unpack_y(k), unpack_z(k))] = voxel_record(vkey, vmean, vcov, v);
  }
}

// Merge of two canonical voxel sets: entries [0, m_old) are the existing voxels, [m_old, ...)
// the voxels of the inserted points; `src` lists them in key order (equal keys: existing
// first), `start` delimits the merged voxels.  Sums are added in that order.
__global__ void k_merge_voxels(const uint32_t* __restrict__ src, const uint32_t* __restrict__ start,
                               const unsigned long long* __restrict__ mkey, int64_t m, int64_t m_old,
                               const double* __restrict__ sum_old, const int32_t* __restrict__ cnt_old,
                               const double* __restrict__ sum_new, const int32_t* __restrict__ cnt_new,
                               unsigned long long* __restrict__ vkey, float* __restrict__ vmean,
                               float* __restrict__ vcov, int32_t* __restrict__ vcount, double* __restrict__ vsum) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= m) return;
  double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int64_t cnt = 0;
  for (uint32_t j = start[v]; j < start[v + 1]; ++j) {
    const int64_t i = src[j];
    const double* a = i < m_old ? sum_old + 9 * i : sum_new + 9 * (i - m_old);
    cnt += i < m_old ? cnt_old[i] : cnt_new[i - m_old];
    for (int c = 0; c < 9; ++c) s[c] += a[c];
  }
  const double inv = 1.0 / double(cnt);
  vkey[v] = mkey[v];
  for (int c = 0; c < 9; ++c) vsum[9 * v + c] = s[c];
  for (int c = 0; c < 3; ++c) vmean[3 * v + c] = float(s[c] * inv);
  for (int c = 0; c < 6; ++c) vcov[6 * v + c] = float(s[3 + c] * inv);
  vcount[v] = int32_t(cnt);
}

__global__ void k_iota_offset(uint32_t* __restrict__ a, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) a[i] = uint32_t(i);
}

__global__ void k_key_bbox(const unsigned long long* __restrict__ vkey, int64_t m, int* __restrict__ bb) {
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < m; v += int64_t(gridDim.x) * blockDim.x) {
    const unsigned long long k = vkey[v];
    const int c[3] = {unpack_x(k), unpack_y(k), unpack_z(k)};
    for (int a = 0; a < 3; ++a) {
      mn[a] = min(mn[a], c[a]);
      mx[a] = max(mx[a], c[a]);
    }
  }
  for (int a = 0; a < 3; ++a) {
    atomicMin(&bb[a], mn[a]);
    atomicMax(&bb[3 + a], mx[a]);
  }
}

// dense layout: the voxel record stored in its grid cell, w0 = {canonical id, kx, ky, c22}
__global__ void k_dense_build(const unsigned long long* __restrict__ vkey, const float* __restrict__ vmean,
                              const float* __restrict__ vcov, int64_t m, VoxSlot* __restrict__ cells,
                              int ox, int oy, int oz, uint32_t ny, uint32_t nz) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= m) return;
  const unsigned long long key = vkey[v];
  const int kx = unpack_x(key), ky = unpack_y(key), kz = unpack_z(key);
  cells[(int64_t(kx - ox) * ny + (ky - oy)) * nz + (kz - oz)] = voxel_record(vkey, vmean, vcov, v);
}

__global__ void k_export(const unsigned long long* __restrict__ vkey, const float* __restrict__ vmean,
                         const float* __restrict__ vcov, const int32_t* __restrict__ vcount, int64_t m,
                         int32_t* keys3, float* mean3, float* cov6, int32_t* count) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= m) return;
  const unsigned long long k = vkey[v];
  if (keys3) {
    keys3[3 * v] = unpack_x(k);
    keys3[3 * v + 1] = unpack_y(k);
    keys3[3 * v + 2] = unpack_z(k);
  }
  if (mean3)
    for (int c = 0; c < 3; ++c) mean3[3 * v + c] = vmean[3 * v + c];
  if (cov6)
    for (int c = 0; c < 6; ++c) cov6[6 * v + c] = vcov[6 * v + c];
  if (count) count[v] = vcount[v];
}

struct CorrArgs {
  const float4* pts;
  const float* nrm;
  int64_t n;
  PoseF pose;
  LevelDev lv[GLIM_MAX_LEVELS];
  int levels;
  int validate;
};

__global__ void k_correspondences(const CorrArgs a, int32_t* __restrict__ ids) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  const float4 m = a.pts[k];
  bool visible = true;
  if (a.validate && a.nrm)
    visible = !behind_surface(m.x, m.y, m.z, a.pose.v, a.nrm[3 * k], a.nrm[3 * k + 1], a.nrm[3 * k + 2]);
  const float3 q = transform_pinned(a.pose.R, a.pose.t, m.x, m.y, m.z);
  for (int l = 0; l < a.levels; ++l) {
    int32_t id = -1;
    int kx, ky, kz;
    if (visible && level_key3(q, a.lv[l].inv_r, kx, ky, kz)) find_voxel(a.lv[l], kx, ky, kz, &id);
    ids[k * a.levels + l] = id;
  }
}

struct OverlapPair {
  const float4* pts;
  int64_t n;
  LevelDev lv;
  PoseF pose;
};

// One block per pair; each thread takes OV_UNROLL points per step so that their point reads,
// and then their voxel reads, are in flight together (a dense level reads only the 4-byte id).
constexpr int OV_UNROLL = 4;

__global__ void __launch_bounds__(256) k_overlap(const OverlapPair* __restrict__ pairs, double* __restrict__ out) {
  const OverlapPair& P = pairs[blockIdx.x];
  const int64_t n = P.n;
  const float4* pts = P.pts;
  const LevelDev L = P.lv;
  float R[9], t[3];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = P.pose.R[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = P.pose.t[i];
  int64_t hits = 0;
  const int64_t step = int64_t(OV_UNROLL) * blockDim.x;
  for (int64_t k0 = threadIdx.x; k0 < n; k0 += step) {
    float4 m[OV_UNROLL];
#pragma unroll
    for (int u = 0; u < OV_UNROLL; ++u) {
      const int64_t k = k0 + int64_t(u) * blockDim.x;
      m[u] = k < n ? ldg4(&pts[k]) : make_float4(NAN, NAN, NAN, 1.f);
    }
    if (L.dense) {
      int id[OV_UNROLL];
#pragma unroll
      for (int u = 0; u < OV_UNROLL; ++u) {
        const float3 q = transform_pinned(R, t, m[u].x, m[u].y, m[u].z);
        int kx, ky, kz;
        const int64_t c = level_key3(q, L.inv_r, kx, ky, kz) ? dense_cell(L, kx, ky, kz) : -1;
        id[u] = c >= 0 ? __ldg(reinterpret_cast<const int*>(&L.slots[c].w0)) : -1;
      }
#pragma unroll
      for (int u = 0; u < OV_UNROLL; ++u) hits += id[u] >= 0 ? 1 : 0;
    } else {
#pragma unroll
      for (int u = 0; u < OV_UNROLL; ++u) {
        const float3 q = transform_pinned(R, t, m[u].x, m[u].y, m[u].z);
        int kx, ky, kz, id;
        if (level_key3(q, L.inv_r, kx, ky, kz) && find_voxel(L, kx, ky, kz, &id) >= 0) ++hits;
      }
    }
  }
  __shared__ unsigned long long s[8];
  unsigned long long h = __reduce_add_sync(0xffffffffu, unsigned(hits));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = h;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += s[w];
    out[blockIdx.x] = P.n > 0 ? double(t) / double(P.n) : 0.0;
  }
}

int log2_ceil(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}

// A map's arrays come from the stream-ordered allocator (cudaMallocAsync on the context
// stream).  free_on returns one in the order of stream s; free_level releases a level's arrays
// at once and does not wait for the device: every caller has made sure first that no launch
// on any stream still reads them.
template <class T>
void free_on(T* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void free_level(glim_vmap* vm, int l) {
  cudaFree(vm->slots_alloc[l]);
  cudaFree(vm->btab[l]);
  cudaFree(vm->vkey[l]);
  cudaFree(vm->vmean[l]);
  cudaFree(vm->vcov[l]);
  cudaFree(vm->vcount[l]);
  cudaFree(vm->vsum[l]);
  vm->slots[l] = nullptr;
  vm->slots_alloc[l] = nullptr;
  vm->btab[l] = nullptr;
  vm->vkey[l] = nullptr;
  vm->vmean[l] = nullptr;
  vm->vcov[l] = nullptr;
  vm->vcount[l] = nullptr;
  vm->vsum[l] = nullptr;
}

void free_levels(glim_vmap* vm) {
  for (int l = 0; l < GLIM_MAX_LEVELS; ++l) free_level(vm, l);
}

// Level l of src replaces level l of dst (whose arrays are freed); src gives up its arrays.
void move_level(glim_vmap* dst, glim_vmap* src, int l) {
  free_level(dst, l);
  dst->n_vox[l] = src->n_vox[l];
  dst->cap[l] = src->cap[l];
  dst->log2cap[l] = src->log2cap[l];
  dst->max_probe[l] = src->max_probe[l];
  dst->dense[l] = src->dense[l];
  for (int c = 0; c < 3; ++c) {
    dst->org[l][c] = src->org[l][c];
    dst->dim[l][c] = src->dim[l][c];
  }
  dst->slots[l] = src->slots[l];
  dst->slots_alloc[l] = src->slots_alloc[l];
  dst->btab[l] = src->btab[l];
  dst->nblk[l] = src->nblk[l];
  dst->vkey[l] = src->vkey[l];
  dst->vmean[l] = src->vmean[l];
  dst->vcov[l] = src->vcov[l];
  dst->vcount[l] = src->vcount[l];
  dst->vsum[l] = src->vsum[l];
  src->slots[l] = nullptr;
  src->slots_alloc[l] = nullptr;
  src->btab[l] = nullptr;
  src->vkey[l] = nullptr;
  src->vmean[l] = nullptr;
  src->vcov[l] = nullptr;
  src->vcount[l] = nullptr;
  src->vsum[l] = nullptr;
}

// Dense grids (48 bytes per cell) are used when the key bounding box has at most this many
// cells per occupied voxel plus a fixed allowance, and at most DENSE_MAX_BYTES per level.
constexpr int64_t DENSE_CELLS_PER_VOXEL = 256;
constexpr int64_t DENSE_CELLS_ALLOWANCE = int64_t(1) << 22;
constexpr int64_t DENSE_MAX_BYTES = int64_t(32) << 30;

// Canonical voxel arrays (sorted keys, FP64 sums, counts, means, covariances) of a point set
// at one resolution; the arrays are allocated here and owned by the caller.
struct Canon {
  int64_t m = 0;
  unsigned long long* key = nullptr;
  double* sum = nullptr;
  int32_t* count = nullptr;
  float* mean = nullptr;
  float* cov = nullptr;
  cudaStream_t s = nullptr;  // the stream the arrays were allocated on (stream-ordered)
  void release() {
    free_on(key, s);
    free_on(sum, s);
    free_on(count, s);
    free_on(mean, s);
    free_on(cov, s);
    key = nullptr;
    sum = nullptr;
    count = nullptr;
    mean = nullptr;
    cov = nullptr;
  }
};

glim_status canon_alloc(glim_ctx* ctx, Canon& c, int64_t m) {
  c.m = m;
  c.s = ctx->stream;
  const size_t mm = size_t(std::max<int64_t>(m, 1));
  GLIM_CUDA(ctx, dmalloc_async(&c.key, mm * sizeof(unsigned long long), ctx->stream));
  GLIM_CUDA(ctx, dmalloc_async(&c.sum, mm * 9 * sizeof(double), ctx->stream));
  GLIM_CUDA(ctx, dmalloc_async(&c.count, mm * sizeof(int32_t), ctx->stream));
  GLIM_CUDA(ctx, dmalloc_async(&c.mean, mm * 3 * sizeof(float), ctx->stream));
  GLIM_CUDA(ctx, dmalloc_async(&c.cov, mm * 6 * sizeof(float), ctx->stream));
  return GLIM_OK;
}

glim_status canon_from_points(glim_ctx* ctx, const float* pts4, const float* cov6, int64_t n, float inv_r, Canon& c) {
  SortedCells cells;
  glim_status st = sort_into_cells(ctx, pts4, n, inv_r, cells, true);
  if (st != GLIM_OK) return st;
  st = take_device_status(ctx, "voxel keys");
  if (st != GLIM_OK) return st;
  st = canon_alloc(ctx, c, cells.m);
  if (st != GLIM_OK) return st;
  if (c.m > 0) {
    k_voxel_stats<<<ceil_div_i(c.m, 128), 128, 0, ctx->stream>>>(
        reinterpret_cast<const float4*>(pts4), cov6, cells.idx_sorted.p, cells.cell_start.p, cells.cell_key.p, c.m,
        c.key, c.mean, c.cov, c.count, c.sum, ctx->d_status);
    GLIM_LAUNCHED(ctx);
  }
  return take_device_status(ctx, "voxel statistics");
}

void adopt_canon(glim_vmap* vm, int l, Canon& c) {
  vm->n_vox[l] = c.m;
  vm->vkey[l] = c.key;
  vm->vsum[l] = c.sum;
  vm->vcount[l] = c.count;
  vm->vmean[l] = c.mean;
  vm->vcov[l] = c.cov;
  c.key = nullptr;
  c.sum = nullptr;
  c.count = nullptr;
  c.mean = nullptr;
  c.cov = nullptr;
}

// Lookup tables of a level (dense grid or hash) from its canonical arrays; replaces any
// existing tables of the level.
glim_status build_tables(glim_ctx* ctx, glim_vmap* vm, int l, int layout) {
  // the level belongs to a map under construction: only this stream has used its tables
  free_on(vm->slots_alloc[l], ctx->stream);
  free_on(vm->btab[l], ctx->stream);
  vm->slots[l] = nullptr;
  vm->slots_alloc[l] = nullptr;
  vm->btab[l] = nullptr;
  vm->nblk[l] = 0;
  vm->dense[l] = 0;
  const int64_t m = vm->n_vox[l];
  // dense grid over the key bounding box when it is small enough (or requested)
  int bb[6] = {0, 0, 0, -1, -1, -1};
  if (m > 0) {
    DevBuf<int> dbb;
    GLIM_CUDA(ctx, dbb.alloc(6, ctx->stream));
    const int init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    GLIM_CUDA(ctx, cudaMemcpyAsync(dbb.p, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    k_key_bbox<<<std::min(ceil_div_i(m, 256), 4 * ctx->num_sms), 256, 0, ctx->stream>>>(vm->vkey[l], m, dbb.p);
    GLIM_LAUNCHED(ctx);
    GLIM_CUDA(ctx, cudaMemcpyAsync(bb, dbb.p, sizeof(bb), cudaMemcpyDeviceToHost, ctx->stream));
    GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  const int64_t nx = int64_t(bb[3]) - bb[0] + 1, ny = int64_t(bb[4]) - bb[1] + 1, nz = int64_t(bb[5]) - bb[2] + 1;
  const int64_t ncell = m > 0 ? nx * ny * nz : 0;
  const bool fits = ncell < (int64_t(1) << 31) && ncell <= DENSE_CELLS_PER_VOXEL * m + DENSE_CELLS_ALLOWANCE &&
                    ncell * int64_t(sizeof(VoxSlot)) <= DENSE_MAX_BYTES;
  if (layout == 1 && !fits)
    return set_error(ctx, GLIM_EINVAL, "build_voxelmap: dense layout requested but the grid has %lld cells",
                     (long long)ncell);
  if (m > 0 && (layout == 1 || (layout == 0 && fits))) {
    vm->dense[l] = 1;
    vm->org[l][0] = bb[0];
    vm->org[l][1] = bb[1];
    vm->org[l][2] = bb[2];
    vm->dim[l][0] = uint32_t(nx);
    vm->dim[l][1] = uint32_t(ny);
    vm->dim[l][2] = uint32_t(nz);
    vm->cap[l] = ncell;
    vm->log2cap[l] = 0;
    vm->max_probe[l] = 1;
    // one empty record before cell 0: lookups outside the box may read it instead of branching
    GLIM_CUDA(ctx, dmalloc_async(&vm->slots_alloc[l], (ncell + 1) * sizeof(VoxSlot), ctx->stream));
    GLIM_CUDA(ctx, cudaMemsetAsync(vm->slots_alloc[l], 0x80, (ncell + 1) * sizeof(VoxSlot), ctx->stream));
    vm->slots[l] = vm->slots_alloc[l] + 1;
    k_dense_build<<<ceil_div_i(m, 256), 256, 0, ctx->stream>>>(vm->vkey[l], vm->vmean[l], vm->vcov[l], m,
                                                               vm->slots[l], bb[0], bb[1], bb[2], uint32_t(ny),
                                                               uint32_t(nz));
    GLIM_LAUNCHED(ctx);
    return take_device_status(ctx, "voxel statistics / dense grid");
  }
  // voxel blocks: the voxels' block keys sorted (stable, so a block's voxels stay in id order)
  // and segmented; a block's index is its rank
  int64_t nblk = 0;
  SortedCells blk;
  {
    DevBuf<unsigned long long> bkey;
    DevBuf<uint32_t> bidx;
    GLIM_CUDA(ctx, bkey.alloc(std::max<int64_t>(m, 1), ctx->stream));
    GLIM_CUDA(ctx, bidx.alloc(std::max<int64_t>(m, 1), ctx->stream));
    GLIM_CUDA(ctx, blk.key_sorted.alloc(std::max<int64_t>(m, 1), ctx->stream));
    GLIM_CUDA(ctx, blk.idx_sorted.alloc(std::max<int64_t>(m, 1), ctx->stream));
    if (m > 0) {
      k_block_keys<<<ceil_div_i(m, 256), 256, 0, ctx->stream>>>(vm->vkey[l], m, bkey.p, bidx.p);
      GLIM_LAUNCHED(ctx);
      unsigned long long varying = 0;
      glim_status st = key_varying_bits(ctx, bkey.p, m, &varying);
      if (st != GLIM_OK) return st;
      st = radix_sort_pairs(ctx, bkey.p, bidx.p, blk.key_sorted.p, blk.idx_sorted.p, m, varying);
      if (st != GLIM_OK) return st;
      st = segment_sorted(ctx, blk.key_sorted.p, m, blk);
      if (st != GLIM_OK) return st;
      nblk = blk.m;
    }
  }
  const int64_t cap = std::max<int64_t>(16, int64_t(1) << log2_ceil(16 * nblk));  // load <= 1/16
  vm->cap[l] = cap;
  vm->log2cap[l] = log2_ceil(cap);
  vm->nblk[l] = nblk;
  GLIM_CUDA(ctx, dmalloc_async(&vm->btab[l], cap * sizeof(int4), ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(vm->btab[l], 0x80, cap * sizeof(int4), ctx->stream));
  // cell records: one empty record before cell 0, then 8 cells per block
  const int64_t nbcell = nblk * GLIM_BLOCK_CELLS;
  GLIM_CUDA(ctx, dmalloc_async(&vm->slots_alloc[l], (nbcell + 1) * sizeof(VoxSlot), ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(vm->slots_alloc[l], 0x80, (nbcell + 1) * sizeof(VoxSlot), ctx->stream));
  vm->slots[l] = vm->slots_alloc[l] + 1;
  if (m == 0) {
    vm->max_probe[l] = 1;
    return GLIM_OK;
  }
  DevBuf<int> maxp;
  GLIM_CUDA(ctx, maxp.alloc(1, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(maxp.p, 0, sizeof(int), ctx->stream));
  k_block_table<<<ceil_div_i(nblk, 256), 256, 0, ctx->stream>>>(blk.cell_key.p, nblk, vm->btab[l], vm->log2cap[l],
                                                                uint32_t(cap - 1), maxp.p, ctx->d_status);
  GLIM_LAUNCHED(ctx);
  k_block_scatter<<<ceil_div_i(nblk, 256), 256, 0, ctx->stream>>>(blk.cell_start.p, blk.idx_sorted.p, nblk, vm->vkey[l],
                                                                  vm->vmean[l], vm->vcov[l], vm->slots[l]);
  GLIM_LAUNCHED(ctx);
  int mp = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&mp, maxp.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  vm->max_probe[l] = mp;
  return take_device_status(ctx, "voxel statistics / block table");
}

glim_status build_level(glim_ctx* ctx, const float* pts4, const float* cov6, int64_t n, glim_vmap* vm, int l,
                        int layout) {
  Canon c;
  glim_status st = canon_from_points(ctx, pts4, cov6, n, vm->inv_r[l], c);
  if (st != GLIM_OK) {
    cudaStreamSynchronize(ctx->stream);
    c.release();
    return st;
  }
  adopt_canon(vm, l, c);
  return build_tables(ctx, vm, l, layout);
}

// Level l of `out` = level l of `vm` with the points added: the canonical voxels of the new
// points are merged with the existing ones by a stable sort of the concatenated keys
// (existing entries first), their FP64 sums added, and the tables rebuilt.  The ids are
// again the ranks of the keys, so the result equals a build from all points up to the
// order of the FP64 additions.
glim_status insert_level(glim_ctx* ctx, const glim_vmap* vm, glim_vmap* out, int l, const float* pts4,
                         const float* cov6, int64_t n, int layout) {
  Canon add, merged;
  auto fail = [&](glim_status st) {
    cudaStreamSynchronize(ctx->stream);
    add.release();
    merged.release();
    return st;
  };
  glim_status st = canon_from_points(ctx, pts4, cov6, n, vm->inv_r[l], add);
  if (st != GLIM_OK) return fail(st);
  const int64_t m0 = vm->n_vox[l], m1 = add.m, mt = m0 + m1;
  if (mt > 0x7FFFFFFFll) return fail(set_error(ctx, GLIM_EINVAL, "vmap_insert: too many voxels"));
  SortedCells seg;
  {
    DevBuf<unsigned long long> ck, ks;
    DevBuf<uint32_t> cv, vs;
    const size_t mm = size_t(std::max<int64_t>(mt, 1));
    if (ck.alloc(mm, ctx->stream) != cudaSuccess || ks.alloc(mm, ctx->stream) != cudaSuccess ||
        cv.alloc(mm, ctx->stream) != cudaSuccess || vs.alloc(mm, ctx->stream) != cudaSuccess)
      return fail(set_error(ctx, GLIM_ENOMEM, "vmap_insert: device allocation failed"));
    if (m0 > 0 && cudaMemcpyAsync(ck.p, vm->vkey[l], m0 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                  ctx->stream) != cudaSuccess)
      return fail(set_error(ctx, GLIM_ECUDA, "vmap_insert: copy failed"));
    if (m1 > 0 && cudaMemcpyAsync(ck.p + m0, add.key, m1 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                                  ctx->stream) != cudaSuccess)
      return fail(set_error(ctx, GLIM_ECUDA, "vmap_insert: copy failed"));
    if (mt > 0) {
      k_iota_offset<<<ceil_div_i(mt, 256), 256, 0, ctx->stream>>>(cv.p, mt);
      if (cudaGetLastError() != cudaSuccess) return fail(set_error(ctx, GLIM_ECUDA, "vmap_insert: launch failed"));
      ctx->launches += 1;
      unsigned long long varying = 0;
      st = key_varying_bits(ctx, ck.p, mt, &varying);
      if (st == GLIM_OK) st = radix_sort_pairs(ctx, ck.p, cv.p, ks.p, vs.p, mt, varying);
      if (st == GLIM_OK) st = segment_sorted(ctx, ks.p, mt, seg);
      if (st != GLIM_OK) return fail(st);
    }
    st = canon_alloc(ctx, merged, seg.m);
    if (st != GLIM_OK) return fail(st);
    if (seg.m > 0) {
      k_merge_voxels<<<ceil_div_i(seg.m, 128), 128, 0, ctx->stream>>>(
          vs.p, seg.cell_start.p, seg.cell_key.p, seg.m, m0, vm->vsum[l], vm->vcount[l], add.sum, add.count,
          merged.key, merged.mean, merged.cov, merged.count, merged.sum);
      if (cudaGetLastError() != cudaSuccess) return fail(set_error(ctx, GLIM_ECUDA, "vmap_insert: launch failed"));
      ctx->launches += 1;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      return fail(set_error(ctx, GLIM_ECUDA, "vmap_insert: merge failed"));
  }
  add.release();
  adopt_canon(out, l, merged);
  return build_tables(ctx, out, l, layout);
}

}  // namespace

extern "C" glim_status glim_build_voxelmap(glim_ctx* ctx, const float* pts4, const float* cov6, int64_t n,
                                           const double* resolutions, int32_t levels, glim_vmap** out) {
  return glim_build_voxelmap_ex(ctx, pts4, cov6, n, resolutions, levels, 0, out);
}

extern "C" glim_status glim_build_voxelmap_ex(glim_ctx* ctx, const float* pts4, const float* cov6, int64_t n,
                                              const double* resolutions, int32_t levels, int32_t layout,
                                              glim_vmap** out) {
  GLIM_RANGE("glim_build_voxelmap_ex");
  if (!ctx || !out) return GLIM_EINVAL;
  if (layout < 0 || layout > 2) return set_error(ctx, GLIM_EINVAL, "build_voxelmap: layout must be 0, 1 or 2");
  *out = nullptr;
  if (n < 0 || (n > 0 && (!pts4 || !cov6)) || !resolutions || levels < 1 || levels > GLIM_MAX_LEVELS)
    return set_error(ctx, GLIM_EINVAL, "build_voxelmap: bad arguments (n=%lld levels=%d)", (long long)n, levels);
  if (n > 0x7FFFFFFFll) return set_error(ctx, GLIM_EINVAL, "build_voxelmap: n too large");
  if ((reinterpret_cast<uintptr_t>(pts4) & 15) || (reinterpret_cast<uintptr_t>(cov6) & 7))
    return set_error(ctx, GLIM_EINVAL, "build_voxelmap: pts4 must be 16-byte and cov6 8-byte aligned");
  for (int l = 0; l < levels; ++l)
    if (!(resolutions[l] > 0.0) || !std::isfinite(resolutions[l]))
      return set_error(ctx, GLIM_EINVAL, "build_voxelmap: resolution %d is not positive", l);
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  glim_vmap* vm = new glim_vmap;
  vm->device = ctx->device;
  vm->levels = levels;
  for (int l = 0; l < levels; ++l) {
    vm->res[l] = resolutions[l];
    vm->inv_r[l] = float(1.0 / resolutions[l]);
    glim_status st = build_level(ctx, pts4, cov6, n, vm, l, layout);
    if (st != GLIM_OK) {
      cudaStreamSynchronize(ctx->stream);
      free_levels(vm);
      delete vm;
      return st;
    }
  }
  vmap_register(vm);
  *out = vm;
  ctx->err.clear();
  return GLIM_OK;
}

extern "C" glim_status glim_vmap_insert(glim_ctx* ctx, glim_vmap* vm, const float* pts4, const float* cov6, int64_t n,
                                        int32_t layout) {
  GLIM_RANGE("glim_vmap_insert");
  if (!ctx || !vm) return GLIM_EINVAL;
  if (layout < 0 || layout > 2) return set_error(ctx, GLIM_EINVAL, "vmap_insert: layout must be 0, 1 or 2");
  if (n < 0 || (n > 0 && (!pts4 || !cov6)))
    return set_error(ctx, GLIM_EINVAL, "vmap_insert: bad arguments (n=%lld)", (long long)n);
  if (n > 0x7FFFFFFFll) return set_error(ctx, GLIM_EINVAL, "vmap_insert: n too large");
  if ((reinterpret_cast<uintptr_t>(pts4) & 15) || (reinterpret_cast<uintptr_t>(cov6) & 7))
    return set_error(ctx, GLIM_EINVAL, "vmap_insert: pts4 must be 16-byte and cov6 8-byte aligned");
  if (vm->device != ctx->device) return set_error(ctx, GLIM_EINVAL, "vmap_insert: map and context devices differ");
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  // every level is rebuilt into a scratch map first, so that a failure leaves vm unchanged
  glim_vmap tmp;
  tmp.device = vm->device;
  tmp.levels = vm->levels;
  for (int l = 0; l < vm->levels; ++l) {
    tmp.res[l] = vm->res[l];
    tmp.inv_r[l] = vm->inv_r[l];
    glim_status st = insert_level(ctx, vm, &tmp, l, pts4, cov6, n, layout);
    if (st != GLIM_OK) {
      cudaStreamSynchronize(ctx->stream);
      free_levels(&tmp);
      return st;
    }
  }
  // no launch on any stream may still read the old tables when they are freed
  const cudaError_t ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) {
    free_levels(&tmp);
    return cuda_check(ctx, ce, "vmap_insert: cudaDeviceSynchronize");
  }
  for (int l = 0; l < vm->levels; ++l) move_level(vm, &tmp, l);
  ++vm->version;
  vmap_bump_epoch();
  ctx->err.clear();
  return GLIM_OK;
}

extern "C" void glim_vmap_free(glim_vmap* vm) {
  if (!vm) return;
  vmap_unregister(vm);  // plans on this map refuse to launch from now on
  DeviceGuard device_guard;
  device_guard.set(vm->device);
  cudaDeviceSynchronize();  // launches on any stream may still read the tables
  free_levels(vm);
  delete vm;
}

extern "C" glim_status glim_vmap_info(const glim_vmap* vm, int32_t level, int64_t* n_voxels, int64_t* capacity,
                                      int32_t* max_probe) {
  if (!vm || level < 0 || level >= vm->levels) return GLIM_EINVAL;
  if (n_voxels) *n_voxels = vm->n_vox[level];
  if (capacity) *capacity = vm->dense[level] ? vm->cap[level] : vm->nblk[level] * GLIM_BLOCK_CELLS;
  if (max_probe) *max_probe = vm->max_probe[level];
  return GLIM_OK;
}

extern "C" glim_status glim_vmap_export(glim_ctx* ctx, const glim_vmap* vm, int32_t level, int32_t* keys3,
                                        float* mean3, float* cov6, int32_t* count) {
  if (!ctx || !vm || level < 0 || level >= vm->levels)
    return ctx ? set_error(ctx, GLIM_EINVAL, "vmap_export: bad level") : GLIM_EINVAL;
  const int64_t m = vm->n_vox[level];
  if (m == 0) return GLIM_OK;
  k_export<<<ceil_div_i(m, 256), 256, 0, ctx->stream>>>(vm->vkey[level], vm->vmean[level], vm->vcov[level],
                                                        vm->vcount[level], m, keys3, mean3, cov6, count);
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}

extern "C" glim_status glim_correspondences(glim_ctx* ctx, const glim_frame* src, const glim_vmap* tgt,
                                            const double* pose_s12, const double* pose_t12,
                                            int32_t validate_surface, int32_t* ids_out) {
  GLIM_RANGE("glim_correspondences");
  if (!ctx || !src || !tgt || !pose_s12 || !pose_t12 || (src->n > 0 && !ids_out))
    return ctx ? set_error(ctx, GLIM_EINVAL, "correspondences: null argument") : GLIM_EINVAL;
  if (src->n <= 0) return GLIM_OK;
  CorrArgs a;
  a.pts = reinterpret_cast<const float4*>(src->pts4);
  a.nrm = src->normal3;
  a.n = src->n;
  a.pose = pose_to_f32(relative_pose(pose_s12, pose_t12));
  a.levels = tgt->levels;
  for (int l = 0; l < tgt->levels; ++l) a.lv[l] = tgt->dev(l);
  a.validate = validate_surface;
  k_correspondences<<<ceil_div_i(src->n, 256), 256, 0, ctx->stream>>>(a, ids_out);
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}

extern "C" glim_status glim_overlap(glim_ctx* ctx, const glim_frame* frames, int32_t nframes, const glim_pair* pairs,
                                    int32_t npairs, const double* poses12, int32_t level, double* overlap_out) {
  GLIM_RANGE("glim_overlap");
  if (!ctx || !frames || !pairs || !poses12 || !overlap_out || npairs < 0)
    return ctx ? set_error(ctx, GLIM_EINVAL, "overlap: null argument") : GLIM_EINVAL;
  if (npairs == 0) return GLIM_OK;
  std::vector<OverlapPair> hp(npairs);
  for (int p = 0; p < npairs; ++p) {
    const glim_pair& q = pairs[p];
    if (q.src_frame < 0 || q.src_frame >= nframes || q.tgt_frame < 0 || q.tgt_frame >= nframes || !q.tgt ||
        level < 0 || level >= q.tgt->levels)
      return set_error(ctx, GLIM_EINVAL, "overlap: bad pair %d", p);
    hp[p].pts = reinterpret_cast<const float4*>(frames[q.src_frame].pts4);
    hp[p].n = frames[q.src_frame].n;
    hp[p].lv = q.tgt->dev(level);
    hp[p].pose = pose_to_f32(relative_pose(poses12 + 12 * q.src_frame, poses12 + 12 * q.tgt_frame));
  }
  DevBuf<OverlapPair> dp;
  GLIM_CUDA(ctx, dp.alloc(npairs, ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(dp.p, hp.data(), npairs * sizeof(OverlapPair), cudaMemcpyHostToDevice, ctx->stream));
  k_overlap<<<npairs, 256, 0, ctx->stream>>>(dp.p, overlap_out);
  GLIM_LAUNCHED(ctx);
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // hp must outlive the copy
  return GLIM_OK;
}

extern "C" int32_t glim_vmap_is_dense(const glim_vmap* vm, int32_t level) {
  if (!vm || level < 0 || level >= vm->levels) return -1;
  return vm->dense[level];
}
