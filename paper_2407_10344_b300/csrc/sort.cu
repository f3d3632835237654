// sort.cu -- device primitives of the voxel build: exclusive scan, stable LSD radix sort of
// (64-bit key, 32-bit value) pairs, and the sort of points into voxel cells.
//
// The voxelmap build sorts the points of a frame by voxel key so that every voxel's members
// are contiguous and in ascending point order; the voxel statistics are then summed in that
// fixed order, which makes the build deterministic run to run.
#include "common.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 2048 values per block

// Block-wide exclusive scan of one tile; writes the tile total to block_sums.
__global__ void k_scan_tile(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                            uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(tid) * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t run = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    uint32_t x = (i < n) ? in[i] : 0u;
    v[j] = run;  // exclusive within the thread
    run += x;
  }
  // inclusive warp scan of the thread totals
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == SCAN_THREADS / 32 - 1 && block_sums) block_sums[blockIdx.x] = ti;
  }
  __syncthreads();
  const uint32_t offset = warp_tot[warp] + (inc - run);
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    if (i < n) out[i] = v[j] + offset;
  }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ block_offs) {
  const int64_t i = int64_t(blockIdx.x) * SCAN_TILE + threadIdx.x;
  const uint32_t add = block_offs[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t k = i + int64_t(j) * SCAN_THREADS;
    if (k < n) out[k] += add;
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;  // one thread per digit value
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void k_radix_hist(const unsigned long long* __restrict__ keys, int64_t n, int shift,
                             uint32_t* __restrict__ counts, int nblocks) {
  __shared__ uint32_t h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    int64_t i = base + int64_t(j) * RS_THREADS + tid;
    if (i < n) atomicAdd(&h[uint32_t(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[int64_t(tid) * nblocks + blockIdx.x] = h[tid];  // digit-major
}

// Stable scatter: items are ranked in their original order within the block, sub-tile by
// sub-tile; within a sub-tile by warp, then by lane.
__global__ void k_radix_scatter(const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
                                unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout,
                                const uint32_t* __restrict__ offsets, int64_t n, int shift, int nblocks) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[RS_THREADS / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offsets[int64_t(tid) * nblocks + blockIdx.x];
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
  for (int it = 0; it < RS_ITEMS; ++it) {
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int64_t i = base + int64_t(it) * RS_THREADS + tid;
    const bool valid = i < n;
    unsigned long long key = valid ? kin[i] : 0ull;
    uint32_t val = valid ? vin[i] : 0u;
    uint32_t d = valid ? (uint32_t(key >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & ((1u << lane) - 1u));
    int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
      uint32_t pos = run[d] + pre + uint32_t(rank);
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) tot += wcnt[w][tid];
    run[tid] += tot;
    __syncthreads();
  }
}

__global__ void k_key_xor_or(const unsigned long long* __restrict__ keys, int64_t n,
                             unsigned long long* __restrict__ out) {
  __shared__ unsigned long long s[256];
  const unsigned long long k0 = keys[0];
  unsigned long long acc = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc |= keys[i] ^ k0;
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] |= s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicOr(out, s[0]);
}

// ---------------------------------------------------------------- points -> cells
__global__ void k_point_keys(const float4* __restrict__ pts, int64_t n, float inv_r,
                             unsigned long long* __restrict__ keys, uint32_t* __restrict__ idx,
                             unsigned int* __restrict__ status, int range_is_error) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 p = pts[i];
  idx[i] = uint32_t(i);
  if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w))) {
    atomicOr(status, GLIM_DS_NONFINITE);
    keys[i] = GLIM_EMPTY_KEY;
    return;
  }
  int kx, ky, kz;
  if (!voxel_coord(p.x, inv_r, kx) || !voxel_coord(p.y, inv_r, ky) || !voxel_coord(p.z, inv_r, kz)) {
    if (range_is_error) atomicOr(status, GLIM_DS_RANGE);
    keys[i] = GLIM_EMPTY_KEY;
    return;
  }
  keys[i] = pack_key(kx, ky, kz);
}

__global__ void k_heads(const unsigned long long* __restrict__ ks, int64_t n, uint32_t* __restrict__ head) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = (ks[i] != GLIM_EMPTY_KEY && (i == 0 || ks[i] != ks[i - 1])) ? 1u : 0u;
}

// cell_start[c] = first sorted position of cell c; cell_key[c] = its key
__global__ void k_cell_starts(const unsigned long long* __restrict__ ks, const uint32_t* __restrict__ head_excl,
                              int64_t n, uint32_t* __restrict__ cell_start, unsigned long long* __restrict__ cell_key) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long k = ks[i];
  if (k != GLIM_EMPTY_KEY && (i == 0 || k != ks[i - 1])) {
    cell_start[head_excl[i]] = uint32_t(i);
    cell_key[head_excl[i]] = k;
  }
}

// the end of the last cell: the first EMPTY key (empty keys sort last) or n
__global__ void k_cell_end(const unsigned long long* __restrict__ ks, int64_t n, uint32_t* __restrict__ cell_start,
                           uint32_t m) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (ks[i] == GLIM_EMPTY_KEY && (i == 0 || ks[i - 1] != GLIM_EMPTY_KEY)) cell_start[m] = uint32_t(i);
  if (i == n - 1 && ks[i] != GLIM_EMPTY_KEY) cell_start[m] = uint32_t(n);
}

// spread the low 21 bits of v so that bit i moves to bit 3 i (Morton interleave)
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1FFFFFull;
  v = (v | (v << 32)) & 0x1F00000000FFFFull;
  v = (v | (v << 16)) & 0x1F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__global__ void k_morton_keys(const float4* __restrict__ pts, int64_t n, float inv_cell,
                              unsigned long long* __restrict__ keys, uint32_t* __restrict__ idx,
                              unsigned int* __restrict__ status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = pts[i];
  idx[i] = uint32_t(i);
  int kx, ky, kz;
  if (!voxel_coord(p.x, inv_cell, kx) || !voxel_coord(p.y, inv_cell, ky) || !voxel_coord(p.z, inv_cell, kz)) {
    atomicOr(status, isfinite(p.x) && isfinite(p.y) && isfinite(p.z) ? GLIM_DS_RANGE : GLIM_DS_NONFINITE);
    keys[i] = 0;
    return;
  }
  keys[i] = (spread3(unsigned(kx + GLIM_KEY_BIAS)) << 2) | (spread3(unsigned(ky + GLIM_KEY_BIAS)) << 1) |
            spread3(unsigned(kz + GLIM_KEY_BIAS));
}

}  // namespace

extern "C" glim_status glim_spatial_order(glim_ctx* ctx, const float* pts4, int64_t n, float cell,
                                          int32_t* perm_out) {
  GLIM_RANGE("glim_spatial_order");
  if (!ctx) return GLIM_EINVAL;
  if (n < 0 || n > 0x7FFFFFFFll || !(cell > 0.f) || (n > 0 && (!pts4 || !perm_out)))
    return set_error(ctx, GLIM_EINVAL, "spatial_order: bad arguments");
  if (reinterpret_cast<uintptr_t>(pts4) & 15) return set_error(ctx, GLIM_EINVAL, "spatial_order: pts4 misaligned");
  if (n == 0) return GLIM_OK;
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  DevBuf<unsigned long long> keys, ks;
  DevBuf<uint32_t> idx;
  GLIM_CUDA(ctx, keys.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, ks.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, idx.alloc(n, ctx->stream));
  k_morton_keys<<<ceil_div_i(n, 256), 256, 0, ctx->stream>>>(reinterpret_cast<const float4*>(pts4), n,
                                                            float(1.0 / double(cell)), keys.p, idx.p, ctx->d_status);
  GLIM_LAUNCHED(ctx);
  glim_status st = take_device_status(ctx, "spatial_order");
  if (st != GLIM_OK) return st;
  unsigned long long varying = 0;
  st = key_varying_bits(ctx, keys.p, n, &varying);
  if (st != GLIM_OK) return st;
  st = radix_sort_pairs(ctx, keys.p, idx.p, ks.p, reinterpret_cast<uint32_t*>(perm_out), n, varying);
  if (st != GLIM_OK) return st;
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->err.clear();
  return GLIM_OK;
}

glim_status scan_exclusive_u32(glim_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n) {
  if (n <= 0) return GLIM_OK;
  const int nb = ceil_div_i(n, SCAN_TILE);
  if (nb == 1) {
    k_scan_tile<<<1, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, nullptr);
    GLIM_LAUNCHED(ctx);
    return GLIM_OK;
  }
  DevBuf<uint32_t> sums;
  GLIM_CUDA(ctx, sums.alloc(nb, ctx->stream));
  k_scan_tile<<<nb, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, sums.p);
  GLIM_LAUNCHED(ctx);
  glim_status st = scan_exclusive_u32(ctx, sums.p, sums.p, nb);
  if (st != GLIM_OK) return st;
  k_scan_add<<<nb, SCAN_THREADS, 0, ctx->stream>>>(out, n, sums.p);
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}

glim_status key_varying_bits(glim_ctx* ctx, const unsigned long long* keys, int64_t n,
                             unsigned long long* varying_host) {
  *varying_host = 0;
  if (n <= 1) return GLIM_OK;
  DevBuf<unsigned long long> acc;
  GLIM_CUDA(ctx, acc.alloc(1, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), ctx->stream));
  int grid = std::min(ceil_div_i(n, 256), 4 * ctx->num_sms);
  k_key_xor_or<<<grid, 256, 0, ctx->stream>>>(keys, n, acc.p);
  GLIM_LAUNCHED(ctx);
  GLIM_CUDA(ctx, cudaMemcpyAsync(varying_host, acc.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return GLIM_OK;
}

glim_status radix_sort_pairs(glim_ctx* ctx, const unsigned long long* keys_in, const uint32_t* vals_in,
                             unsigned long long* keys_out, uint32_t* vals_out, int64_t n,
                             unsigned long long varying) {
  if (n <= 0) return GLIM_OK;
  if (n > 0x7FFFFFFFll) return set_error(ctx, GLIM_EINVAL, "radix sort: n = %lld too large", (long long)n);
  std::vector<int> shifts;
  for (int s = 0; s < 64; s += 8)
    if ((varying >> s) & 0xFFull) shifts.push_back(s);
  if (shifts.empty()) {
    GLIM_CUDA(ctx, cudaMemcpyAsync(keys_out, keys_in, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, ctx->stream));
    GLIM_CUDA(ctx, cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    return GLIM_OK;
  }
  const int nb = ceil_div_i(n, RS_TILE);
  DevBuf<uint32_t> counts;
  DevBuf<unsigned long long> kt;
  DevBuf<uint32_t> vt;
  GLIM_CUDA(ctx, counts.alloc(size_t(256) * nb, ctx->stream));
  GLIM_CUDA(ctx, kt.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, vt.alloc(n, ctx->stream));
  // ping-pong so that the last pass lands in keys_out
  const int passes = int(shifts.size());
  const unsigned long long* ksrc = keys_in;
  const uint32_t* vsrc = vals_in;
  for (int p = 0; p < passes; ++p) {
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    unsigned long long* kdst = to_out ? keys_out : kt.p;
    uint32_t* vdst = to_out ? vals_out : vt.p;
    k_radix_hist<<<nb, RS_THREADS, 0, ctx->stream>>>(ksrc, n, shifts[p], counts.p, nb);
    GLIM_LAUNCHED(ctx);
    glim_status st = scan_exclusive_u32(ctx, counts.p, counts.p, int64_t(256) * nb);
    if (st != GLIM_OK) return st;
    k_radix_scatter<<<nb, RS_THREADS, 0, ctx->stream>>>(ksrc, vsrc, kdst, vdst, counts.p, n, shifts[p], nb);
    GLIM_LAUNCHED(ctx);
    ksrc = kdst;
    vsrc = vdst;
  }
  return GLIM_OK;
}

glim_status sort_into_cells(glim_ctx* ctx, const float* pts4, int64_t n, float inv_r, SortedCells& out,
                            bool range_is_error) {
  out.m = 0;
  if (n <= 0) return GLIM_OK;
  DevBuf<unsigned long long> keys;
  DevBuf<uint32_t> idx;
  GLIM_CUDA(ctx, keys.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, idx.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, out.key_sorted.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, out.idx_sorted.alloc(n, ctx->stream));
  k_point_keys<<<ceil_div_i(n, 256), 256, 0, ctx->stream>>>(reinterpret_cast<const float4*>(pts4), n, inv_r,
                                                            keys.p, idx.p, ctx->d_status, range_is_error ? 1 : 0);
  GLIM_LAUNCHED(ctx);
  unsigned long long varying = 0;
  glim_status st = key_varying_bits(ctx, keys.p, n, &varying);
  if (st != GLIM_OK) return st;
  st = radix_sort_pairs(ctx, keys.p, idx.p, out.key_sorted.p, out.idx_sorted.p, n, varying);
  if (st != GLIM_OK) return st;
  return segment_sorted(ctx, out.key_sorted.p, n, out);
}

glim_status segment_sorted(glim_ctx* ctx, const unsigned long long* key_sorted, int64_t n, SortedCells& out) {
  out.m = 0;
  if (n <= 0) return GLIM_OK;
  glim_status st = GLIM_OK;
  DevBuf<uint32_t> head;
  GLIM_CUDA(ctx, head.alloc(n + 1, ctx->stream));
  k_heads<<<ceil_div_i(n, 256), 256, 0, ctx->stream>>>(key_sorted, n, head.p);
  GLIM_LAUNCHED(ctx);
  GLIM_CUDA(ctx, cudaMemsetAsync(head.p + n, 0, sizeof(uint32_t), ctx->stream));
  st = scan_exclusive_u32(ctx, head.p, head.p, n + 1);
  if (st != GLIM_OK) return st;
  uint32_t m = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&m, head.p + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out.m = m;
  GLIM_CUDA(ctx, out.cell_start.alloc(size_t(m) + 1, ctx->stream));
  GLIM_CUDA(ctx, out.cell_key.alloc(m > 0 ? m : 1, ctx->stream));
  if (m == 0) {
    GLIM_CUDA(ctx, cudaMemsetAsync(out.cell_start.p, 0, sizeof(uint32_t), ctx->stream));
    return GLIM_OK;
  }
  k_cell_starts<<<ceil_div_i(n, 256), 256, 0, ctx->stream>>>(key_sorted, head.p, n, out.cell_start.p,
                                                             out.cell_key.p);
  GLIM_LAUNCHED(ctx);
  k_cell_end<<<ceil_div_i(n, 256), 256, 0, ctx->stream>>>(key_sorted, n, out.cell_start.p, m);
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}
