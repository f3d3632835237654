// lookup.cuh -- device side of the voxel correspondence (Sec. III-C "Correspondence search"):
// FP32 transform of a source point, surface-orientation test, voxel key and hash probe.
#pragma once
#include "common.cuh"

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// q = R mu + t on the FP32 path: one fused multiply-add per term, starting from t and adding
// the x, y, z terms in that order (R row-major).
__device__ __forceinline__ float3 transform_pinned(const float* R, const float* t, float mx, float my, float mz) {
  float3 q;
  q.x = __fmaf_rn(R[2], mz, __fmaf_rn(R[1], my, __fmaf_rn(R[0], mx, t[0])));
  q.y = __fmaf_rn(R[5], mz, __fmaf_rn(R[4], my, __fmaf_rn(R[3], mx, t[1])));
  q.z = __fmaf_rn(R[8], mz, __fmaf_rn(R[7], my, __fmaf_rn(R[6], mx, t[2])));
  return q;
}

// Surface-orientation test: true when the target viewpoint v lies behind the point's surface,
// (mu - v) . n > 0, evaluated as s = n_x d_x; s = fma(n_y, d_y, s); s = fma(n_z, d_z, s).
__device__ __forceinline__ bool behind_surface(float mx, float my, float mz, const float* v, float nx, float ny,
                                               float nz) {
  float dx = __fsub_rn(mx, v[0]), dy = __fsub_rn(my, v[1]), dz = __fsub_rn(mz, v[2]);
  float s = __fmul_rn(nx, dx);
  s = __fmaf_rn(ny, dy, s);
  s = __fmaf_rn(nz, dz, s);
  return s > 0.0f;
}

// floor(c * inv_r) with one round-to-nearest FP32 multiply; false (a miss) when the product
// is outside [-2^20, 2^20) or not a number.  Then floor(product) lies in the same range and
// the conversion rounding down is exact.
__device__ __forceinline__ bool key_coord(float c, float inv_r, int& k) {
  const float p = __fmul_rn(c, inv_r);
  k = __float2int_rd(p);
  return p >= -1048576.0f && p < 1048576.0f;
}

__device__ __forceinline__ bool level_key3(const float3& q, float inv_r, int& kx, int& ky, int& kz) {
  const bool a = key_coord(q.x, inv_r, kx);
  const bool b = key_coord(q.y, inv_r, ky);
  const bool c = key_coord(q.z, inv_r, kz);
  return a && b && c;
}

__device__ __forceinline__ int4 ldg4i(const int4* p) { return __ldg(p); }

// Cell of key (kx, ky, kz) in a hashed level, or -1: the block key's entry is looked up by a
// linear probe from slot h, bounded by the table's longest probe sequence.
__device__ __forceinline__ int block_cell_from(const LevelDev& L, int kx, int ky, int kz, uint32_t h, int first) {
  const int bx = kx >> GLIM_BLOCK_SHIFT, by = ky >> GLIM_BLOCK_SHIFT, bz = kz >> GLIM_BLOCK_SHIFT;
  for (int p = first; p < L.max_probe; ++p) {
    const int4 e = ldg4i(&L.btab[h]);
    if (e.x == bx && e.y == by && e.z == bz) return e.w * GLIM_BLOCK_CELLS + block_local(kx, ky, kz);
    if (e.x == GLIM_EMPTY_COORD) return -1;
    h = (h + 1u) & L.mask;
  }
  return -1;
}

__device__ __forceinline__ uint32_t block_hash(int kx, int ky, int kz, int log2cap) {
  return hash3(kx >> GLIM_BLOCK_SHIFT, ky >> GLIM_BLOCK_SHIFT, kz >> GLIM_BLOCK_SHIFT, log2cap);
}

__device__ __forceinline__ int block_cell(const LevelDev& L, int kx, int ky, int kz) {
  return block_cell_from(L, kx, ky, kz, block_hash(kx, ky, kz, L.log2cap), 0);
}

// Dense grid cell of key (kx, ky, kz), or -1 outside the grid (grids have < 2^31 cells).
__device__ __forceinline__ int64_t dense_cell(const LevelDev& L, int kx, int ky, int kz) {
  const uint32_t x = uint32_t(kx - L.ox), y = uint32_t(ky - L.oy), z = uint32_t(kz - L.oz);
  if (x >= L.nx || y >= L.ny || z >= L.nz) return -1;
  return int64_t((x * L.ny + y) * L.nz + z);
}

// Keys of every level of a map whose resolutions are r_0 2^l (Sec. III-C): the level-0 product
// p = q * inv_r_0 (one FP32 multiply per axis, as on every level) gives floor(p 2^-l) =
// floor(p) >> l exactly, because inv_r_l = inv_r_0 2^-l scales the product by a power of two.
// Valid while |p| < 2^20 on every axis and no product is so small (below 2^-100 but not
// zero) that its scaled copy could become subnormal; otherwise false and the caller computes
// each level.
__device__ __forceinline__ bool level0_ok(float p) {
  const float m = fabsf(p);
  return m < 1048576.0f && (m >= 7.8886091e-31f || m == 0.0f);  // 2^-100
}

__device__ __forceinline__ bool level0_key3(const float3& q, float inv_r0, int& kx, int& ky, int& kz) {
  const float px = __fmul_rn(q.x, inv_r0), py = __fmul_rn(q.y, inv_r0), pz = __fmul_rn(q.z, inv_r0);
  kx = __float2int_rd(px);
  ky = __float2int_rd(py);
  kz = __float2int_rd(pz);
  return level0_ok(px) && level0_ok(py) && level0_ok(pz);
}

// Voxel of key (kx, ky, kz) at a level: the index of its record in L.slots (a grid cell or a
// block cell) or -1, and the canonical id through *id.
__device__ __forceinline__ int find_voxel(const LevelDev& L, int kx, int ky, int kz, int* id) {
  const int64_t c = L.dense ? dense_cell(L, kx, ky, kz) : int64_t(block_cell(L, kx, ky, kz));
  const int v = c < 0 ? -1 : __float_as_int(ldg4(&L.slots[c].w0).x);
  *id = v < 0 ? -1 : v;
  return v < 0 ? -1 : int(c);
}
