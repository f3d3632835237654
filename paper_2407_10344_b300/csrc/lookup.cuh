// lookup.cuh -- device side of the voxel correspondence (Sec. III-C "Correspondence search"):
// FP32 transform of a source point, surface-orientation test, voxel key and hash probe.
#pragma once
#include "common.cuh"

// Read-only loads through the non-coherent path; the voxel tables and source frames are not
// written while a linearization kernel runs.
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

__device__ __forceinline__ unsigned long long slot_key(const float4& w0) {
  return (unsigned long long)__float_as_uint(w0.x) | ((unsigned long long)__float_as_uint(w0.y) << 32);
}

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

// Packed voxel key of q at a level, or false when a component is outside [-2^20, 2^20).
__device__ __forceinline__ bool level_key(const float3& q, float inv_r, unsigned long long& key) {
  int kx, ky, kz;
  if (!voxel_coord(q.x, inv_r, kx) || !voxel_coord(q.y, inv_r, ky) || !voxel_coord(q.z, inv_r, kz)) return false;
  key = pack_key(kx, ky, kz);
  return true;
}

// Linear probe for `key`; returns the slot index or -1.  The loop is bounded by the longest
// probe sequence recorded when the table was built.
__device__ __forceinline__ int probe_slot(const LevelDev& L, unsigned long long key) {
  uint32_t h = hash_slot(key, L.log2cap);
  for (int p = 0; p < L.max_probe; ++p) {
    const float4 w0 = ldg4(&L.slots[h].w0);
    const unsigned long long k = slot_key(w0);
    if (k == key) return int(h);
    if (k == GLIM_EMPTY_KEY) return -1;
    h = (h + 1u) & L.mask;
  }
  return -1;
}
