// lane_hash.cuh -- the per-lane rounds of the linearization on hashed voxel blocks (Sec. III-C
// "Correspondence search": the voxel of a transformed point found through a hash table).
// Included by lin_kernel.cuh after the per-point arithmetic (lane_levels, lane_gform).
//
// A lookup on a hashed level takes two dependent reads: the table entry of the point's voxel
// block, then the cell record.  The rounds are a three-stage software pipeline: a point's
// coordinates are read two rounds ahead; its covariance and the table entries of every level
// one round ahead (hash_fetch); its records are read (hash_resolve) between the previous
// point's level arithmetic and that point's G-form, so the G-form, the next point's fetch
// and the point's own R C R^T cover the records' latency.  Against reading the records at
// the start of the point's own round: 8.12 against 8.27 ms on the urban step.
#pragma once

// What a lane holds between the two lookup stages of a point on hashed levels:
template <int LMAX>
struct HashFetch {
  float3 q;
  float w;
  bool live;
  float2 ca, cb, cc;
  int kx[LMAX], ky[LMAX], kz[LMAX];  // keys of each level (holding the block keys and the
                                     // cells inside the blocks instead measured 2 % slower)
  int4 e[LMAX];  // the table entry at each level's home slot, {bx, by, bz, block}
  int idx;       // IDS: index of the point in its frame, -1 for a masked lane
};

// First stage: transform, the keys of every level and the home-slot table entries of every
// level's block, all in flight together; descriptor {slots, btab} {mask, log2cap, max_probe, pad}.
template <int LMAX, bool IDS>
__device__ __forceinline__ void hash_fetch(const HashView& V, const float4 m, bool live, int validate, int kk,
                                           HashFetch<LMAX>& H) {
  if constexpr (IDS) H.idx = live ? kk : -1;
  const float3 q = lane_transform(V, m, live, validate, kk, H.ca, H.cb, H.cc);
  // level-0 keys, shifted on the coarser levels (resolutions doubling per level, as in lane_fetch)
  const int k0x = __float2int_rd(__fmul_rn(q.x, V.M.inv_r[0]));
  const int k0y = __float2int_rd(__fmul_rn(q.y, V.M.inv_r[0]));
  const int k0z = __float2int_rd(__fmul_rn(q.z, V.M.inv_r[0]));
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const int kx = k0x >> l, ky = k0y >> l, kz = k0z >> l;
    H.kx[l] = kx;
    H.ky[l] = ky;
    H.kz[l] = kz;
    const int4 la = reinterpret_cast<const int4*>(&V.M.lv[l])[0];
    const int4 lb = reinterpret_cast<const int4*>(&V.M.lv[l])[1];
    const int4* btab = reinterpret_cast<const int4*>(uint64_t(uint32_t(la.z)) | (uint64_t(uint32_t(la.w)) << 32));
    H.e[l] = ldg4i(btab + hash3(kx >> GLIM_BLOCK_SHIFT, ky >> GLIM_BLOCK_SHIFT, kz >> GLIM_BLOCK_SHIFT, lb.y));
  }
  H.q = q;
  H.w = m.w;
  H.live = live;
}

// Second stage: per level the lanes whose home entry holds another block continue the probe
// (a warp-uniform branch skips it when no lane needs it), bounded by the table's longest
// probe sequence; then the records of every level, read as on a dense grid (cell -1 is the
// empty record before cell 0).
template <int LMAX, bool IDS>
__device__ __forceinline__ void hash_resolve(const HashView& V, HashFetch<LMAX>& H, LaneFetch<LMAX>& F) {
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const int bx = H.kx[l] >> GLIM_BLOCK_SHIFT, by = H.ky[l] >> GLIM_BLOCK_SHIFT, bz = H.kz[l] >> GLIM_BLOCK_SHIFT;
    int4 e = H.e[l];
    bool match = e.x == bx && e.y == by && e.z == bz;
    const bool more = H.live && !match && e.x != GLIM_EMPTY_COORD;
    const int4 la = reinterpret_cast<const int4*>(&V.M.lv[l])[0];
    if (__any_sync(0xffffffffu, more)) {
      if (more) {
        const int4 lb = reinterpret_cast<const int4*>(&V.M.lv[l])[1];
        const int4* btab = reinterpret_cast<const int4*>(uint64_t(uint32_t(la.z)) | (uint64_t(uint32_t(la.w)) << 32));
        uint32_t hh = hash3(bx, by, bz, lb.y);
        for (int p = 1; p < lb.z; ++p) {
          hh = (hh + 1u) & uint32_t(lb.x);
          e = ldg4i(btab + hh);
          match = e.x == bx && e.y == by && e.z == bz;
          if (match || e.x == GLIM_EMPTY_COORD) break;
        }
      }
    }
    const int cell = (H.live && match) ? e.w * GLIM_BLOCK_CELLS + block_local(H.kx[l], H.ky[l], H.kz[l]) : -1;
    const VoxSlot* sl =
        reinterpret_cast<const VoxSlot*>(uint64_t(uint32_t(la.x)) | (uint64_t(uint32_t(la.y)) << 32)) + cell;
    const float2 h2 = __ldg(reinterpret_cast<const float2*>(&sl->w0));
    F.s0[l] = make_float4(h2.x, h2.y, 0.f, 0.f);
    F.s1[l] = ldg4(&sl->w1);  // {mean, C~00}
    F.s2[l] = ldg4(&sl->w2);  // {C~01, C~02, C~11, C~12}
  }
  F.q = H.q;
  F.w = H.w;
  F.live = H.live;
  F.ca = H.ca;
  F.cb = H.cb;
  F.cc = H.cc;
  if constexpr (IDS) F.idx = H.idx;
}

// The rounds of one work item on hashed levels (see the top of this file).  The buffers
// alternate by unrolling twice; a point past the end of the tile is read as the tile's last
// point and masked, as on dense grids.
template <int BLOCK, int LMAX, bool IDS, class A>
__device__ __forceinline__ void hash_rounds(const HashView& V, int validate, int first, int last, int rounds, A& acc,
                                            int& inl, int32_t* ids, int idl) {
  HashFetch<LMAX> ha, hb;
  LaneFetch<LMAX> f0, f1;
  LaneSums S;
  hash_fetch<LMAX, IDS>(V, ldg4(V.pts + min(first, last)), first <= last, validate, min(first, last), ha);
  float4 pn = ldg4(V.pts + min(first + BLOCK, last));
  hash_resolve<LMAX, IDS>(V, ha, f0);
  hash_fetch<LMAX, IDS>(V, pn, first + BLOCK <= last, validate, min(first + BLOCK, last), hb);
  pn = ldg4(V.pts + min(first + 2 * BLOCK, last));
  int j = 0;
#pragma unroll 1
  for (; j + 1 < rounds; j += 2) {
    const int k = first + j * BLOCK;
    // point j: its level arithmetic, the records of point j + 1, its G-form, the fetch of j + 2
    lane_levels<LMAX, true, IDS>(V, f0, S, inl, ids, idl);
    hash_resolve<LMAX, IDS>(V, hb, f1);
    lane_gform(S, acc);
    hash_fetch<LMAX, IDS>(V, pn, k + 2 * BLOCK <= last, validate, min(k + 2 * BLOCK, last), ha);
    pn = ldg4(V.pts + min(k + 3 * BLOCK, last));
    // point j + 1, the same with the buffers swapped
    lane_levels<LMAX, true, IDS>(V, f1, S, inl, ids, idl);
    hash_resolve<LMAX, IDS>(V, ha, f0);
    lane_gform(S, acc);
    hash_fetch<LMAX, IDS>(V, pn, k + 3 * BLOCK <= last, validate, min(k + 3 * BLOCK, last), hb);
    pn = ldg4(V.pts + min(k + 4 * BLOCK, last));
  }
  if (j < rounds) {
    lane_levels<LMAX, true, IDS>(V, f0, S, inl, ids, idl);
    lane_gform(S, acc);
  }
}
