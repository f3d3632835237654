// lin_kernel.cuh -- the linearization kernel (Sec. III-C "Linearization"): per-point FP32
// work, per-item block reduction, persistent work queue.  Instantiated per accumulation mode
// in lin_fp32.cu, lin_kahan.cu and lin_fp64.cu.
//
// Per point (FP32): the pinned transform q = R mu + t, u = R mu, the rotated covariance
// R C R^T once for all levels; the lookup of every level (a dense grid's cell, or a hashed
// level's block-table entry then the cell) with the reads of all levels in flight together,
// then per hit S = C~ + R C R^T, Omega = S^-1 (adjugate / determinant), d = mu~ - q,
// y = Omega d, e = d^T y, summed over levels as Omega_sum = sum w Omega, g_sum = sum w y, e_sum.
//
// With G = [-(u)x, I] (3 x 6), the same for every level of a point, A_k = -G diag(R, R) and
// B_k = G S_t (S_t = [[I, 0], [-(t)x, I]]), Eqs. (4)-(5).  A point therefore contributes
// M += G^T Omega_sum G (21 unique entries: -u x Omega u x, u x Omega, Omega), g += G^T g_sum
// ([u x g_sum; g_sum]) and e += e_sum: 28 accumulators, expanded once per pair into
// H = Lift^T M Lift and b = Lift^T g with Lift = [-diag(R, R), S_t].
#pragma once
#include <cstddef>
#include <type_traits>

#include "plan.cuh"

namespace glim_detail {

// ---------------------------------------------------------------- accumulation policies
struct AccPlain {  // plain FP32 running sums
  float s[NACC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NACC; ++i) s[i] = 0.f;
  }
  __device__ __forceinline__ void add(int i, float x) { s[i] += x; }
  // s += a b + c d, fused into the running sum
  __device__ __forceinline__ void add2(int i, float a, float b, float c, float d) {
    s[i] = __fmaf_rn(a, b, __fmaf_rn(c, d, s[i]));
  }
};

// Neumaier-compensated FP32 running sums (Neumaier 1974): c collects the rounding error of
// every addition.
struct AccComp {
  float s[NACC], c[NACC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NACC; ++i) s[i] = c[i] = 0.f;
  }
  __device__ __forceinline__ void add(int i, float x) {
    const float t = s[i] + x;
    c[i] += (fabsf(s[i]) >= fabsf(x)) ? ((s[i] - t) + x) : ((x - t) + s[i]);
    s[i] = t;
  }
  __device__ __forceinline__ void add2(int i, float a, float b, float c, float d) {
    add(i, __fmaf_rn(a, b, c * d));
  }
};

template <int ACC>
struct AccOf {
  using type = AccPlain;
};
template <>
struct AccOf<GLIM_ACC_KAHAN> {
  using type = AccComp;
};

// ---------------------------------------------------------------- per-point term
struct PointIn {
  float4 m;
  float2 ca, cb, cc;
};

__device__ __forceinline__ PointIn load_point(const FrameDev& F, int64_t k) {
  PointIn p;
  p.m = ldg4(&F.pts[k]);
  p.ca = __ldg(&F.cov[3 * k]);
  p.cb = __ldg(&F.cov[3 * k + 1]);
  p.cc = __ldg(&F.cov[3 * k + 2]);
  return p;
}

// Phase 2 of one term record {S00, S01, S02, S11} {S12, S22, d.x, d.y} {d.z, u.x, u.y, u.z} of a
// point of weight w: w Omega = w adj(S)/det(S), y = w Omega d, e = d^T y, and the G-form
// contribution [G^T (w Omega) G, G^T y, e] with G = [-(u)x, I].  A term whose S is not positive
// definite contributes nothing and is no inlier (the return value is false).
template <class A>
__device__ __forceinline__ bool accumulate_term(const float4 t0, const float4 t1, const float4 t2, float w, A& acc) {
  const float a = t0.x, b = t0.y, c = t0.z, d = t0.w, e = t1.x, f = t1.y;  // S
  const float A00 = d * f - e * e, A01 = c * e - b * f, A02 = b * e - c * d;
  const float A11 = a * f - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
  const float det = a * A00 + b * A01 + c * A02;
  if (!(det > 0.f) || !(det < INFINITY)) return false;
  const float id = __fdividef(w, det);
  const float o00 = A00 * id, o01 = A01 * id, o02 = A02 * id, o11 = A11 * id, o12 = A12 * id, o22 = A22 * id;
  const float dx = t1.z, dy = t1.w, dz = t2.x;
  const float g0 = o00 * dx + o01 * dy + o02 * dz;  // w Omega d
  const float g1 = o01 * dx + o11 * dy + o12 * dz;
  const float g2 = o02 * dx + o12 * dy + o22 * dz;
  const float ux = t2.y, uy = t2.z, uz = t2.w;
  // W = (u)x (w Omega)
  const float W00 = -uz * o01 + uy * o02, W01 = -uz * o11 + uy * o12, W02 = -uz * o12 + uy * o22;
  const float W10 = uz * o00 - ux * o02, W11 = uz * o01 - ux * o12, W12 = uz * o02 - ux * o22;
  const float W20 = -uy * o00 + ux * o01, W21 = -uy * o01 + ux * o11, W22 = -uy * o02 + ux * o12;
  // M_rr = -(u)x Omega (u)x = W (u)x^T  (symmetric)
  acc.add2(0, -uz, W01, uy, W02);
  acc.add2(1, uz, W00, -ux, W02);
  acc.add2(2, -uy, W00, ux, W01);
  acc.add2(3, uz, W10, -ux, W12);
  acc.add2(4, -uy, W10, ux, W11);
  acc.add2(5, -uy, W20, ux, W21);
  // M_rt = (u)x Omega
  acc.add(6, W00); acc.add(7, W01); acc.add(8, W02);
  acc.add(9, W10); acc.add(10, W11); acc.add(11, W12);
  acc.add(12, W20); acc.add(13, W21); acc.add(14, W22);
  // M_tt = Omega
  acc.add(15, o00); acc.add(16, o01); acc.add(17, o02); acc.add(18, o11); acc.add(19, o12); acc.add(20, o22);
  // g = [u x (w Omega d); w Omega d]
  acc.add2(21, uy, g2, -uz, g1);
  acc.add2(22, uz, g0, -ux, g2);
  acc.add2(23, ux, g1, -uy, g0);
  acc.add(24, g0); acc.add(25, g1); acc.add(26, g2);
  acc.add(27, dx * g0 + dy * g1 + dz * g2);  // w d^T Omega d
  return true;
}

// Per-warp staging of one round: the compacted list of (point, level) hits.  A term record is
// three float4 (48 bytes) and the point's weight, self-contained, so phase 2 reads only its
// own record and lanes reading consecutive records touch distinct banks:
//   {S00, S01, S02, S11} {S12, S22, d.x, d.y} {d.z, u.x, u.y, u.z},  w
// with S = C~ + R C R^T, d = mu~ - q, u = R mu.
template <int LMAX>
struct WarpStage {
  float4 term[32 * LMAX * 3];
  float w[32 * LMAX];
};

// One round for the warp.  Phase 1 (every lane, its own point): transform, keys and one read
// of every level in flight together (collision fallback for hash levels), R C R^T, then each
// hit's record is written to the warp's term list at its compacted position (level-major,
// lane order within a level).  Phase 2 (the lanes share the term list): per hit
// w Omega = adj(S')/det(S'), y = w Omega d, e = d^T y, and the G-form contribution
// [G^T (w Omega) G, G^T y, e] with G = [-(u)x, I].  Misses and discarded points cost no
// phase-2 lanes.  With IDS (the id-recording instantiation) a real point (live on entry)
// also writes the canonical id of the voxel each level resolved to, or -1, to ids[k idl + l].
template <int LMAX, bool IDS, class A>
__device__ __forceinline__ void warp_round(const PairView& P, const PointIn& in, bool live, int64_t k, int validate,
                                           WarpStage<LMAX>& ws, A& acc, int& inl, int32_t* ids, int idl) {
  const int lane = threadIdx.x & 31;
  const bool real = live;
  const unsigned lt = (1u << lane) - 1u;
  const float4 m = in.m;
  if (live && validate && P.F.nrm) {
    const float* nk = P.F.nrm + 3 * k;
    live = !behind_surface(m.x, m.y, m.z, P.v, __ldg(nk), __ldg(nk + 1), __ldg(nk + 2));
  }
  const float* R = P.R;
  const float3 q = transform_pinned(R, P.t, m.x, m.y, m.z);

  int kx[LMAX], ky[LMAX], kz[LMAX];
  bool hit[LMAX];
  uint32_t hh[LMAX];  // hashed level: first probe of the block table
  int4 be[LMAX];      // hashed level: that entry
  int64_t cell[LMAX];
  float4 s0[LMAX], s1[LMAX], s2[LMAX];
  // keys: shifts of the level-0 key when the resolutions double per level, else per level
  int k0x, k0y, k0z;
  const bool shifted = P.M.pow2 && level0_key3(q, P.M.lv[0].inv_r, k0x, k0y, k0z);
  // first reads of every level in flight together: a dense level's cell index is known from
  // its key, a hashed level reads its block's table entry
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const LevelDev& L = P.M.lv[l];
    if (shifted) {
      kx[l] = k0x >> l;
      ky[l] = k0y >> l;
      kz[l] = k0z >> l;
      hit[l] = live && (l < P.M.levels);
    } else {
      hit[l] = live && (l < P.M.levels) && level_key3(q, L.inv_r, kx[l], ky[l], kz[l]);
    }
    cell[l] = -1;
    if (hit[l]) {
      if (L.dense) {
        cell[l] = dense_cell(L, kx[l], ky[l], kz[l]);
      } else {
        hh[l] = block_hash(kx[l], ky[l], kz[l], L.log2cap);
        be[l] = ldg4i(&L.btab[hh[l]]);
      }
    }
  }
  // hashed levels: the entry of the block, or a bounded continuation of the probe
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const LevelDev& L = P.M.lv[l];
    if (hit[l] && !L.dense) {
      const int bx = kx[l] >> GLIM_BLOCK_SHIFT, by = ky[l] >> GLIM_BLOCK_SHIFT, bz = kz[l] >> GLIM_BLOCK_SHIFT;
      if (be[l].x == bx && be[l].y == by && be[l].z == bz)
        cell[l] = int64_t(be[l].w) * GLIM_BLOCK_CELLS + block_local(kx[l], ky[l], kz[l]);
      else if (be[l].x != GLIM_EMPTY_COORD)
        cell[l] = block_cell_from(L, kx[l], ky[l], kz[l], (hh[l] + 1u) & L.mask, 1);
    }
  }
  // the records of every level in flight together
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    hit[l] = cell[l] >= 0;
    if (hit[l]) {
      const VoxSlot* sl = P.M.lv[l].slots + cell[l];
      s0[l] = ldg4(&sl->w0);
      s1[l] = ldg4(&sl->w1);
      s2[l] = ldg4(&sl->w2);
    }
  }
  int nh = 0;
  int vid[LMAX];  // IDS: canonical id of the voxel a level resolved to
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    vid[l] = -1;
    if (hit[l]) {
      hit[l] = __float_as_int(s0[l].x) >= 0;  // occupied cell (its record starts with the id)
      if constexpr (IDS) vid[l] = __float_as_int(s0[l].x);
    }
    nh += hit[l] ? 1 : 0;
  }
  if constexpr (IDS) {
    if (real) {
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l < idl) ids[k * idl + l] = hit[l] ? vid[l] : -1;
    }
  }
  // R C R^T and u, for the records of this lane's hits
  float r00 = 0.f, r01 = 0.f, r02 = 0.f, r11 = 0.f, r12 = 0.f, r22 = 0.f;
  if (nh > 0) {
    const float c00 = in.ca.x, c01 = in.ca.y, c02 = in.cb.x, c11 = in.cb.y, c12 = in.cc.x, c22 = in.cc.y;
    const float w00 = R[0] * c00 + R[1] * c01 + R[2] * c02;
    const float w01 = R[0] * c01 + R[1] * c11 + R[2] * c12;
    const float w02 = R[0] * c02 + R[1] * c12 + R[2] * c22;
    const float w10 = R[3] * c00 + R[4] * c01 + R[5] * c02;
    const float w11 = R[3] * c01 + R[4] * c11 + R[5] * c12;
    const float w12 = R[3] * c02 + R[4] * c12 + R[5] * c22;
    const float w20 = R[6] * c00 + R[7] * c01 + R[8] * c02;
    const float w21 = R[6] * c01 + R[7] * c11 + R[8] * c12;
    const float w22 = R[6] * c02 + R[7] * c12 + R[8] * c22;
    r00 = w00 * R[0] + w01 * R[1] + w02 * R[2];
    r01 = w00 * R[3] + w01 * R[4] + w02 * R[5];
    r02 = w00 * R[6] + w01 * R[7] + w02 * R[8];
    r11 = w10 * R[3] + w11 * R[4] + w12 * R[5];
    r12 = w10 * R[6] + w11 * R[7] + w12 * R[8];
    r22 = w20 * R[6] + w21 * R[7] + w22 * R[8];
  }
  const float ux = q.x - P.t[0], uy = q.y - P.t[1], uz = q.z - P.t[2];
  // compaction of the hits: level-major, lane order within a level
  int base = 0;
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const unsigned mask = __ballot_sync(0xffffffffu, hit[l]);
    if (hit[l]) {
      const int slot = base + __popc(mask & lt);
      float4* t = ws.term + slot * 3;
      // voxel record: s0 = {., ., ., C~22}, s1 = {mean, C~00}, s2 = {C~01, C~02, C~11, C~12}
      t[0] = make_float4(s1[l].w + r00, s2[l].x + r01, s2[l].y + r02, s2[l].z + r11);
      t[1] = make_float4(s2[l].w + r12, s0[l].w + r22, s1[l].x - q.x, s1[l].y - q.y);
      t[2] = make_float4(s1[l].z - q.z, ux, uy, uz);
      ws.w[slot] = m.w;
    }
    base += __popc(mask);
  }
  __syncwarp();
  for (int i = lane; i < base; i += 32)
    inl += accumulate_term(ws.term[3 * i], ws.term[3 * i + 1], ws.term[3 * i + 2], ws.w[i], acc) ? 1 : 0;
  __syncwarp();  // the stage is rewritten by the next round
}

// ---------------------------------------------------------------- block reduction
// Warp transpose-reduction: 32 values per lane -> lane l holds the warp total of value l
// (31 shuffles instead of 5 per value).
__device__ __forceinline__ void warp_transpose_reduce(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, c = 16; o >= 1; o >>= 1, c >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < c; ++j) {
      const float send = upper ? v[j] : v[j + c];
      const float keep = upper ? v[j + c] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// Same with error-free two-sum of the hi parts, collecting the rounding errors in lo.
__device__ __forceinline__ void warp_transpose_reduce_comp(float (&hi)[32], float (&lo)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, c = 16; o >= 1; o >>= 1, c >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < c; ++j) {
      const float sh = upper ? hi[j] : hi[j + c], sl = upper ? lo[j] : lo[j + c];
      const float kh = upper ? hi[j + c] : hi[j], kl = upper ? lo[j + c] : lo[j];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, o), rl = __shfl_xor_sync(0xffffffffu, sl, o);
      const float s = kh + rh;
      const float bp = s - kh;
      const float err = (kh - (s - bp)) + (rh - bp);  // two-sum (Knuth)
      hi[j] = s;
      lo[j] = kl + rl + err;
    }
  }
}

template <int BLOCK, int ACC>
__device__ __forceinline__ void block_reduce_store(const typename AccOf<ACC>::type& acc, int inl, double* out) {
  constexpr int NW = BLOCK / 32;
  __shared__ float s_hi[NW][32];
  __shared__ float s_lo[NW][32];
  __shared__ int s_inl[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float hi[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) hi[i] = (i < NACC) ? acc.s[i] : 0.f;
  if constexpr (ACC == GLIM_ACC_KAHAN) {
    float lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) lo[i] = (i < NACC) ? acc.c[i] : 0.f;
    warp_transpose_reduce_comp(hi, lo);
    s_lo[warp][lane] = lo[0];
  } else {
    warp_transpose_reduce(hi);
  }
  s_hi[warp][lane] = hi[0];
  const int wi = __reduce_add_sync(0xffffffffu, unsigned(inl));
  if (lane == 0) s_inl[warp] = wi;
  __syncthreads();
  if (threadIdx.x < NACC) {
    const int i = threadIdx.x;
    if constexpr (ACC == GLIM_ACC_FP32) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) t += s_hi[w][i];
      out[i] = double(t);
    } else if constexpr (ACC == GLIM_ACC_KAHAN) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) t += double(s_hi[w][i]) + double(s_lo[w][i]);
      out[i] = t;
    } else {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) t += double(s_hi[w][i]);
      out[i] = t;
    }
  } else if (threadIdx.x == NACC) {
    int t = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += s_inl[w];
    out[NACC] = double(t);
  }
  __syncthreads();  // shared buffers are reused by the next item
}

// ---------------------------------------------------------------- items and the kernel
template <int BLOCK, int ACC, int LMAX, bool IDS>
__device__ __forceinline__ void process_item(const LinArgs& a, int item, PairView& V, WarpStage<LMAX>& ws) {
  const Item it = a.items[item];
  int32_t* ids = nullptr;
  int idl = 0;
  if constexpr (IDS) {
    ids = a.ids + a.ids_off[it.pair];
    idl = a.ids_lv[it.pair];
  }
  if (threadIdx.x == 0) {
    const PairDev pd = a.pairs[it.pair];
    const PoseF pf = a.pose[it.pair];
#pragma unroll
    for (int i = 0; i < 9; ++i) V.R[i] = pf.R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      V.t[i] = pf.t[i];
      V.v[i] = pf.v[i];
    }
    V.F = a.frames[pd.src];
    V.M = a.maps[pd.map];
  }
  __syncthreads();
  typename AccOf<ACC>::type acc;
  acc.zero();
  int inl = 0;
  const int64_t n = V.F.n;
  const int64_t base = int64_t(it.start) + threadIdx.x;
  const int64_t end = min(int64_t(it.start) + a.tile, n);
  // software pipeline: the next round's point is read while the current round is processed
  PointIn cur;
  if (base < end) cur = load_point(V.F, base);
  const int rounds = a.ppt;
#pragma unroll 1
  for (int j = 0; j < rounds; ++j) {
    const int64_t k = base + int64_t(j) * BLOCK;
    PointIn nxt;
    const bool more = (j + 1 < rounds) && (k + BLOCK < end);
    if (more) nxt = load_point(V.F, k + BLOCK);
    warp_round<LMAX, IDS>(V, cur, k < end, k, a.validate, ws, acc, inl, ids, idl);
    if (more) cur = nxt;
  }
  // the reduction ends with a barrier, so V is free for the next item afterwards
  block_reduce_store<BLOCK, ACC>(acc, inl, a.part + int64_t(item) * PSTRIDE);
}

// With a.head set: persistent blocks take items from the atomic queue until it is exhausted.
// With a.head null: one block per item, item = a.item_base + blockIdx.x.
template <int BLOCK, int LMAX>
constexpr size_t lin_dyn_smem() {
  return size_t(BLOCK / 32) * sizeof(WarpStage<LMAX>);
}

template <int BLOCK, int ACC, int LMAX, bool IDS>
__device__ __forceinline__ void general_kernel_body(const LinArgs& a) {
  __shared__ PairView V;
  __shared__ int s_item[2];
  extern __shared__ float4 dyn_smem[];
  WarpStage<LMAX>& ws = reinterpret_cast<WarpStage<LMAX>*>(dyn_smem)[threadIdx.x >> 5];
  if (a.head == nullptr) {
    const int item = a.item_base + blockIdx.x;
    if (item < a.nitems) process_item<BLOCK, ACC, LMAX, IDS>(a, item, V, ws);
    return;
  }
  // the next item index is fetched one item ahead, so the queue's atomic latency overlaps work
  if (threadIdx.x == 0) s_item[0] = atomicAdd(a.head, 1);
  __syncthreads();
  int cur = s_item[0];
  for (int b = 1;; b ^= 1) {
    if (cur >= a.nitems) break;
    if (threadIdx.x == 0) s_item[b] = atomicAdd(a.head, 1);
    process_item<BLOCK, ACC, LMAX, IDS>(a, cur, V, ws);  // ends with a barrier
    cur = s_item[b];
  }
}

template <int BLOCK, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize(const LinArgs a) {
  general_kernel_body<BLOCK, ACC, LMAX, false>(a);
}

// The id-recording instantiation of the general kernel (inspection and parity tests): the same
// code plus the stores of the resolved voxel ids.
template <int BLOCK, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize_ids(const LinArgs a) {
  general_kernel_body<BLOCK, ACC, LMAX, true>(a);
}

// ---------------------------------------------------------------- per-lane kernels
// Every target level is a dense grid (k_linearize_dense) or every one is hashed
// (k_linearize_hash): a lane handles its own point from start to end.  Dense grid: a lookup
// is an index computation and one record read, without divergent branches; a key outside the
// grid's box reads the empty record before cell 0.  Hashed: the lookup first reads the
// block's table entry (the lanes of a warp mostly share a few 2 x 2 x 2 blocks, so the entries
// are warp-coherent and cached); a lane whose entry holds another block continues the probe in
// a loop bounded by the table's longest probe sequence (a warp-uniform branch skips it when
// no lane needs it); then the cell record is read as on a dense grid.  A lane past the end of
// its tile reads its tile's last point and is masked.  Because G = [-(u)x, I] is the same for
// all levels of a point, the lane sums w Omega, w Omega d and e over the levels (a miss, or a
// term whose S is not positive definite, adds nothing) and adds the G-form of the sums once:
// 28 accumulator updates per point instead of per hit.  The weight enters as
// w adj(S)/det(S), as in the general kernel; results agree up to FP32 rounding.

template <class MapT>
struct LaneView {  // per-item constants, written by thread 0
  float4 Rt[3];  // rows of [R | t]
  float4 v;      // target viewpoint (surface validation)
  const float4* pts;
  const float2* cov;
  const float* nrm;
  int end;  // one past the item's last point
  int pad;
  MapT M;
};
using DenseView = LaneView<DenseMapDev>;
using HashView = LaneView<HashMapDev>;

// The level descriptors and inverse resolutions are read as 16-byte words.
static_assert(sizeof(DenseLevelDev) == 32 && sizeof(HashLevelDev) == 32 && offsetof(DenseView, M) % 16 == 0 &&
                  offsetof(HashView, M) % 16 == 0 && offsetof(DenseMapDev, inv_r) % 16 == 0 &&
                  offsetof(HashMapDev, inv_r) % 16 == 0,
              "lane-kernel descriptors must sit on 16-byte boundaries");

// What a lane has read for one point: the transformed point, its weight and covariance, and
// the voxel records of every level (on hashed levels, once hash_resolve has found the cell).
// Split from the arithmetic so that one point's reads can be in flight while the previous
// point is computed.
template <int LMAX>
struct LaneFetch {
  float3 q;
  float w;
  bool live;
  float4 s0[LMAX];  // {id, C~22, ., .} (8 bytes read)
  float4 s1[LMAX], s2[LMAX];
  float2 ca, cb, cc;
  int idx;  // IDS: index of the point in its frame, -1 for a masked lane
};

// The part of a fetch that every layout shares: the covariance reads, the surface test, the
// FP32 transform and the masking of non-finite points.
template <class View>
__device__ __forceinline__ float3 lane_transform(const View& V, const float4 m, bool& live, int validate, int kk,
                                                 float2& ca, float2& cb, float2& cc) {
  // the covariance is read here rather than a round ahead: it is needed only after the voxel
  // reads are in flight, and the registers it would hold are worth more as occupancy
  const float2* cp = V.cov + 3 * int64_t(kk);
  ca = __ldg(cp);
  cb = __ldg(cp + 1);
  cc = __ldg(cp + 2);
  if (validate && V.nrm) {
    const float* nk = V.nrm + 3 * int64_t(kk);
    const float vv[3] = {V.v.x, V.v.y, V.v.z};
    live = live && !behind_surface(m.x, m.y, m.z, vv, __ldg(nk), __ldg(nk + 1), __ldg(nk + 2));
  }
  const float4 R0 = V.Rt[0], R1 = V.Rt[1], R2 = V.Rt[2];
  float3 q;  // R mu + t, one fused multiply-add per term from t in x, y, z order
  q.x = __fmaf_rn(R0.z, m.z, __fmaf_rn(R0.y, m.y, __fmaf_rn(R0.x, m.x, R0.w)));
  q.y = __fmaf_rn(R1.z, m.z, __fmaf_rn(R1.y, m.y, __fmaf_rn(R1.x, m.x, R1.w)));
  q.z = __fmaf_rn(R2.z, m.z, __fmaf_rn(R2.y, m.y, __fmaf_rn(R2.x, m.x, R2.w)));
  // keys of infinite or huge coordinates saturate outside every box; a NaN would convert to
  // 0, so a NaN point is masked (and zeroed, so that its masked arithmetic stays finite)
  const bool finite_q = q.x == q.x && q.y == q.y && q.z == q.z;
  live = live && finite_q;
  q.x = finite_q ? q.x : 0.f;
  q.y = finite_q ? q.y : 0.f;
  q.z = finite_q ? q.z : 0.f;
  return q;
}

// Dense grids: per level the key, the cell inside the grid's box and the record reads, the
// levels interleaved (kept in this form: splitting it into per-stage loops measured 6 %
// slower); descriptor {cells, ox, oy} {oz, nx, ny, nz}.
template <int LMAX, bool IDS>
__device__ __forceinline__ void lane_fetch(const DenseView& V, const float4 m, bool live, int validate, int kk,
                                           LaneFetch<LMAX>& F) {
  if constexpr (IDS) F.idx = live ? kk : -1;
  const float3 q = lane_transform(V, m, live, validate, kk, F.ca, F.cb, F.cc);
  // keys floor(q * inv_r_0) (FP32 product) and, on the coarser levels, that key shifted right
  // by the level (the plan runs these kernels only on resolutions doubling per level, where
  // this is floor(q * inv_r_l) exactly: 2.4 % faster than a product per level on the urban
  // step); a key outside [-2^20, 2^20) is in no table
  const int k0x = __float2int_rd(__fmul_rn(q.x, V.M.inv_r[0]));
  const int k0y = __float2int_rd(__fmul_rn(q.y, V.M.inv_r[0]));
  const int k0z = __float2int_rd(__fmul_rn(q.z, V.M.inv_r[0]));
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const int4 la = reinterpret_cast<const int4*>(&V.M.lv[l])[0];
    const uint4 lb = reinterpret_cast<const uint4*>(&V.M.lv[l])[1];
    const VoxSlot* base =
        reinterpret_cast<const VoxSlot*>(uint64_t(uint32_t(la.x)) | (uint64_t(uint32_t(la.y)) << 32));
    const int kx = k0x >> l, ky = k0y >> l, kz = k0z >> l;
    const uint32_t x = uint32_t(kx) - uint32_t(la.z), y = uint32_t(ky) - uint32_t(la.w), z = uint32_t(kz) - lb.x;
    const bool in_box = live && x < lb.y && y < lb.z && z < lb.w;
    const VoxSlot* sl = base + (in_box ? int((x * lb.z + y) * lb.w + z) : -1);  // -1: the empty record
    const float2 h2 = __ldg(reinterpret_cast<const float2*>(&sl->w0));
    F.s0[l] = make_float4(h2.x, h2.y, 0.f, 0.f);
    F.s1[l] = ldg4(&sl->w1);  // {mean, C~00}
    F.s2[l] = ldg4(&sl->w2);  // {C~01, C~02, C~11, C~12}
  }
  F.q = q;
  F.w = m.w;
  F.live = live;
}

// A point's sums over its levels (w Omega, w Omega d, e) and u = R mu, between the level
// arithmetic and the G-form.
struct LaneSums {
  float O00, O01, O02, O11, O12, O22, g0, g1, g2, es, ux, uy, uz;
};

template <int LMAX, bool HASH, bool IDS>
__device__ __forceinline__ void lane_levels(const LaneView<typename std::conditional<HASH, HashMapDev, DenseMapDev>::type>& V,
                                            LaneFetch<LMAX>& F, LaneSums& S, int& inl, int32_t* ids, int idl) {
  const float4 R0 = V.Rt[0], R1 = V.Rt[1], R2 = V.Rt[2];
  const float3 q = F.q;
  const bool live = F.live;
  float4(&s0)[LMAX] = F.s0;
  float4(&s1)[LMAX] = F.s1;
  float4(&s2)[LMAX] = F.s2;
  const float4 irq = *reinterpret_cast<const float4*>(V.M.inv_r);
  const float irv[4] = {irq.x, irq.y, irq.z, irq.w};
  (void)live;
  (void)irv;
  const float2 ca = F.ca, cb = F.cb, cc = F.cc;
  // R C R^T (once for all levels)
  const float w = F.w;
  const float c00 = ca.x, c01 = ca.y, c02 = cb.x, c11 = cb.y, c12 = cc.x, c22 = cc.y;
  const float w00 = R0.x * c00 + R0.y * c01 + R0.z * c02;
  const float w01 = R0.x * c01 + R0.y * c11 + R0.z * c12;
  const float w02 = R0.x * c02 + R0.y * c12 + R0.z * c22;
  const float w10 = R1.x * c00 + R1.y * c01 + R1.z * c02;
  const float w11 = R1.x * c01 + R1.y * c11 + R1.z * c12;
  const float w12 = R1.x * c02 + R1.y * c12 + R1.z * c22;
  const float w20 = R2.x * c00 + R2.y * c01 + R2.z * c02;
  const float w21 = R2.x * c01 + R2.y * c11 + R2.z * c12;
  const float w22 = R2.x * c02 + R2.y * c12 + R2.z * c22;
  const float r00 = w00 * R0.x + w01 * R0.y + w02 * R0.z;
  const float r01 = w00 * R1.x + w01 * R1.y + w02 * R1.z;
  const float r02 = w00 * R2.x + w01 * R2.y + w02 * R2.z;
  const float r11 = w10 * R1.x + w11 * R1.y + w12 * R1.z;
  const float r12 = w10 * R2.x + w11 * R2.y + w12 * R2.z;
  const float r22 = w20 * R2.x + w21 * R2.y + w22 * R2.z;
  // hits (after R C R^T, which overlaps the reads' latency)
  bool hit[LMAX];
  float vc22[LMAX];  // C~22 of the level's voxel
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    hit[l] = __float_as_int(s0[l].x) >= 0;  // occupied cell (empty records hold 0x80808080)
    vc22[l] = s0[l].y;
  }
  if constexpr (IDS) {  // the canonical id of the voxel each level resolved to, or -1
    if (F.idx >= 0) {
#pragma unroll
      for (int l = 0; l < LMAX; ++l) {
        if (l >= idl) continue;
        const int id = hit[l] ? __float_as_int(s0[l].x) : -1;  // a record starts with the id
        ids[int64_t(F.idx) * idl + l] = id;
      }
    }
  }
  // per level: S = C~ + R C R^T, w Omega = w adj(S) / det(S), y = w Omega d, and the sums over
  // levels (a term that is a miss or not positive definite adds nothing).  Skipping a level
  // (or the whole point) when no lane of the warp hits it was measured slower: the vote has
  // to wait for the voxel reads, which stops R C R^T from overlapping their latency.
  float O00 = 0.f, O01 = 0.f, O02 = 0.f, O11 = 0.f, O12 = 0.f, O22 = 0.f;
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, es = 0.f;
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const float a = s1[l].w + r00, b = s2[l].x + r01, c = s2[l].y + r02;
    const float d = s2[l].z + r11, e = s2[l].w + r12, f = vc22[l] + r22;
    const float dx = s1[l].x - q.x, dy = s1[l].y - q.y, dz = s1[l].z - q.z;
    const float A00 = d * f - e * e, A01 = c * e - b * f, A02 = b * e - c * d;
    const float A11 = a * f - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
    const float det = a * A00 + b * A01 + c * A02;
    const float id = __fdividef(w, det);
    // A d and d^T A d; the term enters the sums as w/det times these, by fused multiply-adds
    // predicated on the term's validity, an occupied record (id >= 0) and 0 < det(S) < inf,
    // which the asm forms itself from det and the id word (three compares, no select); a
    // masked term's adj(S) need not be finite, so it is not multiplied by zero: its
    // instructions do not execute.  A valid term counts as an inlier.
    const float a0 = A00 * dx + A01 * dy + A02 * dz;
    const float a1 = A01 * dx + A11 * dy + A12 * dz;
    const float a2 = A02 * dx + A12 * dy + A22 * dz;
    const float el = dx * a0 + dy * a1 + dz * a2;
    asm("{\n\t.reg .pred p;\n\t"
        "setp.gt.f32 p, %11, 0f00000000;\n\t"
        "setp.lt.and.f32 p, %11, 0f7F800000, p;\n\t"
        "setp.ge.and.s32 p, %23, 0, p;\n\t"
        "@p fma.rn.f32 %0, %13, %12, %0;\n\t"
        "@p fma.rn.f32 %1, %14, %12, %1;\n\t"
        "@p fma.rn.f32 %2, %15, %12, %2;\n\t"
        "@p fma.rn.f32 %3, %16, %12, %3;\n\t"
        "@p fma.rn.f32 %4, %17, %12, %4;\n\t"
        "@p fma.rn.f32 %5, %18, %12, %5;\n\t"
        "@p fma.rn.f32 %6, %19, %12, %6;\n\t"
        "@p fma.rn.f32 %7, %20, %12, %7;\n\t"
        "@p fma.rn.f32 %8, %21, %12, %8;\n\t"
        "@p fma.rn.f32 %9, %22, %12, %9;\n\t"
        "@p add.s32 %10, %10, 1;\n\t}"
        : "+f"(O00), "+f"(O01), "+f"(O02), "+f"(O11), "+f"(O12), "+f"(O22), "+f"(g0), "+f"(g1), "+f"(g2),
          "+f"(es), "+r"(inl)
        : "f"(det), "f"(id), "f"(A00), "f"(A01), "f"(A02), "f"(A11), "f"(A12), "f"(A22), "f"(a0), "f"(a1),
          "f"(a2), "f"(el), "r"(__float_as_int(s0[l].x)));
  }
  S.O00 = O00;
  S.O01 = O01;
  S.O02 = O02;
  S.O11 = O11;
  S.O12 = O12;
  S.O22 = O22;
  S.g0 = g0;
  S.g1 = g1;
  S.g2 = g2;
  S.es = es;
  S.ux = q.x - R0.w;
  S.uy = q.y - R1.w;
  S.uz = q.z - R2.w;
}

// The G-form of a point's level sums, G = [-(u)x, I] with u = R mu: 28 accumulator updates.
template <class A>
__device__ __forceinline__ void lane_gform(const LaneSums& S, A& acc) {
  const float O00 = S.O00, O01 = S.O01, O02 = S.O02, O11 = S.O11, O12 = S.O12, O22 = S.O22;
  const float g0 = S.g0, g1 = S.g1, g2 = S.g2, es = S.es;
  const float ux = S.ux, uy = S.uy, uz = S.uz;
  const float W00 = -uz * O01 + uy * O02, W01 = -uz * O11 + uy * O12, W02 = -uz * O12 + uy * O22;
  const float W10 = uz * O00 - ux * O02, W11 = uz * O01 - ux * O12, W12 = uz * O02 - ux * O22;
  const float W20 = -uy * O00 + ux * O01, W21 = -uy * O01 + ux * O11, W22 = -uy * O02 + ux * O12;
  acc.add2(0, -uz, W01, uy, W02);
  acc.add2(1, uz, W00, -ux, W02);
  acc.add2(2, -uy, W00, ux, W01);
  acc.add2(3, uz, W10, -ux, W12);
  acc.add2(4, -uy, W10, ux, W11);
  acc.add2(5, -uy, W20, ux, W21);
  acc.add(6, W00); acc.add(7, W01); acc.add(8, W02);
  acc.add(9, W10); acc.add(10, W11); acc.add(11, W12);
  acc.add(12, W20); acc.add(13, W21); acc.add(14, W22);
  acc.add(15, O00); acc.add(16, O01); acc.add(17, O02); acc.add(18, O11); acc.add(19, O12); acc.add(20, O22);
  acc.add2(21, uy, g2, -uz, g1);
  acc.add2(22, uz, g0, -ux, g2);
  acc.add2(23, ux, g1, -uy, g0);
  acc.add(24, g0); acc.add(25, g1); acc.add(26, g2);
  acc.add(27, es);
}

template <int LMAX, bool HASH, bool IDS, class A>
__device__ __forceinline__ void lane_compute(const LaneView<typename std::conditional<HASH, HashMapDev, DenseMapDev>::type>& V,
                                             LaneFetch<LMAX>& F, A& acc, int& inl, int32_t* ids, int idl) {
  LaneSums S;
  const int inl0 = inl;
  lane_levels<LMAX, HASH, IDS>(V, F, S, inl, ids, idl);
  // a round in which no lane of the warp has a valid term (about a quarter of the urban
  // step's rounds) adds only zeros: its G-form is skipped, after the level arithmetic, which
  // has consumed the records by then (dense grids: 5.60 against 5.69 ms on the urban step,
  // results unchanged; the hashed rounds, whose next records are resolved between the level
  // arithmetic and the G-form, measured 8.30 against 7.92 ms with it, so they do not skip)
  if (__any_sync(0xffffffffu, inl != inl0)) lane_gform(S, acc);
}

#include "lane_hash.cuh"

template <int BLOCK, int ACC, int LMAX, bool HASH, bool IDS>
__device__ __forceinline__ void process_item_lane(const LinArgs& a, int item,
                                                  LaneView<typename std::conditional<HASH, HashMapDev, DenseMapDev>::type>& V) {
  const Item it = a.items[item];
  int32_t* ids = nullptr;
  int idl = 0;
  if constexpr (IDS) {
    ids = a.ids + a.ids_off[it.pair];
    idl = a.ids_lv[it.pair];
  }
  if (threadIdx.x == 0) {
    const PairDev pd = a.pairs[it.pair];
    const PoseF pf = a.pose[it.pair];
#pragma unroll
    for (int r = 0; r < 3; ++r) V.Rt[r] = make_float4(pf.R[3 * r], pf.R[3 * r + 1], pf.R[3 * r + 2], pf.t[r]);
    V.v = make_float4(pf.v[0], pf.v[1], pf.v[2], 0.f);
    const FrameDev F = a.frames[pd.src];
    V.pts = F.pts;
    V.cov = F.cov;
    V.nrm = F.nrm;
    if constexpr (HASH) V.M = a.hmaps[pd.map];
    else V.M = a.dmaps[pd.map];
    V.end = int(min(int64_t(it.start) + a.tile, F.n));
  }
  __syncthreads();
  typename AccOf<ACC>::type acc;
  acc.zero();
  int inl = 0;
  const int last = V.end - 1;  // items are never empty
  const int first = it.start + int(threadIdx.x);
  const int rounds = min(a.ppt, (last - it.start) / BLOCK + 1);
  // A software pipeline over the rounds, unrolled twice so that the two buffers alternate
  // without copies.  Dense grids: a point's coordinates are read two rounds ahead, its voxel
  // records and covariance one round ahead (lane_fetch), so the reads of the next point are
  // in flight while the lane computes the current one (lane_compute): 9 % faster than reading
  // a point's records at the start of its own round.  Hashed levels: hash_rounds.
  if constexpr (!HASH) {
    LaneFetch<LMAX> fa, fb;
    lane_fetch<LMAX, IDS>(V, ldg4(V.pts + min(first, last)), first <= last, a.validate, min(first, last), fa);
    float4 pn = ldg4(V.pts + min(first + BLOCK, last));
    int j = 0;
#pragma unroll 1
    for (; j + 1 < rounds; j += 2) {
      const int k = first + j * BLOCK;
      lane_fetch<LMAX, IDS>(V, pn, k + BLOCK <= last, a.validate, min(k + BLOCK, last), fb);
      pn = ldg4(V.pts + min(k + 2 * BLOCK, last));
      lane_compute<LMAX, HASH, IDS>(V, fa, acc, inl, ids, idl);
      lane_fetch<LMAX, IDS>(V, pn, k + 2 * BLOCK <= last, a.validate, min(k + 2 * BLOCK, last), fa);
      pn = ldg4(V.pts + min(k + 3 * BLOCK, last));
      lane_compute<LMAX, HASH, IDS>(V, fb, acc, inl, ids, idl);
    }
    if (j < rounds) lane_compute<LMAX, HASH, IDS>(V, fa, acc, inl, ids, idl);
  } else {
    hash_rounds<BLOCK, LMAX, IDS>(V, a.validate, first, last, rounds, acc, inl, ids, idl);
  }
  block_reduce_store<BLOCK, ACC>(acc, inl, a.part + int64_t(item) * PSTRIDE);
}

template <int BLOCK, int ACC, int LMAX, bool HASH, bool IDS>
__device__ __forceinline__ void lane_kernel_body(const LinArgs& a) {
  __shared__ LaneView<typename std::conditional<HASH, HashMapDev, DenseMapDev>::type> V;
  __shared__ int s_item[2];
  if (a.head == nullptr) {
    const int item = a.item_base + blockIdx.x;
    if (item < a.nitems) process_item_lane<BLOCK, ACC, LMAX, HASH, IDS>(a, item, V);
    return;
  }
  if (threadIdx.x == 0) s_item[0] = atomicAdd(a.head, 1);
  __syncthreads();
  int cur = s_item[0];
  for (int b = 1;; b ^= 1) {
    if (cur >= a.nitems) break;
    if (threadIdx.x == 0) s_item[b] = atomicAdd(a.head, 1);
    process_item_lane<BLOCK, ACC, LMAX, HASH, IDS>(a, cur, V);  // ends with a barrier
    cur = s_item[b];
  }
}

template <int BLOCK, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize_dense(const LinArgs a) {
  lane_kernel_body<BLOCK, ACC, LMAX, false, false>(a);
}

template <int BLOCK, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize_hash(const LinArgs a) {
  lane_kernel_body<BLOCK, ACC, LMAX, true, false>(a);
}

// The id-recording instantiations of the per-lane kernels (inspection and parity tests): the
// same code plus the stores of the resolved voxel ids.
template <int BLOCK, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize_dense_ids(const LinArgs a) {
  lane_kernel_body<BLOCK, ACC, LMAX, false, true>(a);
}

template <int BLOCK, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize_hash_ids(const LinArgs a) {
  lane_kernel_body<BLOCK, ACC, LMAX, true, true>(a);
}

// Kernel and its dynamic shared memory (bytes) for a configuration; the attribute allowing
// that much dynamic shared memory is set on first use.
template <int B, int ACC, int L>
LinKernelInfo lin_info() {
  LinKernelInfo k;
  k.fn = k_linearize<B, ACC, L>;
  k.smem = lin_dyn_smem<B, L>();
  return k;
}

template <int ACC>
LinKernelInfo pick_lin(int block, int lmax) {
#define GLIM_PICK_L(B)                            \
  switch (lmax) {                                 \
    case 1: return lin_info<B, ACC, 1>();         \
    case 2: return lin_info<B, ACC, 2>();         \
    case 3: return lin_info<B, ACC, 3>();         \
    case 4: return lin_info<B, ACC, 4>();         \
  }                                               \
  return LinKernelInfo{};
  switch (block) {
    case 128: { GLIM_PICK_L(128) }
    case 256: { GLIM_PICK_L(256) }
  }
  return LinKernelInfo{};
#undef GLIM_PICK_L
}

template <int B, int ACC, int L, bool HASH>
LinKernelInfo lin_lane_info() {
  LinKernelInfo k;
  if constexpr (HASH) k.fn = k_linearize_hash<B, ACC, L>;
  else k.fn = k_linearize_dense<B, ACC, L>;
  k.smem = 0;
  return k;
}

template <int ACC, bool HASH>
LinKernelInfo pick_lin_lane(int block, int lmax) {
#define GLIM_PICK_LANE_L(B)                             \
  switch (lmax) {                                       \
    case 1: return lin_lane_info<B, ACC, 1, HASH>();    \
    case 2: return lin_lane_info<B, ACC, 2, HASH>();    \
    case 3: return lin_lane_info<B, ACC, 3, HASH>();    \
    case 4: return lin_lane_info<B, ACC, 4, HASH>();    \
  }                                                     \
  return LinKernelInfo{};
  switch (block) {  // 64-thread blocks: two warps share an item's barriers (2 % faster on the urban step)
    case 64: { GLIM_PICK_LANE_L(64) }
    case 128: { GLIM_PICK_LANE_L(128) }
    case 256: { GLIM_PICK_LANE_L(256) }
  }
#undef GLIM_PICK_LANE_L
  return LinKernelInfo{};
}

// The id-recording instantiations (accumulation mode GLIM_ACC_FP64; the lookup and the hit
// decisions are the same code in every mode): LANE 0 general, 1 dense grid, 2 hash.
template <int B, int L, int LANE>
LinKernelInfo lin_ids_info() {
  LinKernelInfo k;
  if constexpr (LANE == 1) {
    k.fn = k_linearize_dense_ids<B, GLIM_ACC_FP64, L>;
  } else if constexpr (LANE == 2) {
    k.fn = k_linearize_hash_ids<B, GLIM_ACC_FP64, L>;
  } else {
    k.fn = k_linearize_ids<B, GLIM_ACC_FP64, L>;
    k.smem = lin_dyn_smem<B, L>();
  }
  return k;
}

template <int LANE>
LinKernelInfo pick_lin_ids_lane(int block, int lmax) {
#define GLIM_PICK_IDS_L(B)                          \
  switch (lmax) {                                   \
    case 1: return lin_ids_info<B, 1, LANE>();      \
    case 2: return lin_ids_info<B, 2, LANE>();      \
    case 3: return lin_ids_info<B, 3, LANE>();      \
    case 4: return lin_ids_info<B, 4, LANE>();      \
  }                                                 \
  return LinKernelInfo{};
  switch (block) {
    case 64:
      if constexpr (LANE != 0) {  // the per-lane kernels only
        GLIM_PICK_IDS_L(64)
      }
      break;
    case 128: { GLIM_PICK_IDS_L(128) }
    case 256: { GLIM_PICK_IDS_L(256) }
  }
#undef GLIM_PICK_IDS_L
  return LinKernelInfo{};
}

LinKernelInfo pick_lin_ids_general(int block, int lmax);
LinKernelInfo pick_lin_ids_dense(int block, int lmax);
LinKernelInfo pick_lin_ids_hash(int block, int lmax);
LinKernelInfo pick_lin_fp32(int block, int lmax);
LinKernelInfo pick_lin_kahan(int block, int lmax);
LinKernelInfo pick_lin_fp64(int block, int lmax);
LinKernelInfo pick_lin_dense_fp32(int block, int lmax);
LinKernelInfo pick_lin_dense_kahan(int block, int lmax);
LinKernelInfo pick_lin_dense_fp64(int block, int lmax);
LinKernelInfo pick_lin_hash_fp32(int block, int lmax);
LinKernelInfo pick_lin_hash_kahan(int block, int lmax);
LinKernelInfo pick_lin_hash_fp64(int block, int lmax);

}  // namespace glim_detail
