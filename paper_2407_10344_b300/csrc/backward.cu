// backward.cu -- gradient of the summed matching cost E = sum_pairs e (Eq. (2) with the
// per-point weights) for automatic differentiation.  Correspondences are held fixed
// (piecewise constant); the per-point Jacobians are recomputed rather than stored.
//
// For a hit (point k, level l) with y = Omega d, e = d^T y, z = R^T y:
//   dE/dxi_s, dE/dxi_t (Omega fixed)  = 2 Lift^T g   with g = sum G^T (w y)  (the forward's 2 b)
//   dE/domega_s (through Omega)      += 2 w (z x C_k z)
//   dE/domega_t (through Omega)      += -R (2 w (z x C_k z))
//   dE/dmu_k                          = -2 w R^T sum_l y_l
//   dE/dw_k                           = sum_l e_l
// The Omega terms follow from dE/dS = -w y y^T and dS/domega_s,a = R (e_a x C - C e_a x) R^T,
// dS/domega_t,a = -(e_a x) S' + S' (e_a x) with S' = R C R^T.
//
// Work decomposition: an item is a tile of BWD_TILE points of one source frame and a group of
// that frame's pairs (all of them, unless the batch has too few tiles to fill the GPU: then a
// frame's pairs are split into up to `groups` contiguous groups); a persistent kernel takes
// items from an atomic queue and walks the pairs of its group in pair order.  Per pair, the
// points' contributions to the 9 pose sums (g: 6, the Omega term: 3) are block-reduced into
// the (item, pair) slot, while each point keeps its dE/dmu and dE/dw summed over the group's
// pairs in registers and writes them once (directly, or into its group's slot, summed over the
// groups in order afterwards).  Then fixed-order FP64 sums per pair and per frame.  No float
// atomics, so the gradient repeats bit for bit; no per-(pair, point) scratch.
#include <algorithm>
#include <cstring>

#include "lin_kernel.cuh"

namespace glim_detail {

// Scratch of the gradient pass of a plan, created at the first glim_plan_backward and kept by
// the plan: the work list of (source frame, point tile, group of the frame's pairs) items, the
// pairs grouped by source frame, one partial slot of 9 sums per (item, pair of its group), the
// per-pair gradients, and (only when a frame's pairs are split into several groups) one
// per-point gradient slot per group.
struct BwdScratch {
  int4* items = nullptr;               // nitems: (frame, first point, first pair of the group in src_list, pairs)
  int32_t* item_grp = nullptr;         // nitems: the item's group
  int64_t* item_slot = nullptr;        // nitems: first partial slot of the item
  int32_t* src_begin = nullptr;        // nframes + 1: pairs grouped by source frame
  int32_t* src_list = nullptr;
  int32_t* pair_item0 = nullptr;       // npairs: first item of the pair's group
  int32_t* pair_nitems = nullptr;      // npairs: items of that group (the frame's tiles)
  int32_t* pair_jj = nullptr;          // npairs: position of the pair in its group
  int32_t* tgt = nullptr;              // npairs: target frame
  int64_t* frame_off = nullptr;        // nframes + 1: first point of each frame in the outputs
  int32_t* frame_groups = nullptr;     // nframes: groups of the frame's pairs
  float4* pp = nullptr;                // groups > 1: groups x ntot per-point (dE/dmu, dE/dw) slots
  double* part = nullptr;              // nslots x 9
  double* pair_grad = nullptr;         // npairs x 12
  int* head = nullptr;                 // work-queue head
  void* views = nullptr;               // npairs: per-pair constants of the pipelined kernel (in src_list order)
  int nitems = 0, grid = 0, groups = 1;
  int grid_lane = 0;  // grid of the pipelined kernel (all-dense or all-hashed batches), else 0
  int64_t ntot = 0, nslots = 0;
  void release() {
    cudaFree(items);
    cudaFree(item_grp);
    cudaFree(item_slot);
    cudaFree(src_begin);
    cudaFree(src_list);
    cudaFree(pair_item0);
    cudaFree(pair_nitems);
    cudaFree(pair_jj);
    cudaFree(tgt);
    cudaFree(frame_off);
    cudaFree(frame_groups);
    cudaFree(pp);
    cudaFree(part);
    cudaFree(pair_grad);
    cudaFree(head);
    cudaFree(views);
    *this = BwdScratch{};
  }
};

void bwd_scratch_free(BwdScratch* sc) {
  if (!sc) return;
  sc->release();
  delete sc;
}

}  // namespace glim_detail

namespace {

constexpr int BWD_BLOCK = 256;
constexpr int BWD_PPT = 4;  // points per thread of an item
constexpr int BWD_TILE = BWD_BLOCK * BWD_PPT;
constexpr int BSTRIDE = 9;  // doubles per partial slot: g (6), Omega term (3)

struct BwdArgs {
  const int4* items;
  const int32_t* item_grp;
  const int64_t* item_slot;
  int32_t nitems;
  int* head;
  const PairDev* pairs;
  const FrameDev* frames;
  const MapDev* maps;
  const DenseMapDev* dmaps;  // per map, when every target level is a dense grid
  const HashMapDev* hmaps;   // per map, when every target level is hashed
  const PoseF* pose;
  const int32_t* src_list;
  const int64_t* frame_off;
  int64_t ntot;
  int32_t validate;
  int32_t full;
  double* part;
  float4* pp;  // groups > 1: per-point slots of the groups; else null
  float* dmu;
  float* dw;
};

// One point against one pair: adds its 9 pose sums to acc and its (dE/dmu, dE/dw) to out.
__device__ __forceinline__ void point_gradient(const PairView& V, int64_t k, int validate, int full, float (&acc)[9],
                                               float4& out) {
  const float4 m = V.F.pts[k];
  if (validate && V.F.nrm &&
      behind_surface(m.x, m.y, m.z, V.v, V.F.nrm[3 * k], V.F.nrm[3 * k + 1], V.F.nrm[3 * k + 2]))
    return;
  const float2 ca = V.F.cov[3 * k], cb = V.F.cov[3 * k + 1], cc = V.F.cov[3 * k + 2];
  const float c00 = ca.x, c01 = ca.y, c02 = cb.x, c11 = cb.y, c12 = cc.x, c22 = cc.y;
  const float* R = V.R;
  const float3 q = transform_pinned(R, V.t, m.x, m.y, m.z);
  const float3 u = make_float3(q.x - V.t[0], q.y - V.t[1], q.z - V.t[2]);
  // R C R^T
  float W[3][3], S[3][3];
  const float C[3][3] = {{c00, c01, c02}, {c01, c11, c12}, {c02, c12, c22}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W[i][j] = R[3 * i] * C[0][j] + R[3 * i + 1] * C[1][j] + R[3 * i + 2] * C[2][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = W[i][0] * R[3 * j] + W[i][1] * R[3 * j + 1] + W[i][2] * R[3 * j + 2];
  float Y[3] = {0, 0, 0}, E = 0.f, av[3] = {0, 0, 0};
  for (int l = 0; l < V.M.levels; ++l) {
    const LevelDev& L = V.M.lv[l];
    int kx, ky, kz;
    if (!level_key3(q, L.inv_r, kx, ky, kz)) continue;
    int vid;
    const int s = find_voxel(L, kx, ky, kz, &vid);
    if (s < 0) continue;
    const float4 v0 = L.slots[s].w0, v1 = L.slots[s].w1, v2 = L.slots[s].w2;
    const float sa = v1.w + S[0][0], sb = v2.x + S[0][1], sc = v2.y + S[0][2], sd = v2.z + S[1][1],
                se = v2.w + S[1][2], sf = v0.w + S[2][2];
    const float A00 = sd * sf - se * se, A01 = sc * se - sb * sf, A02 = sb * se - sc * sd;
    const float A11 = sa * sf - sc * sc, A12 = sb * sc - sa * se, A22 = sa * sd - sb * sb;
    const float det = sa * A00 + sb * A01 + sc * A02;
    if (!(det > 0.f) || !isfinite(det)) continue;
    const float id = __fdividef(1.f, det);
    const float O[3][3] = {{A00 * id, A01 * id, A02 * id}, {A01 * id, A11 * id, A12 * id},
                           {A02 * id, A12 * id, A22 * id}};
    const float d[3] = {v1.x - q.x, v1.y - q.y, v1.z - q.z};
    float y[3];
    for (int i = 0; i < 3; ++i) y[i] = O[i][0] * d[0] + O[i][1] * d[1] + O[i][2] * d[2];
    E += d[0] * y[0] + d[1] * y[1] + d[2] * y[2];
    for (int i = 0; i < 3; ++i) Y[i] += y[i];
    if (full) {
      float z[3], Cz[3];
      for (int i = 0; i < 3; ++i) z[i] = R[i] * y[0] + R[3 + i] * y[1] + R[6 + i] * y[2];  // R^T y
      for (int i = 0; i < 3; ++i) Cz[i] = C[i][0] * z[0] + C[i][1] * z[1] + C[i][2] * z[2];
      av[0] += z[1] * Cz[2] - z[2] * Cz[1];
      av[1] += z[2] * Cz[0] - z[0] * Cz[2];
      av[2] += z[0] * Cz[1] - z[1] * Cz[0];
    }
  }
  const float w = m.w;
  // dE/dmu = -2 w R^T Y, dE/dw = E
  out.x += -2.f * w * (R[0] * Y[0] + R[3] * Y[1] + R[6] * Y[2]);
  out.y += -2.f * w * (R[1] * Y[0] + R[4] * Y[1] + R[7] * Y[2]);
  out.z += -2.f * w * (R[2] * Y[0] + R[5] * Y[1] + R[8] * Y[2]);
  out.w += E;
  const float wy[3] = {w * Y[0], w * Y[1], w * Y[2]};
  acc[0] += u.y * wy[2] - u.z * wy[1];
  acc[1] += u.z * wy[0] - u.x * wy[2];
  acc[2] += u.x * wy[1] - u.y * wy[0];
  acc[3] += wy[0];
  acc[4] += wy[1];
  acc[5] += wy[2];
  acc[6] += 2.f * w * av[0];
  acc[7] += 2.f * w * av[1];
  acc[8] += 2.f * w * av[2];
}

__device__ __forceinline__ void backward_item(const BwdArgs& a, int g, PairView& V, float (&s_red)[BWD_BLOCK / 32][9]) {
  const int4 it = a.items[g];
  const int f = it.x;
  const int64_t start = it.y;
  const int pb = it.z, npf = it.w;
  const int64_t slot0 = a.item_slot[g];
  const int64_t n = a.frames[f].n;
  const int64_t end = min(start + int64_t(BWD_TILE), n);
  float4 pacc[BWD_PPT];
#pragma unroll
  for (int r = 0; r < BWD_PPT; ++r) pacc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int j = 0; j < npf; ++j) {
    if (threadIdx.x == 0) {
      const int p = a.src_list[pb + j];
      const PairDev pd = a.pairs[p];
      const PoseF pf = a.pose[p];
      for (int i = 0; i < 9; ++i) V.R[i] = pf.R[i];
      for (int i = 0; i < 3; ++i) {
        V.t[i] = pf.t[i];
        V.v[i] = pf.v[i];
      }
      V.F = a.frames[f];
      V.M = a.maps[pd.map];
    }
    __syncthreads();
    float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int r = 0; r < BWD_PPT; ++r) {
      const int64_t k = start + int64_t(r) * BWD_BLOCK + threadIdx.x;
      if (k < end) point_gradient(V, k, a.validate, a.full, acc, pacc[r]);
    }
    // block reduction: warp trees in FP32, warps summed in FP64 (fixed order)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float v = acc[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_red[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < BWD_BLOCK / 32; ++w) t += double(s_red[w][threadIdx.x]);
      a.part[(slot0 + j) * BSTRIDE + threadIdx.x] = t;
    }
    __syncthreads();  // V and s_red are rewritten for the next pair
  }
  const int64_t base = a.frame_off[f];
#pragma unroll
  for (int r = 0; r < BWD_PPT; ++r) {
    const int64_t k = start + int64_t(r) * BWD_BLOCK + threadIdx.x;
    if (k < end && a.pp) {
      a.pp[int64_t(a.item_grp[g]) * a.ntot + base + k] = pacc[r];
    } else if (k < end) {
      if (a.dmu) {
        a.dmu[3 * (base + k)] = pacc[r].x;
        a.dmu[3 * (base + k) + 1] = pacc[r].y;
        a.dmu[3 * (base + k) + 2] = pacc[r].z;
      }
      if (a.dw) a.dw[base + k] = pacc[r].w;
    }
  }
  // the queue's next item index (written by thread 0 during this item) is read after this
  // barrier: an item of a frame that is the source of no pair has no other barrier
  __syncthreads();
}

// Persistent blocks over the item queue (the next item fetched one item ahead).
__global__ void __launch_bounds__(BWD_BLOCK) k_backward_items(const BwdArgs a) {
  __shared__ PairView V;
  __shared__ float s_red[BWD_BLOCK / 32][9];
  __shared__ int s_item[2];
  if (threadIdx.x == 0) s_item[0] = atomicAdd(a.head, 1);
  __syncthreads();
  int cur = s_item[0];
  for (int b = 1;; b ^= 1) {
    if (cur >= a.nitems) break;
    if (threadIdx.x == 0) s_item[b] = atomicAdd(a.head, 1);
    backward_item(a, cur, V, s_red);  // ends with a barrier
    cur = s_item[b];
  }
}

// ---------------------------------------------------------------- pipelined form
// Batches whose target maps are all dense grids, or all hashed voxel blocks, take the
// per-lane form of the linearization kernels: a block of BWL_BLOCK threads, BWL_PPT points
// per thread and pair (the same 1024-point tiles), the records of a (pair, point) read one
// round ahead of its arithmetic (lane_fetch, or hash_fetch then hash_resolve), across the
// pairs of the group too.  The per-pair constants of the group (at most BWL_VMAX pairs) are
// built once per gradient call in the order of the pairs by source frame (k_backward_views)
// and copied into shared memory once per item, so a pair starts without a wait; each warp
// keeps its 9 pose sums of every pair in shared memory and the block sums them once at the
// end of the item (FP32 warp trees, warps in FP64, fixed order).  A point's dE/dmu and dE/dw,
// summed over the pairs, stay in shared memory (one float4 per point of the tile).
constexpr int BWL_BLOCK = 128;
constexpr int BWL_PPT = BWD_TILE / BWL_BLOCK;
constexpr int BWL_VMAX = 16;  // pairs per group at most (bwd_prepare splits larger groups)
static_assert(BWL_PPT % 2 == 0, "the rounds alternate two fetch buffers");

template <bool HASH>
using BwlView = LaneView<typename std::conditional<HASH, HashMapDev, DenseMapDev>::type>;
static_assert(sizeof(BwlView<false>) % 16 == 0 && sizeof(BwlView<true>) % 16 == 0, "views are copied as float4");

template <int LMAX, bool HASH, class View>
__device__ __forceinline__ void bwl_fetch(const View& V, const float4* pts, int k, int last, int validate,
                                          LaneFetch<LMAX>& F) {
  const int kk = min(k, last);
  const float4 m = ldg4(pts + kk);
  if constexpr (HASH) {
    HashFetch<LMAX> h;
    hash_fetch<LMAX, false>(V, m, k <= last, validate, kk, h);
    hash_resolve<LMAX, false>(V, h, F);
  } else {
    lane_fetch<LMAX, false>(V, m, k <= last, validate, kk, F);
  }
}

// One (pair, point) from its fetched records: the same terms as point_gradient.
template <int LMAX, class View>
__device__ __forceinline__ void bwl_point(const View& V, const LaneFetch<LMAX>& F, int full, float (&acc)[9],
                                          float4& pg) {
  const float4 R0 = V.Rt[0], R1 = V.Rt[1], R2 = V.Rt[2];
  const float3 q = F.q;
  const float c00 = F.ca.x, c01 = F.ca.y, c02 = F.cb.x, c11 = F.cb.y, c12 = F.cc.x, c22 = F.cc.y;
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
  float Y0 = 0.f, Y1 = 0.f, Y2 = 0.f, E = 0.f, av0 = 0.f, av1 = 0.f, av2 = 0.f;
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const float4 v0 = F.s0[l], v1 = F.s1[l], v2 = F.s2[l];
    const bool hit = __float_as_int(v0.x) >= 0;  // occupied cell
    const float sa = v1.w + r00, sb = v2.x + r01, sc = v2.y + r02, sd = v2.z + r11, se = v2.w + r12, sf = v0.y + r22;
    const float A00 = sd * sf - se * se, A01 = sc * se - sb * sf, A02 = sb * se - sc * sd;
    const float A11 = sa * sf - sc * sc, A12 = sb * sc - sa * se, A22 = sa * sd - sb * sb;
    const float det = sa * A00 + sb * A01 + sc * A02;
    const bool ok = hit && det > 0.f && det < INFINITY;
    const float id = __fdividef(1.f, det);
    const float d0 = v1.x - q.x, d1 = v1.y - q.y, d2 = v1.z - q.z;
    // y = Omega d = adj(S) d / det (Omega itself is not needed here)
    const float y0 = (A00 * d0 + A01 * d1 + A02 * d2) * id;
    const float y1 = (A01 * d0 + A11 * d1 + A12 * d2) * id;
    const float y2 = (A02 * d0 + A12 * d1 + A22 * d2) * id;
    const float el = d0 * y0 + d1 * y1 + d2 * y2;
    // a term that is a miss or not positive definite adds nothing: its additions are
    // predicated on `ok` (its values need not be finite, so it is not multiplied by zero);
    // 2.6 % faster than selecting zero
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "@p add.f32 %0, %0, %5;\n\t"
        "@p add.f32 %1, %1, %6;\n\t"
        "@p add.f32 %2, %2, %7;\n\t"
        "@p add.f32 %3, %3, %8;\n\t}"
        : "+f"(Y0), "+f"(Y1), "+f"(Y2), "+f"(E)
        : "r"(ok ? 1u : 0u), "f"(y0), "f"(y1), "f"(y2), "f"(el));
    if (full) {
      const float z0 = R0.x * y0 + R1.x * y1 + R2.x * y2;  // R^T y
      const float z1 = R0.y * y0 + R1.y * y1 + R2.y * y2;
      const float z2 = R0.z * y0 + R1.z * y1 + R2.z * y2;
      const float Cz0 = c00 * z0 + c01 * z1 + c02 * z2;
      const float Cz1 = c01 * z0 + c11 * z1 + c12 * z2;
      const float Cz2 = c02 * z0 + c12 * z1 + c22 * z2;
      // av += z x C z
      asm("{\n\t.reg .pred p;\n\t"
          "setp.ne.u32 p, %3, 0;\n\t"
          "@p fma.rn.f32 %0, %4, %5, %0;\n\t"
          "@p fma.rn.f32 %0, %6, %7, %0;\n\t"
          "@p fma.rn.f32 %1, %8, %9, %1;\n\t"
          "@p fma.rn.f32 %1, %10, %11, %1;\n\t"
          "@p fma.rn.f32 %2, %12, %13, %2;\n\t"
          "@p fma.rn.f32 %2, %14, %15, %2;\n\t}"
          : "+f"(av0), "+f"(av1), "+f"(av2)
          : "r"(ok ? 1u : 0u), "f"(z1), "f"(Cz2), "f"(-z2), "f"(Cz1), "f"(z2), "f"(Cz0), "f"(-z0), "f"(Cz2),
            "f"(z0), "f"(Cz1), "f"(-z1), "f"(Cz0));
    }
  }
  const float w = F.w;
  // dE/dmu = -2 w R^T Y, dE/dw = E
  pg.x += -2.f * w * (R0.x * Y0 + R1.x * Y1 + R2.x * Y2);
  pg.y += -2.f * w * (R0.y * Y0 + R1.y * Y1 + R2.y * Y2);
  pg.z += -2.f * w * (R0.z * Y0 + R1.z * Y1 + R2.z * Y2);
  pg.w += E;
  const float ux = q.x - R0.w, uy = q.y - R1.w, uz = q.z - R2.w;
  const float wy0 = w * Y0, wy1 = w * Y1, wy2 = w * Y2;
  acc[0] += uy * wy2 - uz * wy1;
  acc[1] += uz * wy0 - ux * wy2;
  acc[2] += ux * wy1 - uy * wy0;
  acc[3] += wy0;
  acc[4] += wy1;
  acc[5] += wy2;
  acc[6] += 2.f * w * av0;
  acc[7] += 2.f * w * av1;
  acc[8] += 2.f * w * av2;
}

// The constants of every pair, in the order of the pairs by source frame (src_list), for the
// poses of this gradient call.
template <bool HASH>
__global__ void k_backward_views(const BwdArgs a, int npairs, BwlView<HASH>* __restrict__ views) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= npairs) return;
  const int p = a.src_list[pos];
  const PairDev pd = a.pairs[p];
  const PoseF pf = a.pose[p];
  BwlView<HASH> V;
#pragma unroll
  for (int r = 0; r < 3; ++r) V.Rt[r] = make_float4(pf.R[3 * r], pf.R[3 * r + 1], pf.R[3 * r + 2], pf.t[r]);
  V.v = make_float4(pf.v[0], pf.v[1], pf.v[2], 0.f);
  const FrameDev F = a.frames[pd.src];
  V.pts = F.pts;
  V.cov = F.cov;
  V.nrm = F.nrm;
  if constexpr (HASH) V.M = a.hmaps[pd.map];
  else V.M = a.dmaps[pd.map];
  V.end = 0;  // unused: the item knows its tile
  V.pad = 0;
  views[pos] = V;
}

template <int LMAX, bool HASH>
__device__ __forceinline__ void bwl_item(const BwdArgs& a, const BwlView<HASH>* __restrict__ views, int g,
                                         BwlView<HASH> (&Vs)[BWL_VMAX], float (&s_red)[BWL_VMAX][BWL_BLOCK / 32][9],
                                         float4 (&s_pg)[BWL_PPT][BWL_BLOCK]) {
  const int4 it = a.items[g];
  const int f = it.x;
  const int start = it.y;
  const int pb = it.z, npf = it.w;
  const int64_t slot0 = a.item_slot[g];
  const int end = int(min(int64_t(start) + BWD_TILE, a.frames[f].n));
  const int last = end - 1;  // items are never empty
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int r = 0; r < BWL_PPT; ++r) s_pg[r][tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  {  // the group's views (a frame that is the source of no pair has items with none)
    constexpr int W = int(sizeof(BwlView<HASH>) / 16);
    const float4* src = reinterpret_cast<const float4*>(views + pb);
    float4* dst = reinterpret_cast<float4*>(Vs);
    for (int i = tid; i < npf * W; i += BWL_BLOCK) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const float4* pts = a.frames[f].pts;
  LaneFetch<LMAX> fa, fb;
  if (npf > 0) bwl_fetch<LMAX, HASH>(Vs[0], pts, start + tid, last, a.validate, fa);
#pragma unroll 1
  for (int j = 0; j < npf; ++j) {
    const auto& V = Vs[j];
    const bool more = j + 1 < npf;
    float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    // two rounds per iteration (the buffers alternate); not unrolled further, so that the
    // code of a pair stays small enough for the instruction cache
#pragma unroll 1
    for (int r = 0; r < BWL_PPT; r += 2) {
      bwl_fetch<LMAX, HASH>(V, pts, start + (r + 1) * BWL_BLOCK + tid, last, a.validate, fb);
      bwl_point<LMAX>(V, fa, a.full, acc, s_pg[r][tid]);
      // round r + 2 of this pair, or the first round of the next pair
      const bool in_pair = r + 2 < BWL_PPT;
      if (in_pair || more)
        bwl_fetch<LMAX, HASH>(Vs[in_pair ? j : j + 1], pts, start + (in_pair ? r + 2 : 0) * BWL_BLOCK + tid, last,
                              a.validate, fa);
      bwl_point<LMAX>(V, fb, a.full, acc, s_pg[r + 1][tid]);
    }
    // this warp's pose sums of pair j (FP32 tree)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float v = acc[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_red[j][warp][i] = v;
    }
  }
  __syncthreads();
  // the pairs' pose sums over the warps in FP64, in warp order
  for (int t = tid; t < npf * 9; t += BWL_BLOCK) {
    const int j = t / 9, i = t - 9 * j;
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < BWL_BLOCK / 32; ++w) sum += double(s_red[j][w][i]);
    a.part[(slot0 + j) * BSTRIDE + i] = sum;
  }
  const int64_t base = a.frame_off[f];
#pragma unroll
  for (int r = 0; r < BWL_PPT; ++r) {
    const int64_t k = start + r * BWL_BLOCK + tid;
    const float4 pg = s_pg[r][tid];
    if (k < end && a.pp) {
      a.pp[int64_t(a.item_grp[g]) * a.ntot + base + k] = pg;
    } else if (k < end) {
      if (a.dmu) {
        a.dmu[3 * (base + k)] = pg.x;
        a.dmu[3 * (base + k) + 1] = pg.y;
        a.dmu[3 * (base + k) + 2] = pg.z;
      }
      if (a.dw) a.dw[base + k] = pg.w;
    }
  }
  // the queue's next item index (written by thread 0 during this item) is read after this
  // barrier, and the views and pose sums are rewritten by the next item
  __syncthreads();
}

template <int LMAX, bool HASH>
__global__ void __launch_bounds__(BWL_BLOCK, 4) k_backward_lane(const BwdArgs a, const BwlView<HASH>* views) {
  __shared__ BwlView<HASH> Vs[BWL_VMAX];
  __shared__ float s_red[BWL_VMAX][BWL_BLOCK / 32][9];
  __shared__ float4 s_pg[BWL_PPT][BWL_BLOCK];
  __shared__ int s_item[2];
  if (threadIdx.x == 0) s_item[0] = atomicAdd(a.head, 1);
  __syncthreads();
  int cur = s_item[0];
  for (int b = 1;; b ^= 1) {
    if (cur >= a.nitems) break;
    if (threadIdx.x == 0) s_item[b] = atomicAdd(a.head, 1);
    bwl_item<LMAX, HASH>(a, views, cur, Vs, s_red, s_pg);  // ends with a barrier
    cur = s_item[b];
  }
}

// Launch of the pipelined gradient pass for a plan whose target maps are all dense grids or
// all hashed, with 1 to 4 levels: the views, then the items.  false: the general kernel runs.
template <bool HASH>
bool launch_backward_lane_t(const glim_plan* p, const BwdScratch& sc, const BwdArgs& a, cudaStream_t st) {
  auto* views = reinterpret_cast<BwlView<HASH>*>(sc.views);
  if (p->npairs > 0) k_backward_views<HASH><<<ceil_div_i(p->npairs, 128), 128, 0, st>>>(a, p->npairs, views);
  switch (p->lmax) {
    case 1: k_backward_lane<1, HASH><<<sc.grid_lane, BWL_BLOCK, 0, st>>>(a, views); return true;
    case 2: k_backward_lane<2, HASH><<<sc.grid_lane, BWL_BLOCK, 0, st>>>(a, views); return true;
    case 3: k_backward_lane<3, HASH><<<sc.grid_lane, BWL_BLOCK, 0, st>>>(a, views); return true;
    case 4: k_backward_lane<4, HASH><<<sc.grid_lane, BWL_BLOCK, 0, st>>>(a, views); return true;
  }
  return false;
}

// Blocks per SM of the pipelined kernel for a plan, or 0 when the plan takes the general one.
int backward_lane_occupancy(const glim_plan* p) {
  const bool dense = p->d_dmaps != nullptr, hash = p->d_hmaps != nullptr;
  if ((!dense && !hash) || p->lmax < 1 || p->lmax > 4) return 0;
  const void* fn = nullptr;
  switch (p->lmax) {
    case 1: fn = dense ? reinterpret_cast<const void*>(k_backward_lane<1, false>) : reinterpret_cast<const void*>(k_backward_lane<1, true>); break;
    case 2: fn = dense ? reinterpret_cast<const void*>(k_backward_lane<2, false>) : reinterpret_cast<const void*>(k_backward_lane<2, true>); break;
    case 3: fn = dense ? reinterpret_cast<const void*>(k_backward_lane<3, false>) : reinterpret_cast<const void*>(k_backward_lane<3, true>); break;
    default: fn = dense ? reinterpret_cast<const void*>(k_backward_lane<4, false>) : reinterpret_cast<const void*>(k_backward_lane<4, true>); break;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BWL_BLOCK, 0) != cudaSuccess) {
    cudaGetLastError();  // the general kernel runs instead
    return 0;
  }
  return std::max(per_sm, 1);
}

// per pair: dxi_pair (12) = 2 Lift^T g + [a; 0; -R a; 0], g and a summed over the items of
// the pair's group in item order
__global__ void k_backward_pairs(const double* __restrict__ part, const int64_t* __restrict__ item_slot,
                                 const int32_t* __restrict__ pair_item0, const int32_t* __restrict__ pair_nitems,
                                 const int32_t* __restrict__ pair_jj, const double* __restrict__ pose64, int npairs,
                                 double* __restrict__ pair_grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int i0 = pair_item0[p], ni = pair_nitems[p], jj = pair_jj[p];
  double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = i0; i < i0 + ni; ++i) {
    const double* sl = part + (item_slot[i] + jj) * BSTRIDE;
    for (int c = 0; c < 9; ++c) s[c] += sl[c];
  }
  const double* P = pose64 + 12 * int64_t(p);
  const double* R = P;
  const double t[3] = {P[9], P[10], P[11]};
  const double gr[3] = {s[0], s[1], s[2]}, gt[3] = {s[3], s[4], s[5]}, av[3] = {s[6], s[7], s[8]};
  double* o = pair_grad + 12 * int64_t(p);
  for (int i = 0; i < 3; ++i) {
    // source: 2 b_s = -2 [R^T g_r; R^T g_t]
    o[i] = -2.0 * (R[i] * gr[0] + R[3 + i] * gr[1] + R[6 + i] * gr[2]) + av[i];
    o[3 + i] = -2.0 * (R[i] * gt[0] + R[3 + i] * gt[1] + R[6 + i] * gt[2]);
  }
  // target: 2 b_t = 2 [g_r + t x g_t; g_t]
  const double txg[3] = {t[1] * gt[2] - t[2] * gt[1], t[2] * gt[0] - t[0] * gt[2], t[0] * gt[1] - t[1] * gt[0]};
  for (int i = 0; i < 3; ++i) {
    o[6 + i] = 2.0 * (gr[i] + txg[i]) - (R[3 * i] * av[0] + R[3 * i + 1] * av[1] + R[3 * i + 2] * av[2]);
    o[9 + i] = 2.0 * gt[i];
  }
}

__global__ void k_backward_frames(const double* __restrict__ pair_grad, const PairDev* __restrict__ pairs,
                                  const int32_t* __restrict__ tgt, int npairs, int nframes, double* __restrict__ dxi) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nframes) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int p = 0; p < npairs; ++p) {
    if (pairs[p].src == f)
      for (int c = 0; c < 6; ++c) s[c] += pair_grad[12 * int64_t(p) + c];
    if (tgt[p] == f)
      for (int c = 0; c < 6; ++c) s[c] += pair_grad[12 * int64_t(p) + 6 + c];
  }
  for (int c = 0; c < 6; ++c) dxi[6 * int64_t(f) + c] = s[c];
}

// groups > 1: per point, the sum of its frame's group slots in group order.
__global__ void k_backward_points(const float4* __restrict__ pp, const int64_t* __restrict__ frame_off,
                                  const int32_t* __restrict__ frame_groups, int nframes, int64_t ntot,
                                  float* __restrict__ dmu, float* __restrict__ dw) {
  const int64_t gi = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gi >= ntot) return;
  int lo = 0, hi = nframes - 1;  // the frame of point gi
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frame_off[mid] <= gi) lo = mid;
    else hi = mid - 1;
  }
  float4 t = pp[gi];
  for (int g = 1; g < frame_groups[lo]; ++g) {
    const float4 v = pp[int64_t(g) * ntot + gi];
    t.x += v.x;
    t.y += v.y;
    t.z += v.z;
    t.w += v.w;
  }
  if (dmu) {
    dmu[3 * gi] = t.x;
    dmu[3 * gi + 1] = t.y;
    dmu[3 * gi + 2] = t.z;
  }
  if (dw) dw[gi] = t.w;
}

// Host tables of a batch, uploaded into freshly allocated scratch (synchronous copies).
glim_status bwd_prepare(glim_plan* p, BwdScratch& sc) {
  glim_ctx* ctx = p->ctx;
  const int npairs = p->npairs, nframes = p->nframes;
  std::vector<int32_t> src_begin(nframes + 1, 0), src_list, pos(std::max(npairs, 1), 0), tgt(std::max(npairs, 1), 0);
  for (int f = 0; f < nframes; ++f) {
    src_begin[f] = int32_t(src_list.size());
    for (int q = 0; q < npairs; ++q)
      if (p->pairs[q].src_frame == f) {
        pos[q] = int32_t(src_list.size()) - src_begin[f];
        src_list.push_back(q);
      }
  }
  src_begin[nframes] = int32_t(src_list.size());
  for (int q = 0; q < npairs; ++q) tgt[q] = p->pairs[q].tgt_frame;
  // groups: enough items (tiles x groups) to fill the GPU about eight times over
  std::vector<int64_t> frame_off(nframes + 1, 0), ntiles(std::max(nframes, 1), 0);
  int64_t base_work = 0;
  int max_npf = 1;
  for (int f = 0; f < nframes; ++f) {
    const int64_t n = p->frames[f].n;
    frame_off[f + 1] = frame_off[f] + n;
    ntiles[f] = (n + BWD_TILE - 1) / BWD_TILE;
    const int npf = src_begin[f + 1] - src_begin[f];
    if (npf > 0) base_work += ntiles[f];
    max_npf = std::max(max_npf, npf);
  }
  const int64_t target = 8 * int64_t(ctx->num_sms);
  const int G = int(std::max<int64_t>(1, std::min<int64_t>(max_npf, base_work > 0 ? (target + base_work - 1) / base_work : 1)));
  std::vector<int4> items;
  std::vector<int32_t> item_grp, frame_groups(std::max(nframes, 1), 1);
  std::vector<int64_t> item_slot;
  std::vector<int32_t> pair_item0(std::max(npairs, 1), 0), pair_nitems(std::max(npairs, 1), 0),
      pair_jj(std::max(npairs, 1), 0);
  int64_t nslots = 0;
  int Gmax = 1;
  for (int f = 0; f < nframes; ++f) {
    const int npf = src_begin[f + 1] - src_begin[f];
    // at most BWL_VMAX pairs per group: the pipelined kernel stages a group's pairs at once
    const int Gf = std::max({1, std::min(G, npf), (npf + BWL_VMAX - 1) / BWL_VMAX});
    frame_groups[f] = Gf;
    Gmax = std::max(Gmax, Gf);
    for (int g = 0; g < Gf; ++g) {
      const int jb = int(int64_t(g) * npf / Gf), je = int(int64_t(g + 1) * npf / Gf);
      const int32_t it0 = int32_t(items.size());
      for (int64_t t = 0; t < ntiles[f]; ++t) {
        items.push_back(make_int4(f, int32_t(t * BWD_TILE), src_begin[f] + jb, je - jb));
        item_grp.push_back(g);
        item_slot.push_back(nslots);
        nslots += je - jb;
      }
      for (int j = jb; j < je; ++j) {
        const int q = src_list[src_begin[f] + j];
        pair_item0[q] = it0;
        pair_nitems[q] = int32_t(ntiles[f]);
        pair_jj[q] = j - jb;
      }
    }
  }
  (void)pos;
  if (src_list.empty()) src_list.push_back(0);
  sc.nitems = int(items.size());
  if (items.empty()) {
    items.push_back(make_int4(0, 0, 0, 0));
    item_grp.push_back(0);
    item_slot.push_back(0);
  }
  sc.ntot = frame_off[nframes];
  sc.nslots = nslots;
  sc.groups = Gmax;
  int per_sm = 1;
  GLIM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_items, BWD_BLOCK, 0));
  sc.grid = std::max(1, std::min(std::max(per_sm, 1) * ctx->num_sms, std::max(sc.nitems, 1)));
  if (const int per_sm_lane = backward_lane_occupancy(p))
    sc.grid_lane = std::max(1, std::min(per_sm_lane * ctx->num_sms, std::max(sc.nitems, 1)));
  const size_t npp = Gmax > 1 ? size_t(Gmax) * size_t(std::max<int64_t>(sc.ntot, 1)) : 0;
  const size_t view_bytes = std::max(sizeof(BwlView<false>), sizeof(BwlView<true>));
  if (dmalloc(&sc.items, items.size() * sizeof(int4)) != cudaSuccess ||
      dmalloc(&sc.item_grp, item_grp.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.item_slot, item_slot.size() * sizeof(int64_t)) != cudaSuccess ||
      dmalloc(&sc.src_begin, src_begin.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.src_list, src_list.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.pair_item0, pair_item0.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.pair_nitems, pair_nitems.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.pair_jj, pair_jj.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.tgt, tgt.size() * sizeof(int32_t)) != cudaSuccess ||
      dmalloc(&sc.frame_off, frame_off.size() * sizeof(int64_t)) != cudaSuccess ||
      dmalloc(&sc.frame_groups, frame_groups.size() * sizeof(int32_t)) != cudaSuccess ||
      (npp > 0 && dmalloc(&sc.pp, npp * sizeof(float4)) != cudaSuccess) ||
      dmalloc(&sc.part, size_t(std::max<int64_t>(nslots, 1)) * BSTRIDE * sizeof(double)) != cudaSuccess ||
      dmalloc(&sc.pair_grad, size_t(std::max(npairs, 1)) * 12 * sizeof(double)) != cudaSuccess ||
      dmalloc(&sc.head, sizeof(int)) != cudaSuccess ||
      (sc.grid_lane > 0 && dmalloc(&sc.views, size_t(std::max(npairs, 1)) * view_bytes) != cudaSuccess)) {
    sc.release();
    return set_error(ctx, GLIM_ENOMEM, "backward: scratch allocation failed");
  }
  cudaError_t e = cudaMemcpy(sc.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(sc.item_grp, item_grp.data(), item_grp.size() * sizeof(int32_t));
  up(sc.item_slot, item_slot.data(), item_slot.size() * sizeof(int64_t));
  up(sc.src_begin, src_begin.data(), src_begin.size() * sizeof(int32_t));
  up(sc.src_list, src_list.data(), src_list.size() * sizeof(int32_t));
  up(sc.pair_item0, pair_item0.data(), pair_item0.size() * sizeof(int32_t));
  up(sc.pair_nitems, pair_nitems.data(), pair_nitems.size() * sizeof(int32_t));
  up(sc.pair_jj, pair_jj.data(), pair_jj.size() * sizeof(int32_t));
  up(sc.tgt, tgt.data(), tgt.size() * sizeof(int32_t));
  up(sc.frame_off, frame_off.data(), frame_off.size() * sizeof(int64_t));
  up(sc.frame_groups, frame_groups.data(), frame_groups.size() * sizeof(int32_t));
  if (e != cudaSuccess) {
    sc.release();
    return cuda_check(ctx, e, "backward: table upload");
  }
  return GLIM_OK;
}

// The gradient kernels of a batch whose poses are already uploaded into p->d_in (no wait).
glim_status bwd_run(glim_plan* p, const BwdScratch& sc, int32_t omega_grad_full, int32_t validate_surface,
                    double* dxi_out, float* dmu_out, float* dw_out) {
  glim_ctx* ctx = p->ctx;
  const int npairs = p->npairs, nframes = p->nframes;
  if (sc.nitems > 0) {
    BwdArgs a;
    a.items = sc.items;
    a.item_grp = sc.item_grp;
    a.item_slot = sc.item_slot;
    a.nitems = sc.nitems;
    a.head = sc.head;
    a.pairs = p->d_pairs;
    a.frames = p->d_frames;
    a.maps = p->d_maps;
    a.dmaps = p->d_dmaps;
    a.hmaps = p->d_hmaps;
    a.pose = p->in_pose32();
    a.src_list = sc.src_list;
    a.frame_off = sc.frame_off;
    a.ntot = sc.ntot;
    a.validate = validate_surface;
    a.full = omega_grad_full;
    a.part = sc.part;
    a.pp = sc.groups > 1 ? sc.pp : nullptr;
    a.dmu = dmu_out;
    a.dw = dw_out;
    GLIM_CUDA(ctx, cudaMemsetAsync(sc.head, 0, sizeof(int), ctx->stream));
    bool lane = false;
    if (sc.grid_lane > 0)
      lane = p->d_dmaps ? launch_backward_lane_t<false>(p, sc, a, ctx->stream)
                        : launch_backward_lane_t<true>(p, sc, a, ctx->stream);
    if (!lane) k_backward_items<<<sc.grid, BWD_BLOCK, 0, ctx->stream>>>(a);
    else if (npairs > 0) ctx->launches++;  // the views
    GLIM_LAUNCHED(ctx);
  }
  if (sc.groups > 1 && sc.ntot > 0 && (dmu_out || dw_out)) {
    k_backward_points<<<ceil_div_i(sc.ntot, 256), 256, 0, ctx->stream>>>(sc.pp, sc.frame_off, sc.frame_groups, nframes,
                                                                         sc.ntot, dmu_out, dw_out);
    GLIM_LAUNCHED(ctx);
  }
  if (npairs > 0) {
    k_backward_pairs<<<ceil_div_i(npairs, 64), 64, 0, ctx->stream>>>(sc.part, sc.item_slot, sc.pair_item0,
                                                                     sc.pair_nitems, sc.pair_jj, p->in_pose64(), npairs,
                                                                     sc.pair_grad);
    GLIM_LAUNCHED(ctx);
  }
  if (nframes > 0) {
    k_backward_frames<<<ceil_div_i(nframes, 64), 64, 0, ctx->stream>>>(sc.pair_grad, p->d_pairs, sc.tgt, npairs,
                                                                       nframes, dxi_out);
    GLIM_LAUNCHED(ctx);
  }
  // the outputs are device arrays ordered on the context stream: no host wait here
  ctx->err.clear();
  return GLIM_OK;
}

}  // namespace

extern "C" glim_status glim_backward(glim_ctx* ctx, const glim_frame* frames, int32_t nframes, const glim_pair* pairs,
                                     int32_t npairs, const double* poses12, int32_t omega_grad_full,
                                     int32_t validate_surface, double* dxi_out, float* dmu_out, float* dw_out) {
  GLIM_RANGE("glim_backward");
  if (!ctx) return GLIM_EINVAL;
  if (!poses12 || (nframes > 0 && !dxi_out)) return set_error(ctx, GLIM_EINVAL, "backward: null argument");
  glim_lin_opts o{};
  o.accum_mode = GLIM_ACC_FP64;
  o.validate_surface = validate_surface;
  glim_plan* p = nullptr;
  glim_status st = glim_plan_create(ctx, frames, nframes, pairs, npairs, &o, &p);
  if (st != GLIM_OK) return st;
  BwdScratch sc;
  st = bwd_prepare(p, sc);
  if (st == GLIM_OK) {
    st = plan_upload_poses(p, poses12);
  }
  if (st == GLIM_OK) st = bwd_run(p, sc, omega_grad_full, validate_surface, dxi_out, dmu_out, dw_out);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && st == GLIM_OK)
    st = set_error(ctx, GLIM_ECUDA, "backward: sync failed");
  sc.release();
  glim_plan_destroy(p);
  return st;
}

extern "C" glim_status glim_plan_backward(glim_plan* p, const double* poses12, int32_t omega_grad_full,
                                          double* dxi_out, float* dmu_out, float* dw_out) {
  GLIM_RANGE("glim_plan_backward");
  if (!p || !poses12) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  if (p->nframes > 0 && !dxi_out) return set_error(ctx, GLIM_EINVAL, "plan_backward: null argument");
  if (!plan_maps_current(p)) return set_error(ctx, GLIM_EINVAL, "plan_backward: a target voxelmap changed");
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  // The device pose block already holds these poses when the last linearization of the plan
  // used them (the usual forward-then-gradient sequence): then nothing is uploaded and the
  // call does not wait for the stream.  Otherwise the pinned staging block may still be read
  // by an earlier upload, so the stream is drained before it is overwritten.
  const bool same_poses = p->fposes_on_device && p->nframes > 0 &&
                          std::memcmp(p->h_fposes, poses12, size_t(p->nframes) * 12 * sizeof(double)) == 0;
  if (!same_poses) GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (!p->bwd) {
    BwdScratch* sc = new BwdScratch;
    const glim_status st = bwd_prepare(p, *sc);
    if (st != GLIM_OK) {
      delete sc;
      return st;
    }
    p->bwd = sc;
  }
  if (!same_poses) {
    const glim_status st = plan_upload_poses(p, poses12);
    if (st != GLIM_OK) return st;
  }
  return bwd_run(p, *p->bwd, omega_grad_full, p->opts.validate_surface, dxi_out, dmu_out, dw_out);
}
