// linearize.cu -- batched linearization of matching-cost factors (Sec. III-C "Linearization"
// and "Implementation"), the hot path of the library.
//
// Work decomposition: every factor (pair) is cut into tiles of block * pts_per_thread source
// points; a work item is (pair, tile).  A persistent kernel with one resident wave of blocks
// takes items from an atomic queue; each block reduces its item to 28 partial sums plus an
// inlier count and writes them to the item's own slot (no float atomics, so results repeat
// bit for bit).  A second kernel sums each pair's slots in a fixed order in FP64 and expands
// them into e, H (12 x 12) and b (12).
//
// Per point (FP32): the pinned transform q = R mu + t, u = R mu, the rotated covariance
// R C R^T once for all levels, then per level the voxel key, one hash probe sequence and, on
// a hit, S = C~ + R C R^T, Omega = S^-1 (adjugate / determinant), d = mu~ - q, e = d^T Omega d.
// Across levels the point keeps Omega_sum = sum w Omega, g_sum = sum w Omega d, e_sum.
//
// Per-point quadratic factor in 28 numbers: with G = [-(u)x, I] (3 x 6), which is the same
// for every level of a point,
//     A_k = -G diag(R, R),   B_k = G S_t,   S_t = [[I, 0], [-(t)x, I]]
// (Eqs. (4)-(5); u x R = R (mu)x and q = u + t).  Hence with Lift = [-diag(R,R), S_t] (6 x 12)
//     H = Lift^T M Lift,  b = Lift^T g,   M = sum G^T Omega_sum G,   g = sum G^T g_sum,
// so a point accumulates the 21 unique entries of M (blocks -u x Omega u x, u x Omega, Omega),
// the 6 entries of g ([u x g_sum; g_sum]) and e: 28 accumulators instead of the 91 of H and b.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lin_kernel.cuh"

namespace {

// ---------------------------------------------------------------- FP64 reduce + expand
struct ReduceArgs {
  const double* part;
  const int32_t* item_begin;  // npairs + 1 (items of pair p are item_begin[p] .. item_begin[p+1]-1)
  const double* pose64;       // per pair: R (9), t (3) of T_rel in FP64
  int32_t pair_base;
  int32_t npairs;
  int32_t fp32_sum;           // 1: sum the partials in FP32 (naive mode)
  double* e;
  double* H;
  double* b;
  long long* inl;
  double* rec = nullptr;  // optional: per pair the GLIM_RECORD_DOUBLES-double factor record
};

__global__ void __launch_bounds__(128) k_reduce_expand(const ReduceArgs a) {
  const int p = a.pair_base + blockIdx.x;
  if (p >= a.npairs) return;
  __shared__ double s[PSTRIDE];
  __shared__ double M[6][6], g[6], L[6][12], T[6][12];
  const int tid = threadIdx.x;
  const int ib = a.item_begin[p], ie = a.item_begin[p + 1];
  if (tid <= NACC) {
    if (a.fp32_sum) {
      float t = 0.f;
      for (int i = ib; i < ie; ++i) t += float(a.part[int64_t(i) * PSTRIDE + tid]);
      s[tid] = double(t);
    } else {
      double t = 0.0;
      for (int i = ib; i < ie; ++i) t += a.part[int64_t(i) * PSTRIDE + tid];
      s[tid] = t;
    }
  }
  // Lift = [-diag(R, R), S_t],  S_t = [[I, 0], [-(t)x, I]]
  const double* P = a.pose64 + 12 * int64_t(p);
  if (tid < 72) {
    const int r = tid / 12, c = tid % 12;
    double v = 0.0;
    if (c < 6) {
      if ((r < 3) == (c < 3)) v = -P[3 * (r % 3) + (c % 3)];
    } else {
      const int cc = c - 6;
      if (r == cc) v = 1.0;
      else if (r >= 3 && cc < 3) {
        const double tx = P[9], ty = P[10], tz = P[11];
        // -(t)x = [[0, tz, -ty], [-tz, 0, tx], [ty, -tx, 0]]
        const double neg_hat[3][3] = {{0.0, tz, -ty}, {-tz, 0.0, tx}, {ty, -tx, 0.0}};
        v = neg_hat[r - 3][cc];
      }
    }
    L[r][c] = v;
  }
  __syncthreads();
  if (tid < 36) {
    // M from the 21 unique sums: [[M_rr, M_rt], [M_rt^T, M_tt]]
    const int r = tid / 6, c = tid % 6;
    const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double v;
    if (r < 3 && c < 3) v = s[sym[r][c]];
    else if (r < 3) v = s[6 + 3 * r + (c - 3)];
    else if (c < 3) v = s[6 + 3 * c + (r - 3)];
    else v = s[15 + sym[r - 3][c - 3]];
    M[r][c] = v;
  } else if (tid < 42) {
    g[tid - 36] = s[21 + (tid - 36)];
  }
  __syncthreads();
  if (tid < 72) {  // T = M Lift
    const int r = tid / 12, c = tid % 12;
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) v += M[r][k] * L[k][c];
    T[r][c] = v;
  }
  __syncthreads();
  // H = Lift^T T: the 78 entries of the upper triangle (row-major, r <= c), each mirrored,
  // so that H is exactly symmetric and its record holds every entry
  double* rec = a.rec ? a.rec + int64_t(p) * GLIM_RECORD_DOUBLES : nullptr;
  for (int i = tid; i < 78; i += blockDim.x) {
    int r = 0, rem = i;
    while (rem >= 12 - r) {  // i-th entry of the row-major upper triangle
      rem -= 12 - r;
      ++r;
    }
    const int c = r + rem;
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) v += L[k][r] * T[k][c];
    a.H[int64_t(p) * 144 + r * 12 + c] = v;
    a.H[int64_t(p) * 144 + c * 12 + r] = v;
    if (rec) rec[1 + i] = v;
  }
  if (tid < 12) {  // b = Lift^T g
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) v += L[k][tid] * g[k];
    a.b[int64_t(p) * 12 + tid] = v;
    if (rec) rec[79 + tid] = v;
  }
  if (tid == 0) {
    a.e[p] = s[27];
    const long long n_in = (long long)(s[NACC] + 0.5);
    if (a.inl) a.inl[p] = n_in;
    if (rec) {
      rec[0] = s[27];
      rec[91] = double(n_in);
    }
  }
}

// ---------------------------------------------------------------- kernel table
LinKernelInfo pick_kernel(int block, int acc, int lmax, int lane) {
  if (lane == 1) {
    switch (acc) {
      case GLIM_ACC_FP32: return pick_lin_dense_fp32(block, lmax);
      case GLIM_ACC_KAHAN: return pick_lin_dense_kahan(block, lmax);
      case GLIM_ACC_FP64: return pick_lin_dense_fp64(block, lmax);
    }
    return LinKernelInfo{};
  }
  if (lane == 2) {
    switch (acc) {
      case GLIM_ACC_FP32: return pick_lin_hash_fp32(block, lmax);
      case GLIM_ACC_KAHAN: return pick_lin_hash_kahan(block, lmax);
      case GLIM_ACC_FP64: return pick_lin_hash_fp64(block, lmax);
    }
    return LinKernelInfo{};
  }
  switch (acc) {
    case GLIM_ACC_FP32: return pick_lin_fp32(block, lmax);
    case GLIM_ACC_KAHAN: return pick_lin_kahan(block, lmax);
    case GLIM_ACC_FP64: return pick_lin_fp64(block, lmax);
  }
  return LinKernelInfo{};
}

void fill_defaults(glim_lin_opts& o) {
  if (o.block == 0) o.block = 256;
  if (o.pts_per_thread == 0) o.pts_per_thread = 16;
  if (o.persistent == 0) o.persistent = 1;
}

bool opts_valid(const glim_lin_opts& o) {
  return (o.block == 64 || o.block == 128 || o.block == 256) &&
         (o.pts_per_thread >= 1 && o.pts_per_thread <= 256) &&
         (o.accum_mode >= 0 && o.accum_mode <= 2) && (o.persistent == 1 || o.persistent == 2) &&
         o.blocks_per_sm >= 0 && o.blocks_per_sm <= 32 && o.kernel >= 0 && o.kernel <= 3;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace {

void drop_graphs(glim_plan* p) {
  if (p->g_full) cudaGraphExecDestroy(p->g_full);
  if (p->g_dev) cudaGraphExecDestroy(p->g_dev);
  p->g_full = p->g_dev = nullptr;
  gn_graph_free(p->gn);
  p->gn = nullptr;
}

}  // namespace

glim_status plan_configure(glim_plan* p, const glim_lin_opts& o) {
  glim_ctx* ctx = p->ctx;
  // Everything that can fail comes first; the plan changes only once all of it succeeded, so
  // a failed reconfiguration (an autotuner candidate that meets an out-of-memory condition)
  // leaves a plan that still launches its previous configuration.
  if (o.kernel == 2 && !p->d_dmaps)
    return set_error(ctx, GLIM_EINVAL,
                     "the dense-grid kernel needs every target level to be a dense grid and resolutions doubling per level");
  if (o.kernel == 3 && !p->d_hmaps)
    return set_error(ctx, GLIM_EINVAL,
                     "the hash kernel needs every target level to be a hash table and resolutions doubling per level");
  const int lane = o.kernel == 1 ? 0 : (p->d_dmaps ? 1 : (p->d_hmaps ? 2 : 0));
  const LinKernelInfo ki = pick_kernel(o.block, o.accum_mode, p->lmax, lane);
  if (!ki.fn) return set_error(ctx, GLIM_EINVAL, "no kernel for block=%d ppt=%d acc=%d", o.block, o.pts_per_thread, o.accum_mode);
  GLIM_CUDA(ctx, cudaFuncSetAttribute(reinterpret_cast<const void*>(ki.fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(ki.smem)));
  const int tile = o.block * o.pts_per_thread;
  std::vector<Item> items;
  std::vector<int32_t> begin(p->npairs + 1, 0);
  for (int q = 0; q < p->npairs; ++q) {
    begin[q] = int32_t(items.size());
    const int64_t n = p->frames[p->pairs[q].src_frame].n;
    for (int64_t s = 0; s < n; s += tile) items.push_back(Item{q, int32_t(s)});
  }
  begin[p->npairs] = int32_t(items.size());
  const int nitems = int(items.size());
  int grid = std::max(1, nitems);
  if (o.persistent == 1) {
    int per_sm = o.blocks_per_sm;
    if (per_sm == 0) {
      GLIM_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, o.block, ki.smem));
      per_sm = std::max(per_sm, 1);
    }
    grid = std::max(1, std::min(per_sm * ctx->num_sms, nitems));
  }
  const size_t ni = std::max<size_t>(items.size(), 1);
  Item* d_items = nullptr;
  int32_t* d_begin = nullptr;
  double* d_part = nullptr;
  cudaError_t e = dmalloc(&d_items, ni * sizeof(Item));
  if (e == cudaSuccess) e = dmalloc(&d_begin, begin.size() * sizeof(int32_t));
  if (e == cudaSuccess) e = dmalloc(&d_part, ni * PSTRIDE * sizeof(double));
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_begin, begin.data(), begin.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d_items);
    cudaFree(d_begin);
    cudaFree(d_part);
    return cuda_check(ctx, e, "plan: work list");
  }
  // commit; launches in flight may still read the previous work list
  cudaStreamSynchronize(ctx->stream);
  drop_graphs(p);
  cudaFree(p->d_items);
  cudaFree(p->d_item_begin);
  cudaFree(p->d_part);
  p->d_items = d_items;
  p->d_item_begin = d_begin;
  p->d_part = d_part;
  p->opts = o;
  p->tile = tile;
  p->nitems = nitems;
  p->lane_kernel = lane;
  p->opts.kernel = lane == 1 ? 2 : (lane == 2 ? 3 : 1);  // the kernel actually used
  p->kernel = ki.fn;
  p->kernel_smem = ki.smem;
  p->grid = grid;
  return GLIM_OK;
}

namespace {

// Enqueue queue reset + linearize + reduce on the ctx stream (no sync); with slot >= 0,
// record that timing slot's events around the linearization kernel.
glim_status plan_enqueue_kernels(glim_plan* p, int slot = -1) {
  glim_ctx* ctx = p->ctx;
  if (p->nitems > 0) {
    LinArgs a;
    a.items = p->d_items;
    a.nitems = p->nitems;
    a.item_base = 0;
    a.pairs = p->d_pairs;
    a.frames = p->d_frames;
    a.maps = p->d_maps;
    a.dmaps = p->lane_kernel == 1 ? p->d_dmaps : nullptr;
    a.hmaps = p->lane_kernel == 2 ? p->d_hmaps : nullptr;
    a.pose = p->in_pose32();
    a.head = p->opts.persistent == 1 ? p->d_head : nullptr;
    a.part = p->d_part;
    a.tile = p->tile;
    a.ppt = p->opts.pts_per_thread;
    a.validate = p->opts.validate_surface;
    if (p->opts.persistent == 1) GLIM_CUDA(ctx, cudaMemsetAsync(p->d_head, 0, sizeof(int), ctx->stream));
    if (slot >= 0) GLIM_CUDA(ctx, cudaEventRecord(p->ev[2 * slot], ctx->stream));
    p->kernel<<<p->grid, p->opts.block, p->kernel_smem, ctx->stream>>>(a);
    GLIM_LAUNCHED(ctx);
    if (slot >= 0) GLIM_CUDA(ctx, cudaEventRecord(p->ev[2 * slot + 1], ctx->stream));
  }
  ReduceArgs r;
  r.part = p->d_part;
  r.item_begin = p->d_item_begin;
  r.pose64 = p->in_pose64();
  r.pair_base = 0;
  r.npairs = p->npairs;
  r.fp32_sum = p->opts.accum_mode == GLIM_ACC_FP32 ? 1 : 0;
  r.e = p->out_e();
  r.H = p->out_H();
  r.b = p->out_b();
  r.inl = p->out_inl();
  r.rec = p->d_rec;
  if (p->npairs > 0) {
    k_reduce_expand<<<p->npairs, 128, 0, ctx->stream>>>(r);
    GLIM_LAUNCHED(ctx);
  }
  return GLIM_OK;
}

}  // namespace

LinKernelInfo pick_lin_kernel(int block, int acc, int lmax, int lane) { return pick_kernel(block, acc, lmax, lane); }

// The per-lane kernels take the key of level l as the level-0 key shifted right by l, which
// is floor(q * inv_r_l) exactly when inv_r_l = inv_r_0 2^-l (a power-of-two scaling of an
// FP32 product is exact, and floor(floor(x) / 2^l) = floor(x / 2^l)); maps whose resolutions
// do not double from level to level run the general kernel.
static bool map_pow2(const glim_vmap* m) {
  for (int l = 1; l < m->levels; ++l)
    if (m->inv_r[l] != std::ldexp(m->inv_r[0], -l)) return false;
  return true;
}

bool map_all_dense(const glim_vmap* m) {
  for (int l = 0; l < m->levels; ++l)
    if (!m->dense[l] || !m->slots[l]) return false;
  return map_pow2(m);
}

bool map_all_hash(const glim_vmap* m) {
  for (int l = 0; l < m->levels; ++l)
    if (m->dense[l] || !m->slots[l] || !m->btab[l] || m->max_probe[l] < 1) return false;
  return map_pow2(m);
}

void fill_dense_map(const glim_vmap* m, DenseMapDev& d) {
  std::memset(&d, 0, sizeof(DenseMapDev));
  for (int l = 0; l < GLIM_MAX_LEVELS; ++l) {
    DenseLevelDev& v = d.lv[l];
    if (l < m->levels) {
      v.cells = m->slots[l];
      v.ox = m->org[l][0];
      v.oy = m->org[l][1];
      v.oz = m->org[l][2];
      v.nx = m->dim[l][0];
      v.ny = m->dim[l][1];
      v.nz = m->dim[l][2];
      d.inv_r[l] = m->inv_r[l];
    } else {  // an absent level: empty box, reads level 0's empty record
      v.cells = m->slots[0];
      d.inv_r[l] = m->inv_r[0];
    }
  }
}

void fill_hash_map(const glim_vmap* m, const VoxSlot* empty16, HashMapDev& d) {
  std::memset(&d, 0, sizeof(HashMapDev));
  for (int l = 0; l < GLIM_MAX_LEVELS; ++l) {
    HashLevelDev& v = d.lv[l];
    if (l < m->levels) {
      v.slots = m->slots[l];
      v.btab = m->btab[l];
      v.mask = uint32_t(m->cap[l] - 1);
      v.log2cap = m->log2cap[l];
      v.max_probe = m->max_probe[l];
      d.inv_r[l] = m->inv_r[l];
    } else {  // an absent level: an all-empty table of 16 entries, and its empty record
      v.slots = empty16 + 1;
      v.btab = reinterpret_cast<const int4*>(empty16);
      v.mask = 15u;
      v.log2cap = 4;
      v.max_probe = 1;
      d.inv_r[l] = m->inv_r[0];
    }
  }
}

// The plan holds device pointers to its maps' tables; a map freed since, or changed (an
// insertion frees and replaces its tables), makes the plan unusable.  A freed map is
// recognised through the registry of live maps, without reading the freed object; the
// per-map check runs only when the registry's epoch moved since the last check.
bool plan_maps_current(glim_plan* p) {
  const uint64_t epoch = vmap_epoch();
  if (epoch == p->maps_checked_epoch) return true;
  for (const auto& mv : p->map_versions)
    if (!vmap_alive(mv.m, mv.serial) || mv.m->version != mv.version) return false;
  p->maps_checked_epoch = epoch;
  return true;
}

namespace {

// S0 on the device: T_rel = T_t^-1 T_s in FP64 for every pair, its FP32 rounding and the
// target viewpoint v = -R^T t.  Every product and sum is rounded on its own, in the order of
// the host helpers relative_pose / pose_to_f32 (no fused multiply-add), so the results are
// the same bits as the host's.
__global__ void k_pack_poses(const double* __restrict__ fposes, const int2* __restrict__ pair_frames, int npairs,
                             PoseF* __restrict__ pose32, double* __restrict__ pose64) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npairs) return;
  const int2 f = pair_frames[q];
  const double* s = fposes + 12 * int64_t(f.x);
  const double* t = fposes + 12 * int64_t(f.y);
  double R[9], tr[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v = __dadd_rn(v, __dmul_rn(t[4 * k + i], s[4 * k + j]));
      R[3 * i + j] = v;
    }
  const double dt[3] = {__dsub_rn(s[3], t[3]), __dsub_rn(s[7], t[7]), __dsub_rn(s[11], t[11])};
  for (int i = 0; i < 3; ++i)
    tr[i] = __dadd_rn(__dadd_rn(__dmul_rn(t[i], dt[0]), __dmul_rn(t[4 + i], dt[1])), __dmul_rn(t[8 + i], dt[2]));
  PoseF o;
  for (int i = 0; i < 9; ++i) o.R[i] = __double2float_rn(R[i]);
  for (int i = 0; i < 3; ++i) {
    o.t[i] = __double2float_rn(tr[i]);
    double v = 0.0;
    for (int k = 0; k < 3; ++k) v = __dadd_rn(v, __dmul_rn(R[3 * k + i], tr[k]));
    o.v[i] = __double2float_rn(-v);
  }
  o.pad = 0.f;
  pose32[q] = o;
  double* d = pose64 + 12 * int64_t(q);
  for (int i = 0; i < 9; ++i) d[i] = R[i];
  for (int i = 0; i < 3; ++i) d[9 + i] = tr[i];
}

}  // namespace

void plan_stage_poses(glim_plan* p, const double* poses12) {
  p->fposes_on_device = false;
  std::memcpy(p->h_fposes, poses12, size_t(p->nframes) * 12 * sizeof(double));
}

glim_status plan_enqueue_poses(glim_plan* p) {
  glim_ctx* ctx = p->ctx;
  if (p->npairs == 0) return GLIM_OK;
  GLIM_CUDA(ctx, cudaMemcpyAsync(p->d_fposes, p->h_fposes, size_t(p->nframes) * 12 * sizeof(double),
                                 cudaMemcpyHostToDevice, ctx->stream));
  k_pack_poses<<<ceil_div_i(p->npairs, 128), 128, 0, ctx->stream>>>(p->d_fposes, p->d_pair_frames, p->npairs,
                                                                     p->in_pose32(), p->in_pose64());
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}

namespace {

glim_status maps_current(glim_plan* p) {
  if (!plan_maps_current(p))
    return set_error(p->ctx, GLIM_EINVAL, "plan: a target voxelmap changed after the plan was created");
  return GLIM_OK;
}

glim_status capture(glim_plan* p, bool full, cudaGraphExec_t* out) {
  glim_ctx* ctx = p->ctx;
  cudaGraph_t g = nullptr;
  GLIM_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  glim_status st = GLIM_OK;
  if (full) st = plan_enqueue_poses(p);
  if (st == GLIM_OK) st = plan_enqueue_kernels(p);
  if (st == GLIM_OK && full &&
      cudaMemcpyAsync(p->h_out, p->d_out, p->out_bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    st = GLIM_ECUDA;
  cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
  if (st != GLIM_OK) {
    if (g) cudaGraphDestroy(g);
    return st == GLIM_ECUDA ? set_error(ctx, st, "graph capture failed") : st;
  }
  if (ce != cudaSuccess) return cuda_check(ctx, ce, "cudaStreamEndCapture");
  ce = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return cuda_check(ctx, ce, "cudaGraphInstantiate");
  return GLIM_OK;
}

glim_status copy_outputs(glim_plan* p, double* e_out, double* H_out, double* b_out, int64_t* inl_out, bool from_host) {
  glim_ctx* ctx = p->ctx;
  const int P = p->npairs;
  if (from_host) {
    const char* base = reinterpret_cast<const char*>(p->h_out);
    std::memcpy(e_out, base, P * sizeof(double));
    std::memcpy(H_out, base + P * sizeof(double), size_t(P) * 144 * sizeof(double));
    std::memcpy(b_out, base + size_t(P) * 145 * sizeof(double), size_t(P) * 12 * sizeof(double));
    if (inl_out) std::memcpy(inl_out, base + size_t(P) * 157 * sizeof(double), P * sizeof(int64_t));
    return GLIM_OK;
  }
  GLIM_CUDA(ctx, cudaMemcpyAsync(e_out, p->out_e(), P * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(H_out, p->out_H(), size_t(P) * 144 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(b_out, p->out_b(), size_t(P) * 12 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (inl_out)
    GLIM_CUDA(ctx, cudaMemcpyAsync(inl_out, p->out_inl(), P * sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx->stream));
  return GLIM_OK;
}

glim_status validate_batch(glim_ctx* ctx, const glim_frame* frames, int32_t nframes, const glim_pair* pairs,
                           int32_t npairs) {
  if (nframes < 0 || npairs < 0 || (nframes > 0 && !frames) || (npairs > 0 && !pairs))
    return set_error(ctx, GLIM_EINVAL, "linearize: bad batch sizes");
  for (int f = 0; f < nframes; ++f) {
    const glim_frame& F = frames[f];
    if (F.n < 0 || F.n > 0x7FFFFFFFll || (F.n > 0 && (!F.pts4 || !F.cov6)))
      return set_error(ctx, GLIM_EINVAL, "linearize: frame %d has bad size or null arrays", f);
    if ((reinterpret_cast<uintptr_t>(F.pts4) & 15) || (reinterpret_cast<uintptr_t>(F.cov6) & 7))
      return set_error(ctx, GLIM_EINVAL, "linearize: frame %d arrays misaligned", f);
  }
  for (int q = 0; q < npairs; ++q) {
    const glim_pair& P = pairs[q];
    if (P.src_frame < 0 || P.src_frame >= nframes || P.tgt_frame < 0 || P.tgt_frame >= nframes || !P.tgt)
      return set_error(ctx, GLIM_EINVAL, "linearize: pair %d is invalid", q);
    if (P.tgt->device != ctx->device) return set_error(ctx, GLIM_EINVAL, "linearize: pair %d map on another device", q);
  }
  return GLIM_OK;
}

}  // namespace

extern "C" glim_status glim_plan_create(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                        const glim_pair* pairs, int32_t npairs, const glim_lin_opts* opts,
                                        glim_plan** out) {
  GLIM_RANGE("glim_plan_create");
  if (!ctx || !out) return GLIM_EINVAL;
  *out = nullptr;
  glim_status st = validate_batch(ctx, frames, nframes, pairs, npairs);
  if (st != GLIM_OK) return st;
  glim_lin_opts o{};
  if (opts) o = *opts;
  fill_defaults(o);
  if (!opts_valid(o)) return set_error(ctx, GLIM_EINVAL, "linearize: invalid options");
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  glim_plan* p = new glim_plan;
  p->ctx = ctx;
  p->nframes = nframes;
  p->npairs = npairs;
  p->frames.assign(frames, frames + nframes);
  p->pairs.assign(pairs, pairs + npairs);
  // frames and maps
  std::vector<FrameDev> fd(std::max(nframes, 1));
  for (int f = 0; f < nframes; ++f) {
    fd[f].pts = reinterpret_cast<const float4*>(frames[f].pts4);
    fd[f].cov = reinterpret_cast<const float2*>(frames[f].cov6);
    fd[f].nrm = frames[f].normal3;
    fd[f].n = frames[f].n;
  }
  std::vector<const glim_vmap*> maps;
  std::vector<PairDev> pd(std::max(npairs, 1));
  for (int q = 0; q < npairs; ++q) {
    auto it = std::find(maps.begin(), maps.end(), pairs[q].tgt);
    if (it == maps.end()) {
      maps.push_back(pairs[q].tgt);
      it = maps.end() - 1;
    }
    pd[q].src = pairs[q].src_frame;
    pd[q].map = int32_t(it - maps.begin());
  }
  std::vector<MapDev> md(std::max<size_t>(maps.size(), 1));
  for (size_t i = 0; i < maps.size(); ++i) {
    std::memset(&md[i], 0, sizeof(MapDev));
    md[i].levels = maps[i]->levels;
    md[i].pow2 = 1;
    for (int l = 0; l < maps[i]->levels; ++l) {
      md[i].lv[l] = maps[i]->dev(l);
      if (maps[i]->inv_r[l] != std::ldexp(maps[i]->inv_r[0], -l)) md[i].pow2 = 0;
    }
  }
  // per-lane kernel descriptors when every level of every target map is a dense grid, or
  // every one a hash table
  bool all_dense = !maps.empty(), all_hash = !maps.empty();
  for (const glim_vmap* m : maps) {
    all_dense = all_dense && map_all_dense(m);
    all_hash = all_hash && map_all_hash(m);
  }
  // the per-lane kernels index points in 32 bits, up to two blocks past an item's end
  for (int f = 0; f < nframes; ++f)
    if (frames[f].n > 0x7FFFFFFFll - (1 << 17)) all_dense = all_hash = false;
  std::vector<DenseMapDev> dmd(std::max<size_t>(maps.size(), 1));
  if (all_dense)
    for (size_t i = 0; i < maps.size(); ++i) fill_dense_map(maps[i], dmd[i]);
  std::vector<HashMapDev> hmd(std::max<size_t>(maps.size(), 1));
  if (all_hash) {
    if (dmalloc(&p->d_empty_slots, 16 * sizeof(VoxSlot)) != cudaSuccess ||
        cudaMemset(p->d_empty_slots, 0x80, 16 * sizeof(VoxSlot)) != cudaSuccess) {
      glim_plan_destroy(p);
      return set_error(ctx, GLIM_ENOMEM, "plan: device allocation failed");
    }
    for (size_t i = 0; i < maps.size(); ++i) fill_hash_map(maps[i], p->d_empty_slots, hmd[i]);
  }
  p->nmaps = int(maps.size());
  for (const glim_vmap* m : maps) p->map_versions.push_back(glim_plan::MapSeen{m, m->serial, m->version});
  if (!plan_maps_current(p)) {
    glim_plan_destroy(p);
    return set_error(ctx, GLIM_EINVAL, "plan: a target voxelmap is not a live map of this library");
  }
  p->lmax = 1;
  for (const glim_vmap* m : maps) p->lmax = std::max(p->lmax, m->levels);
  auto fail = [&](glim_status s) {
    glim_plan_destroy(p);
    return s;
  };
  if (dmalloc(&p->d_frames, fd.size() * sizeof(FrameDev)) != cudaSuccess ||
      dmalloc(&p->d_pairs, pd.size() * sizeof(PairDev)) != cudaSuccess ||
      dmalloc(&p->d_maps, md.size() * sizeof(MapDev)) != cudaSuccess ||
      dmalloc(&p->d_head, sizeof(int)) != cudaSuccess)
    return fail(set_error(ctx, GLIM_ENOMEM, "plan: device allocation failed"));
  cudaMemcpy(p->d_frames, fd.data(), fd.size() * sizeof(FrameDev), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_pairs, pd.data(), pd.size() * sizeof(PairDev), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_maps, md.data(), md.size() * sizeof(MapDev), cudaMemcpyHostToDevice);
  if (all_dense) {
    if (dmalloc(&p->d_dmaps, dmd.size() * sizeof(DenseMapDev)) != cudaSuccess)
      return fail(set_error(ctx, GLIM_ENOMEM, "plan: device allocation failed"));
    cudaMemcpy(p->d_dmaps, dmd.data(), dmd.size() * sizeof(DenseMapDev), cudaMemcpyHostToDevice);
  }
  if (all_hash) {
    if (dmalloc(&p->d_hmaps, hmd.size() * sizeof(HashMapDev)) != cudaSuccess)
      return fail(set_error(ctx, GLIM_ENOMEM, "plan: device allocation failed"));
    cudaMemcpy(p->d_hmaps, hmd.data(), hmd.size() * sizeof(HashMapDev), cudaMemcpyHostToDevice);
  }
  p->in_bytes = std::max<size_t>(size_t(npairs) * (sizeof(PoseF) + 12 * sizeof(double)), 16);
  p->out_bytes = std::max<size_t>(size_t(npairs) * (157 * sizeof(double) + sizeof(int64_t)), 16);
  const size_t fpose_bytes = std::max<size_t>(size_t(nframes) * 12 * sizeof(double), 16);
  if (dmalloc(&p->d_in, p->in_bytes) != cudaSuccess || dmalloc(&p->d_out, p->out_bytes) != cudaSuccess ||
      dmalloc(&p->d_fposes, fpose_bytes) != cudaSuccess ||
      dmalloc(&p->d_pair_frames, std::max(npairs, 1) * sizeof(int2)) != cudaSuccess ||
      dmalloc(&p->d_rec, std::max<size_t>(size_t(npairs) * GLIM_RECORD_DOUBLES, 1) * sizeof(double)) != cudaSuccess ||
      hmalloc(&p->h_fposes, fpose_bytes) != cudaSuccess ||
      hmalloc(&p->h_out, p->out_bytes) != cudaSuccess)
    return fail(set_error(ctx, GLIM_ENOMEM, "plan: serialized block allocation failed"));
  {
    std::vector<int2> pf(std::max(npairs, 1), make_int2(0, 0));
    for (int q = 0; q < npairs; ++q) pf[q] = make_int2(pairs[q].src_frame, pairs[q].tgt_frame);
    cudaMemcpy(p->d_pair_frames, pf.data(), pf.size() * sizeof(int2), cudaMemcpyHostToDevice);
  }
  st = plan_configure(p, o);
  if (st != GLIM_OK) return fail(st);
  *out = p;
  ctx->err.clear();
  return GLIM_OK;
}

extern "C" void glim_plan_destroy(glim_plan* p) {
  if (!p) return;
  DeviceGuard device_guard;
  device_guard.set(p->ctx->device);
  cudaStreamSynchronize(p->ctx->stream);
  drop_graphs(p);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  cudaFree(p->d_frames);
  cudaFree(p->d_pairs);
  cudaFree(p->d_maps);
  cudaFree(p->d_dmaps);
  cudaFree(p->d_hmaps);
  cudaFree(p->d_empty_slots);
  bwd_scratch_free(p->bwd);
  cudaFree(p->d_items);
  cudaFree(p->d_item_begin);
  cudaFree(p->d_part);
  cudaFree(p->d_head);
  cudaFree(p->d_in);
  cudaFree(p->d_fposes);
  cudaFree(p->d_pair_frames);
  cudaFree(p->d_rec);
  if (p->h_fposes) cudaFreeHost(p->h_fposes);
  cudaFree(p->d_out);
  if (p->h_out) cudaFreeHost(p->h_out);
  delete p;
}

extern "C" glim_status glim_plan_set_poses(glim_plan* p, const double* poses12) {
  GLIM_RANGE("glim_plan_set_poses");
  if (!p || !poses12) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  // the pinned block may still be read by an earlier upload
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return plan_upload_poses(p, poses12);
}

namespace {

// ---------------------------------------------------------------- Gauss-Newton on the device
// S9 (Sec. III-C, "Linearization" and the Gauss-Newton step it feeds): the 6 x 6 system of one
// frame with every other frame fixed, summed over the pairs in pair order (the source block
// of the pairs whose source it is, the target block of the pairs whose target it is), and the
// batch's total cost; FP64.
__global__ void k_gn_frame_system(const double* __restrict__ e, const double* __restrict__ H,
                                  const double* __restrict__ b, const int2* __restrict__ pair_frames, int npairs,
                                  int frame, double* __restrict__ sys, double* __restrict__ cost) {
  const int i = threadIdx.x;  // 0..35: H (row-major), 36..41: b, 42: the cost
  if (i > 42) return;
  double s = 0.0;
  for (int q = 0; q < npairs; ++q) {
    const int2 f = pair_frames[q];
    if (i == 42) {
      s += e[q];
      continue;
    }
    for (int side = 0; side < 2; ++side) {  // source block, then target block
      if ((side == 0 ? f.x : f.y) != frame) continue;
      const int o = 6 * side;
      s += i < 36 ? H[144 * int64_t(q) + 12 * (o + i / 6) + o + i % 6] : b[12 * int64_t(q) + o + i - 36];
    }
  }
  if (i == 42) *cost = s;
  else sys[i] = s;
}

// xi = -H^-1 b by Cholesky (a system that is not positive definite takes no step and sets
// *status), then T_frame <- T_frame Exp(xi) with Exp(xi) = [Exp(omega) | V v] (Rodrigues; V the
// left Jacobian of SO(3)), in FP64.
__global__ void k_gn_frame_step(const double* __restrict__ sys, double* __restrict__ T, int32_t* __restrict__ status) {
  double L[6][6], x[6];
  bool ok = true;
  for (int j = 0; j < 6 && ok; ++j) {
    double d = sys[6 * j + j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !isfinite(d)) {
      ok = false;
      break;
    }
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double v = sys[6 * i + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  if (!ok) {
    *status = GLIM_ENOTPD;
    return;
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {  // L y = -b
    double v = -sys[36 + i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {  // L^T x = y
    double v = y[i];
    for (int k = i + 1; k < 6; ++k) v -= L[k][i] * x[k];
    x[i] = v / L[i][i];
  }
  const double w[3] = {x[0], x[1], x[2]}, u[3] = {x[3], x[4], x[5]};
  const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  const double K[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
  double K2[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) K2[r][c] = K[r][0] * K[0][c] + K[r][1] * K[1][c] + K[r][2] * K[2][c];
  double a, bb, cc;  // Exp(omega) = I + a K + bb K^2, V = I + bb K + cc K^2
  if (th < 1e-12) {
    a = 1.0;
    bb = 0.5;
    cc = 1.0 / 6.0;
  } else {
    a = sin(th) / th;
    bb = (1.0 - cos(th)) / (th * th);
    cc = (th - sin(th)) / (th * th * th);
  }
  double E[3][3], Vv[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) E[r][c] = (r == c ? 1.0 : 0.0) + a * K[r][c] + bb * K2[r][c];
    double v = u[r];
    for (int c = 0; c < 3; ++c) v += (bb * K[r][c] + cc * K2[r][c]) * u[c];
    Vv[r] = v;
  }
  double Rn[3][3], tn[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) Rn[r][c] = T[4 * r] * E[0][c] + T[4 * r + 1] * E[1][c] + T[4 * r + 2] * E[2][c];
    tn[r] = T[4 * r] * Vv[0] + T[4 * r + 1] * Vv[1] + T[4 * r + 2] * Vv[2] + T[4 * r + 3];
  }
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) T[4 * r + c] = Rn[r][c];
    T[4 * r + 3] = tn[r];
  }
}

}  // namespace

namespace glim_detail {

struct GnGraph {
  cudaGraphExec_t exec = nullptr;
  int frame = -1, iters = 0;
  double* sys = nullptr;   // device: the frame's 6 x 6 system and b
  double* cost = nullptr;  // device: the batch's cost per iteration
  int32_t* st = nullptr;   // device: status
  double* h_cost = nullptr;  // pinned: the costs read back by the graph
  int32_t* h_st = nullptr;   // pinned: the status read back by the graph
};

void gn_graph_free(GnGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  cudaFree(g->sys);
  cudaFree(g->cost);
  cudaFree(g->st);
  cudaFreeHost(g->h_cost);
  cudaFreeHost(g->h_st);
  delete g;
}

}  // namespace glim_detail

namespace {

// The device loop of glim_plan_gauss_newton on ctx->stream: reset, the upload of the staged
// frame poses, `iters` x (pair poses, linearization, the frame's system, step), the final pair
// poses, and the read-back of the poses (into the plan's pinned staging block), costs and status.
glim_status gn_enqueue(glim_plan* p, const GnGraph& g) {
  glim_ctx* ctx = p->ctx;
  GLIM_CUDA(ctx, cudaMemsetAsync(g.st, 0, sizeof(int32_t), ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(g.cost, 0, size_t(g.iters) * sizeof(double), ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(p->d_fposes, p->h_fposes, size_t(p->nframes) * 12 * sizeof(double),
                                 cudaMemcpyHostToDevice, ctx->stream));
  for (int it = 0; it <= g.iters; ++it) {
    if (p->npairs > 0) {  // the last packing makes the pairs' device poses follow the final frame poses
      k_pack_poses<<<ceil_div_i(p->npairs, 128), 128, 0, ctx->stream>>>(p->d_fposes, p->d_pair_frames, p->npairs,
                                                                         p->in_pose32(), p->in_pose64());
      GLIM_LAUNCHED(ctx);
    }
    if (it == g.iters) break;
    glim_status s = plan_enqueue_kernels(p);
    if (s != GLIM_OK) return s;
    k_gn_frame_system<<<1, 64, 0, ctx->stream>>>(p->out_e(), p->out_H(), p->out_b(), p->d_pair_frames, p->npairs,
                                                 g.frame, g.sys, g.cost + it);
    GLIM_LAUNCHED(ctx);
    k_gn_frame_step<<<1, 1, 0, ctx->stream>>>(g.sys, p->d_fposes + 12 * int64_t(g.frame), g.st);
    GLIM_LAUNCHED(ctx);
  }
  GLIM_CUDA(ctx, cudaMemcpyAsync(p->h_fposes, p->d_fposes, size_t(p->nframes) * 12 * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(g.h_cost, g.cost, size_t(g.iters) * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(g.h_st, g.st, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  return GLIM_OK;
}

}  // namespace

extern "C" glim_status glim_plan_gauss_newton(glim_plan* p, const double* poses12, int32_t frame, int32_t iters,
                                              double* poses12_out, double* cost_out, int32_t* status_out) {
  GLIM_RANGE("glim_plan_gauss_newton");
  if (!p || !poses12 || !poses12_out) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  if (frame < 0 || frame >= p->nframes || iters < 1)
    return set_error(ctx, GLIM_EINVAL, "plan_gauss_newton: bad frame %d or iterations %d", frame, iters);
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the pinned staging block may be in use
  if (p->gn && (p->gn->frame != frame || p->gn->iters != iters)) {
    gn_graph_free(p->gn);
    p->gn = nullptr;
  }
  if (!p->gn) {
    GnGraph* g = new GnGraph;
    g->frame = frame;
    g->iters = iters;
    if (dmalloc(&g->sys, 42 * sizeof(double)) != cudaSuccess ||
        dmalloc(&g->cost, size_t(iters) * sizeof(double)) != cudaSuccess ||
        dmalloc(&g->st, sizeof(int32_t)) != cudaSuccess ||
        hmalloc(&g->h_cost, size_t(iters) * sizeof(double)) != cudaSuccess ||
        hmalloc(&g->h_st, sizeof(int32_t)) != cudaSuccess) {
      gn_graph_free(g);
      return set_error(ctx, GLIM_ENOMEM, "plan_gauss_newton: allocation failed");
    }
    if (p->use_graph) {  // the loop as one graph, captured once per (frame, iterations)
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) {
        gn_graph_free(g);
        return cuda_check(ctx, ce, "plan_gauss_newton: begin capture");
      }
      const glim_status st = gn_enqueue(p, *g);
      ce = cudaStreamEndCapture(ctx->stream, &graph);
      if (st == GLIM_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&g->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (st != GLIM_OK || ce != cudaSuccess) {
        gn_graph_free(g);
        return st != GLIM_OK ? st : cuda_check(ctx, ce, "plan_gauss_newton: graph");
      }
    }
    p->gn = g;
  }
  plan_stage_poses(p, poses12);
  if (p->gn->exec) {
    GLIM_CUDA(ctx, cudaGraphLaunch(p->gn->exec, ctx->stream));
    ctx->launches += (p->npairs > 0 ? iters + 1 : 0) + iters * (2 + glim_plan_kernels_per_launch(p));
  } else {
    const glim_status st = gn_enqueue(p, *p->gn);
    if (st != GLIM_OK) return st;
  }
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // h_fposes now holds the final poses, which the device pose block also holds (its outputs:
  // the last linearization, at the poses before the last step)
  std::memcpy(poses12_out, p->h_fposes, size_t(p->nframes) * 12 * sizeof(double));
  p->fposes_on_device = true;
  if (cost_out) std::memcpy(cost_out, p->gn->h_cost, size_t(iters) * sizeof(double));
  if (status_out) *status_out = *p->gn->h_st;
  ctx->err.clear();
  return GLIM_OK;
}

extern "C" glim_status glim_plan_relative_poses(glim_plan* p, double* rt64_out, float* pose32_out) {
  if (!p) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  if (p->npairs == 0) return GLIM_OK;
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (rt64_out)
    GLIM_CUDA(ctx, cudaMemcpy(rt64_out, p->in_pose64(), size_t(p->npairs) * 12 * sizeof(double), cudaMemcpyDeviceToHost));
  if (pose32_out) {
    static_assert(sizeof(PoseF) == 16 * sizeof(float), "PoseF is 16 floats");
    GLIM_CUDA(ctx, cudaMemcpy(pose32_out, p->in_pose32(), size_t(p->npairs) * sizeof(PoseF), cudaMemcpyDeviceToHost));
  }
  return GLIM_OK;
}

extern "C" glim_status glim_plan_launch(glim_plan* p) {
  GLIM_RANGE("glim_plan_launch");
  if (!p) return GLIM_EINVAL;
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  if (!p->use_graph) return plan_enqueue_kernels(p);
  if (!p->g_dev) {
    glim_status st = capture(p, false, &p->g_dev);
    if (st != GLIM_OK) return st;
  }
  GLIM_CUDA(ctx, cudaGraphLaunch(p->g_dev, ctx->stream));
  ctx->launches += glim_plan_kernels_per_launch(p);
  return GLIM_OK;
}

extern "C" glim_status glim_plan_launch_timed(glim_plan* p, int32_t slot) {
  GLIM_RANGE("glim_plan_launch_timed");
  if (!p || slot < 0 || slot >= 4096) return GLIM_EINVAL;
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  while (int(p->ev.size()) < 2 * (slot + 1)) {
    cudaEvent_t e;
    GLIM_CUDA(ctx, cudaEventCreate(&e));
    p->ev.push_back(e);
  }
  return plan_enqueue_kernels(p, slot);
}

extern "C" glim_status glim_plan_kernel_ms(glim_plan* p, int32_t nslots, float* ms_out) {
  if (!p || nslots < 0 || 2 * nslots > int(p->ev.size()) || (nslots > 0 && !ms_out)) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  for (int s = 0; s < nslots; ++s) {
    GLIM_CUDA(ctx, cudaEventSynchronize(p->ev[2 * s + 1]));
    GLIM_CUDA(ctx, cudaEventElapsedTime(&ms_out[s], p->ev[2 * s], p->ev[2 * s + 1]));
  }
  return GLIM_OK;
}

extern "C" int32_t glim_plan_kernels_per_launch(const glim_plan* p) {
  if (!p) return 0;
  return (p->nitems > 0 ? 1 : 0) + (p->npairs > 0 ? 1 : 0);
}

extern "C" glim_status glim_plan_device_outputs(glim_plan* p, double** e, double** H, double** b, int64_t** inl) {
  if (!p) return GLIM_EINVAL;
  if (e) *e = p->out_e();
  if (H) *H = p->out_H();
  if (b) *b = p->out_b();
  if (inl) *inl = reinterpret_cast<int64_t*>(p->out_inl());
  return GLIM_OK;
}

extern "C" glim_status glim_plan_device_records(glim_plan* p, double** rec) {
  if (!p || !rec) return GLIM_EINVAL;
  *rec = p->d_rec;
  return GLIM_OK;
}

extern "C" glim_status glim_plan_linearize(glim_plan* p, const double* poses12, double* e_out, double* H_out,
                                           double* b_out, int64_t* inliers_out) {
  GLIM_RANGE("glim_plan_linearize");
  if (!p || !poses12) return GLIM_EINVAL;
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  if (p->npairs > 0 && (!e_out || !H_out || !b_out))
    return set_error(ctx, GLIM_EINVAL, "plan_linearize: null output");
  const bool dev_out = p->npairs > 0 && is_device_ptr(e_out);
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  plan_stage_poses(p, poses12);
  if (dev_out || !p->use_graph) {
    glim_status st = plan_enqueue_poses(p);
    if (st != GLIM_OK) return st;
    p->fposes_on_device = true;
    st = plan_enqueue_kernels(p);
    if (st != GLIM_OK) return st;
    if (dev_out) return copy_outputs(p, e_out, H_out, b_out, inliers_out, false);
    GLIM_CUDA(ctx, cudaMemcpyAsync(p->h_out, p->d_out, p->out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
  } else {
    if (!p->g_full) {
      glim_status st = capture(p, true, &p->g_full);
      if (st != GLIM_OK) return st;
    }
    GLIM_CUDA(ctx, cudaGraphLaunch(p->g_full, ctx->stream));
    p->fposes_on_device = true;
    ctx->launches += glim_plan_kernels_per_launch(p) + (p->npairs > 0 ? 1 : 0);
  }
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return copy_outputs(p, e_out, H_out, b_out, inliers_out, true);
}

extern "C" glim_status glim_plan_linearize_pinned(glim_plan* p, const double* poses12, const double** e,
                                                  const double** H, const double** b, const int64_t** inl) {
  GLIM_RANGE("glim_plan_linearize_pinned");
  if (!p || !poses12) return GLIM_EINVAL;
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  plan_stage_poses(p, poses12);
  if (p->use_graph) {
    if (!p->g_full) {
      glim_status st = capture(p, true, &p->g_full);
      if (st != GLIM_OK) return st;
    }
    GLIM_CUDA(ctx, cudaGraphLaunch(p->g_full, ctx->stream));
    p->fposes_on_device = true;
    ctx->launches += glim_plan_kernels_per_launch(p) + (p->npairs > 0 ? 1 : 0);
  } else {
    glim_status st = plan_enqueue_poses(p);
    if (st != GLIM_OK) return st;
    p->fposes_on_device = true;
    st = plan_enqueue_kernels(p);
    if (st != GLIM_OK) return st;
    GLIM_CUDA(ctx, cudaMemcpyAsync(p->h_out, p->d_out, p->out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
  }
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double* base = reinterpret_cast<const double*>(p->h_out);
  const int P = p->npairs;
  if (e) *e = base;
  if (H) *H = base + P;
  if (b) *b = base + size_t(P) * 145;
  if (inl) *inl = reinterpret_cast<const int64_t*>(base + size_t(P) * 157);
  ctx->err.clear();
  return GLIM_OK;
}

// Inspection of the correspondences that the plan's own kernel resolves (Sec. III-C
// "Correspondence search"): the id-recording instantiation of the kernel the plan runs (same
// lookup and hit code, same launch configuration) linearizes the batch at poses12 and writes
// the canonical voxel id of every (pair, point, level), or -1.
extern "C" glim_status glim_plan_correspondence_ids(glim_plan* p, const double* poses12, int32_t* ids_out,
                                                    double* e_out, double* H_out, double* b_out,
                                                    int64_t* inliers_out) {
  GLIM_RANGE("glim_plan_correspondence_ids");
  if (!p || !poses12) return GLIM_EINVAL;
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  if (p->npairs > 0 && !ids_out) return set_error(ctx, GLIM_EINVAL, "plan_correspondence_ids: null ids_out");
  const int P = p->npairs;
  std::vector<int64_t> off(std::max(P, 1), 0);
  std::vector<int32_t> lv(std::max(P, 1), 0);
  int64_t tot = 0;
  for (int q = 0; q < P; ++q) {
    off[q] = tot;
    lv[q] = p->pairs[q].tgt->levels;
    tot += p->frames[p->pairs[q].src_frame].n * lv[q];
  }
  LinKernelInfo ki;
  if (p->lane_kernel == 1) ki = pick_lin_ids_dense(p->opts.block, p->lmax);
  else if (p->lane_kernel == 2) ki = pick_lin_ids_hash(p->opts.block, p->lmax);
  else ki = pick_lin_ids_general(p->opts.block, p->lmax);
  if (!ki.fn) return set_error(ctx, GLIM_EINVAL, "plan_correspondence_ids: no kernel for this configuration");
  GLIM_CUDA(ctx, cudaFuncSetAttribute(reinterpret_cast<const void*>(ki.fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(ki.smem)));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the pinned pose block may still be read
  glim_status st = plan_upload_poses(p, poses12);
  if (st != GLIM_OK) return st;
  DevBuf<int64_t> d_off;
  DevBuf<int32_t> d_lv;
  GLIM_CUDA(ctx, d_off.alloc(off.size(), ctx->stream));
  GLIM_CUDA(ctx, d_lv.alloc(lv.size(), ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(d_off.p, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  GLIM_CUDA(ctx, cudaMemcpyAsync(d_lv.p, lv.data(), lv.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  if (p->nitems > 0) {
    LinArgs a;
    a.items = p->d_items;
    a.nitems = p->nitems;
    a.item_base = 0;
    a.pairs = p->d_pairs;
    a.frames = p->d_frames;
    a.maps = p->d_maps;
    a.dmaps = p->lane_kernel == 1 ? p->d_dmaps : nullptr;
    a.hmaps = p->lane_kernel == 2 ? p->d_hmaps : nullptr;
    a.pose = p->in_pose32();
    a.head = p->opts.persistent == 1 ? p->d_head : nullptr;
    a.part = p->d_part;
    a.tile = p->tile;
    a.ppt = p->opts.pts_per_thread;
    a.validate = p->opts.validate_surface;
    a.ids = ids_out;
    a.ids_off = d_off.p;
    a.ids_lv = d_lv.p;
    if (p->opts.persistent == 1) GLIM_CUDA(ctx, cudaMemsetAsync(p->d_head, 0, sizeof(int), ctx->stream));
    ki.fn<<<p->grid, p->opts.block, ki.smem, ctx->stream>>>(a);
    GLIM_LAUNCHED(ctx);
  }
  st = enqueue_reduce_expand(ctx, p->d_part, p->d_item_begin, p->in_pose64(), P,
                             p->opts.accum_mode == GLIM_ACC_FP32 ? 1 : 0, p->out_e(), p->out_H(), p->out_b(),
                             p->out_inl());
  if (st != GLIM_OK) return st;
  const bool want = e_out || H_out || b_out || inliers_out;
  if (want && P > 0)
    GLIM_CUDA(ctx, cudaMemcpyAsync(p->h_out, p->d_out, p->out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (want && P > 0) {
    const char* base = reinterpret_cast<const char*>(p->h_out);
    if (e_out) std::memcpy(e_out, base, P * sizeof(double));
    if (H_out) std::memcpy(H_out, base + P * sizeof(double), size_t(P) * 144 * sizeof(double));
    if (b_out) std::memcpy(b_out, base + size_t(P) * 145 * sizeof(double), size_t(P) * 12 * sizeof(double));
    if (inliers_out) std::memcpy(inliers_out, base + size_t(P) * 157 * sizeof(double), P * sizeof(int64_t));
  }
  ctx->err.clear();
  return GLIM_OK;
}

extern "C" glim_status glim_plan_get_opts(const glim_plan* p, glim_lin_opts* out) {
  if (!p || !out) return GLIM_EINVAL;
  *out = p->opts;
  return GLIM_OK;
}

extern "C" glim_status glim_plan_autotune(glim_plan* p, const double* poses12, int32_t iters, glim_lin_opts* best_out,
                                          float* best_ms_out) {
  GLIM_RANGE("glim_plan_autotune");
  if (!p || !poses12 || iters < 1) return GLIM_EINVAL;
  if (maps_current(p) != GLIM_OK) return GLIM_EINVAL;
  glim_ctx* ctx = p->ctx;
  glim_status st = glim_plan_set_poses(p, poses12);
  if (st != GLIM_OK) return st;
  const glim_lin_opts base = p->opts;
  glim_lin_opts best = base;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  GLIM_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(ctx, GLIM_ECUDA, "plan_autotune: cudaEventCreate failed");
  }
  // candidates: block 128 or 256 with 4 to 64 points per thread, plus per block size the
  // points per thread that make the batch's tiles one resident wave of the persistent kernel
  // (small batches: an under-filled or ragged last wave decides their time)
  int64_t total = 0;
  for (int q = 0; q < p->npairs; ++q) total += p->frames[p->pairs[q].src_frame].n;
  std::vector<std::pair<int, int>> cand;
  const int lane = base.kernel == 1 ? 0 : (p->d_dmaps ? 1 : (p->d_hmaps ? 2 : 0));
  for (int b : {64, 128, 256}) {
    if (b == 64 && lane == 0) continue;  // 64-thread blocks: the per-lane kernels only
    for (int t : {4, 8, 16, 32, 64}) cand.emplace_back(b, t);
    const LinKernelInfo ki = pick_kernel(b, base.accum_mode, p->lmax, lane);
    int per_sm = 0;
    if (ki.fn && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.fn, b, ki.smem) != cudaSuccess) {
      cudaGetLastError();  // a failed query only drops this candidate
      per_sm = 0;
    }
    if (per_sm > 0) {
      const int64_t slots = int64_t(per_sm) * ctx->num_sms * b;
      const int fill = int(std::min<int64_t>(256, std::max<int64_t>(1, (total + slots - 1) / slots)));
      if (fill != 4 && fill != 8 && fill != 16 && fill != 32 && fill != 64) cand.emplace_back(b, fill);
    }
  }
  for (size_t c = 0; c < cand.size() && st == GLIM_OK; ++c) {
    glim_lin_opts o = base;
    o.block = cand[c].first;
    o.pts_per_thread = cand[c].second;
    o.persistent = 1;
    o.blocks_per_sm = 0;
    st = plan_configure(p, o);
    if (st == GLIM_OK) st = plan_enqueue_kernels(p);  // warm-up
    if (st != GLIM_OK) break;
    cudaEventRecord(e0, ctx->stream);
    for (int i = 0; i < iters && st == GLIM_OK; ++i) st = plan_enqueue_kernels(p);
    cudaEventRecord(e1, ctx->stream);
    if (st != GLIM_OK) break;
    const cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      st = cuda_check(ctx, ce, "plan_autotune: cudaEventSynchronize");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= iters;
    if (ms < best_ms) {
      best_ms = ms;
      best = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GLIM_OK) {
    // keep the error, and go back to the original configuration where that is possible (a
    // failed reconfiguration leaves the plan in the last one that succeeded)
    const std::string msg = ctx->err;
    plan_configure(p, base);
    ctx->err = msg;
    return st;
  }
  st = plan_configure(p, best);
  if (st != GLIM_OK) {  // the plan still holds the last candidate: back to the original one
    const std::string msg = ctx->err;
    plan_configure(p, base);
    ctx->err = msg;
    return st;
  }
  if (best_out) *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return GLIM_OK;
}

extern "C" glim_status glim_linearize_factors(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                              const glim_pair* pairs, int32_t npairs, const double* poses12,
                                              const glim_lin_opts* opts, double* e_out, double* H_out,
                                              double* b_out, int64_t* inliers_out) {
  GLIM_RANGE("glim_linearize_factors");
  if (!ctx) return GLIM_EINVAL;
  if (!poses12 && nframes > 0) return set_error(ctx, GLIM_EINVAL, "linearize: null poses");
  glim_plan* p = nullptr;
  glim_status st = glim_plan_create(ctx, frames, nframes, pairs, npairs, opts, &p);
  if (st != GLIM_OK) return st;
  p->use_graph = false;
  st = glim_plan_linearize(p, poses12, e_out, H_out, b_out, inliers_out);
  if (st == GLIM_OK) cudaStreamSynchronize(ctx->stream);
  glim_plan_destroy(p);
  return st;
}

extern "C" glim_status glim_linearize_factors_plain(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                                    const glim_pair* pairs, int32_t npairs, const double* poses12,
                                                    const glim_lin_opts* opts, double* e_out, double* H_out,
                                                    double* b_out, int64_t* inliers_out) {
  GLIM_RANGE("glim_linearize_factors_plain");
  if (!ctx) return GLIM_EINVAL;
  glim_lin_opts o{};
  if (opts) o = *opts;
  o.accum_mode = GLIM_ACC_FP32;
  o.persistent = 2;
  glim_plan* p = nullptr;
  glim_status st = glim_plan_create(ctx, frames, nframes, pairs, npairs, &o, &p);
  if (st != GLIM_OK) return st;
  o = p->opts;  // with the defaults filled in
  const bool dev_out = npairs > 0 && is_device_ptr(e_out);
  st = plan_upload_poses(p, poses12);
  if (st != GLIM_OK) {
    glim_plan_destroy(p);
    return st;
  }
  std::vector<int32_t> begin(npairs + 1);
  cudaMemcpy(begin.data(), p->d_item_begin, (npairs + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
  double* h = reinterpret_cast<double*>(p->h_out);
  for (int q = 0; q < npairs && st == GLIM_OK; ++q) {
    // one factor: its items, its reduction, its download, and a synchronization
    LinArgs a;
    a.items = p->d_items;
    a.nitems = begin[q + 1];
    a.item_base = begin[q];
    a.pairs = p->d_pairs;
    a.frames = p->d_frames;
    a.maps = p->d_maps;
    a.dmaps = p->lane_kernel == 1 ? p->d_dmaps : nullptr;
    a.hmaps = p->lane_kernel == 2 ? p->d_hmaps : nullptr;
    a.pose = p->in_pose32();
    a.head = nullptr;  // one block per item of this factor
    a.part = p->d_part;
    a.tile = p->tile;
    a.ppt = o.pts_per_thread;
    a.validate = o.validate_surface;
    const int nb = begin[q + 1] - begin[q];
    if (nb > 0) {
      p->kernel<<<nb, o.block, p->kernel_smem, ctx->stream>>>(a);
      ctx->launches++;
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) { st = cuda_check(ctx, le, "plain: linearize launch"); break; }
    }
    ReduceArgs r;
    r.part = p->d_part;
    r.item_begin = p->d_item_begin;
    r.pose64 = p->in_pose64();
    r.pair_base = q;
    r.npairs = q + 1;
    r.fp32_sum = 1;
    r.e = p->out_e();
    r.H = p->out_H();
    r.b = p->out_b();
    r.inl = p->out_inl();
    k_reduce_expand<<<1, 128, 0, ctx->stream>>>(r);
    ctx->launches++;
    const cudaError_t re = cudaGetLastError();
    if (re != cudaSuccess) { st = cuda_check(ctx, re, "plain: reduce launch"); break; }
    cudaMemcpyAsync(h + q, p->out_e() + q, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(h + npairs + size_t(q) * 144, p->out_H() + size_t(q) * 144, 144 * sizeof(double),
                    cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(h + size_t(npairs) * 145 + size_t(q) * 12, p->out_b() + size_t(q) * 12, 12 * sizeof(double),
                    cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(reinterpret_cast<long long*>(h + size_t(npairs) * 157) + q, p->out_inl() + q, sizeof(long long),
                    cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = set_error(ctx, GLIM_ECUDA, "plain: sync failed");
  }
  if (st == GLIM_OK) {
    if (dev_out) {
      st = copy_outputs(p, e_out, H_out, b_out, inliers_out, false);
      cudaStreamSynchronize(ctx->stream);
    } else {
      st = copy_outputs(p, e_out, H_out, b_out, inliers_out, true);
    }
  }
  glim_plan_destroy(p);
  return st;
}

// Enqueue the FP64 reduce-and-expand kernel of pairs [0, npairs) on `stream` (used by the
// entry point that works without device allocations).
glim_status enqueue_reduce_expand(glim_ctx* ctx, const double* part, const int32_t* item_begin,
                                  const double* pose64, int32_t npairs, int32_t fp32_sum, double* e, double* H,
                                  double* b, long long* inl) {
  if (npairs <= 0) return GLIM_OK;
  ReduceArgs r;
  r.part = part;
  r.item_begin = item_begin;
  r.pose64 = pose64;
  r.pair_base = 0;
  r.npairs = npairs;
  r.fp32_sum = fp32_sum;
  r.e = e;
  r.H = H;
  r.b = b;
  r.inl = inl;
  k_reduce_expand<<<npairs, 128, 0, ctx->stream>>>(r);
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}
