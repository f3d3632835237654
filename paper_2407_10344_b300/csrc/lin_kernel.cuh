// lin_kernel.cuh -- the linearization kernel (Sec. III-C "Linearization"): per-point FP32
// work, per-item block reduction, persistent work queue.  Instantiated per accumulation mode
// in lin_fp32.cu, lin_kahan.cu and lin_fp64.cu.
//
// Per point (FP32): the pinned transform q = R mu + t, u = R mu, the rotated covariance
// R C R^T once for all levels; the first hash probe of every level is issued at once (the
// 48-byte slot carries key and statistics, so one read resolves a probe), then per hit
// S = C~ + R C R^T, Omega = S^-1 (adjugate / determinant), d = mu~ - q, y = Omega d,
// e = d^T y, summed over levels as Omega_sum = sum w Omega, g_sum = sum w y, e_sum.
//
// With G = [-(u)x, I] (3 x 6), the same for every level of a point, A_k = -G diag(R, R) and
// B_k = G S_t (S_t = [[I, 0], [-(t)x, I]]), Eqs. (4)-(5).  A point therefore contributes
// M += G^T Omega_sum G (21 unique entries: -u x Omega u x, u x Omega, Omega), g += G^T g_sum
// ([u x g_sum; g_sum]) and e += e_sum: 28 accumulators, expanded once per pair into
// H = Lift^T M Lift and b = Lift^T g with Lift = [-diag(R, R), S_t].
#pragma once
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

template <int LMAX, class A>
__device__ __forceinline__ void point_term(const PairView& P, const PointIn& in, int64_t k, int validate, A& acc,
                                           int& inl) {
  const float4 m = in.m;
  if (validate && P.F.nrm) {
    const float* nk = P.F.nrm + 3 * k;
    if (behind_surface(m.x, m.y, m.z, P.v, __ldg(nk), __ldg(nk + 1), __ldg(nk + 2))) return;
  }
  const float* R = P.R;
  const float3 q = transform_pinned(R, P.t, m.x, m.y, m.z);

  // first probe of every level, all reads in flight together
  int kx[LMAX], ky[LMAX], kz[LMAX];
  bool ok[LMAX];
  uint32_t hh[LMAX];
  float4 s0[LMAX], s1[LMAX], s2[LMAX];
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    const LevelDev& L = P.M.lv[l];
    ok[l] = (l < P.M.levels) && level_key3(q, L.inv_r, kx[l], ky[l], kz[l]);
    if (ok[l]) {
      hh[l] = hash3(kx[l], ky[l], kz[l], L.log2cap);
      const VoxSlot* sl = L.slots + hh[l];
      s0[l] = ldg4(&sl->w0);
      s1[l] = ldg4(&sl->w1);
      s2[l] = ldg4(&sl->w2);
    }
  }

  // R C R^T while the probes are in flight (W = R C, then the 6 entries of W R^T)
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
  const float r00 = w00 * R[0] + w01 * R[1] + w02 * R[2];
  const float r01 = w00 * R[3] + w01 * R[4] + w02 * R[5];
  const float r02 = w00 * R[6] + w01 * R[7] + w02 * R[8];
  const float r11 = w10 * R[3] + w11 * R[4] + w12 * R[5];
  const float r12 = w10 * R[6] + w11 * R[7] + w12 * R[8];
  const float r22 = w20 * R[6] + w21 * R[7] + w22 * R[8];

  float o00 = 0.f, o01 = 0.f, o02 = 0.f, o11 = 0.f, o12 = 0.f, o22 = 0.f;  // sum Omega
  float g0 = 0.f, g1 = 0.f, g2 = 0.f;                                      // sum Omega d
  float es = 0.f;
  int hits = 0;
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (!ok[l]) continue;
    float4 v0 = s0[l], v1 = s1[l], v2 = s2[l];
    const int sx = __float_as_int(v0.x);
    if (!(sx == kx[l] && __float_as_int(v0.y) == ky[l] && __float_as_int(v0.z) == kz[l])) {
      if (sx == GLIM_EMPTY_COORD) continue;
      // collision: continue the probe sequence (rare at load factor <= 1/2)
      const LevelDev& L = P.M.lv[l];
      const int s = probe_from(L, kx[l], ky[l], kz[l], (hh[l] + 1u) & L.mask, 1);
      if (s < 0) continue;
      v0 = ldg4(&L.slots[s].w0);
      v1 = ldg4(&L.slots[s].w1);
      v2 = ldg4(&L.slots[s].w2);
    }
    // S = C~ + R C R^T, Omega = adj(S) / det(S)
    const float a = v1.w + r00, b = v2.x + r01, c = v2.y + r02, d = v2.z + r11, e = v2.w + r12, f = v0.w + r22;
    const float A00 = d * f - e * e, A01 = c * e - b * f, A02 = b * e - c * d;
    const float A11 = a * f - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
    const float det = a * A00 + b * A01 + c * A02;
    if (!(det > 0.f) || !(det < INFINITY)) continue;  // S not positive definite: skip the term
    const float id = __fdividef(1.0f, det);
    const float O00 = A00 * id, O01 = A01 * id, O02 = A02 * id, O11 = A11 * id, O12 = A12 * id, O22 = A22 * id;
    const float dx = v1.x - q.x, dy = v1.y - q.y, dz = v1.z - q.z;
    const float y0 = O00 * dx + O01 * dy + O02 * dz;
    const float y1 = O01 * dx + O11 * dy + O12 * dz;
    const float y2 = O02 * dx + O12 * dy + O22 * dz;
    es += dx * y0 + dy * y1 + dz * y2;
    o00 += O00; o01 += O01; o02 += O02; o11 += O11; o12 += O12; o22 += O22;
    g0 += y0; g1 += y1; g2 += y2;
    ++hits;
  }
  if (hits == 0) return;
  inl += hits;
  const float wk = m.w;
  o00 *= wk; o01 *= wk; o02 *= wk; o11 *= wk; o12 *= wk; o22 *= wk;
  g0 *= wk; g1 *= wk; g2 *= wk;
  es *= wk;
  const float3 u = make_float3(q.x - P.t[0], q.y - P.t[1], q.z - P.t[2]);
  // W = (u)x Omega_sum
  const float W00 = -u.z * o01 + u.y * o02, W01 = -u.z * o11 + u.y * o12, W02 = -u.z * o12 + u.y * o22;
  const float W10 = u.z * o00 - u.x * o02, W11 = u.z * o01 - u.x * o12, W12 = u.z * o02 - u.x * o22;
  const float W20 = -u.y * o00 + u.x * o01, W21 = -u.y * o01 + u.x * o11, W22 = -u.y * o02 + u.x * o12;
  // M_rr = -(u)x Omega (u)x = W (u)x^T  (symmetric)
  acc.add(0, -u.z * W01 + u.y * W02);
  acc.add(1, u.z * W00 - u.x * W02);
  acc.add(2, -u.y * W00 + u.x * W01);
  acc.add(3, u.z * W10 - u.x * W12);
  acc.add(4, -u.y * W10 + u.x * W11);
  acc.add(5, -u.y * W20 + u.x * W21);
  // M_rt = (u)x Omega
  acc.add(6, W00); acc.add(7, W01); acc.add(8, W02);
  acc.add(9, W10); acc.add(10, W11); acc.add(11, W12);
  acc.add(12, W20); acc.add(13, W21); acc.add(14, W22);
  // M_tt = Omega
  acc.add(15, o00); acc.add(16, o01); acc.add(17, o02); acc.add(18, o11); acc.add(19, o12); acc.add(20, o22);
  // g = [u x g_sum; g_sum]
  acc.add(21, u.y * g2 - u.z * g1);
  acc.add(22, u.z * g0 - u.x * g2);
  acc.add(23, u.x * g1 - u.y * g0);
  acc.add(24, g0); acc.add(25, g1); acc.add(26, g2);
  acc.add(27, es);
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
template <int BLOCK, int PPT, int ACC, int LMAX>
__device__ __forceinline__ void process_item(const LinArgs& a, int item, PairView& V) {
  const Item it = a.items[item];
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
  // software pipeline: the next point's data is read while the current one is processed
  PointIn cur;
  if (base < end) cur = load_point(V.F, base);
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int64_t k = base + int64_t(j) * BLOCK;
    PointIn nxt;
    if (j + 1 < PPT && k + BLOCK < end) nxt = load_point(V.F, k + BLOCK);
    if (k < end) point_term<LMAX>(V, cur, k, a.validate, acc, inl);
    if (j + 1 < PPT) cur = nxt;
  }
  // the reduction ends with a barrier, so V is free for the next item afterwards
  block_reduce_store<BLOCK, ACC>(acc, inl, a.part + int64_t(item) * PSTRIDE);
}

// With a.head set: persistent blocks take items from the atomic queue until it is exhausted.
// With a.head null: one block per item, item = a.item_base + blockIdx.x.
template <int BLOCK, int PPT, int ACC, int LMAX>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_linearize(const LinArgs a) {
  __shared__ PairView V;
  __shared__ int s_item[2];
  if (a.head == nullptr) {
    const int item = a.item_base + blockIdx.x;
    if (item < a.nitems) process_item<BLOCK, PPT, ACC, LMAX>(a, item, V);
    return;
  }
  // the next item index is fetched one item ahead, so the queue's atomic latency overlaps work
  if (threadIdx.x == 0) s_item[0] = atomicAdd(a.head, 1);
  __syncthreads();
  int cur = s_item[0];
  for (int b = 1;; b ^= 1) {
    if (cur >= a.nitems) break;
    if (threadIdx.x == 0) s_item[b] = atomicAdd(a.head, 1);
    process_item<BLOCK, PPT, ACC, LMAX>(a, cur, V);  // ends with a barrier
    cur = s_item[b];
  }
}

template <int ACC>
LinKernel pick_lin(int block, int ppt, int lmax) {
#define GLIM_PICK_L(B, P)                                 \
  switch (lmax) {                                         \
    case 1: return k_linearize<B, P, ACC, 1>;             \
    case 2: return k_linearize<B, P, ACC, 2>;             \
    case 3: return k_linearize<B, P, ACC, 3>;             \
    case 4: return k_linearize<B, P, ACC, 4>;             \
  }                                                       \
  return nullptr;
#define GLIM_PICK_P(B)                 \
  switch (ppt) {                       \
    case 1: { GLIM_PICK_L(B, 1) }      \
    case 2: { GLIM_PICK_L(B, 2) }      \
    case 4: { GLIM_PICK_L(B, 4) }      \
    case 8: { GLIM_PICK_L(B, 8) }      \
  }                                    \
  return nullptr;
  switch (block) {
    case 128: { GLIM_PICK_P(128) }
    case 256: { GLIM_PICK_P(256) }
  }
  return nullptr;
#undef GLIM_PICK_P
#undef GLIM_PICK_L
}

LinKernel pick_lin_fp32(int block, int ppt, int lmax);
LinKernel pick_lin_kahan(int block, int ppt, int lmax);
LinKernel pick_lin_fp64(int block, int ppt, int lmax);

}  // namespace glim_detail
