// covariance.cu -- per-point covariances from the k nearest neighbours (Sec. III-C
// "Preprocessing", Sec. IV-A "Preprocessing": exact kNN once per frame).
//
// Exact kNN on a uniform grid: the points are sorted into cells of size h (the voxel-build
// sort), the cells are hashed, and each query visits the cells in shells of growing
// Chebyshev radius r around its own cell.  After shell r every point within r*h - delta of
// the query has been seen (delta covers the FP32 rounding of the cell assignment), so the
// search stops once the k-th best squared distance is below (r*h - delta)^2.  Queries that
// still lack an answer after MAX_SHELL shells (isolated points) are listed and scanned
// against the whole frame by one warp each (the lanes split the points and merge their k
// best); frames of at most 4096 points are scanned that way throughout.  Squared distances
// that decide the order are FP64 sums (dx*dx + dy*dy) + dz*dz of exact FP64 differences,
// and ties are broken by point index, so the neighbour sets are exactly those of a
// brute-force search; an FP32 distance, within a relative 4e-7 of the exact one, first
// rejects the candidates that cannot beat the current k-th best (B300's FP64 rate is a
// small fraction of its FP32 rate).
//
// Covariance: 1/k sample covariance of the neighbours in FP64; the normal is the eigenvector
// of the smallest eigenvalue, from the closed-form eigenvalues of a symmetric 3x3 matrix
// (Smith, "Eigenvalues of a symmetric 3x3 matrix", CACM 4(4), 1961) and a cross product of
// two rows of A - lambda I; then plane regularisation (GICP, Segal et al. 2009).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

constexpr int MAX_SHELL = 3;

struct CellSlot {
  unsigned long long key;
  uint32_t start, count;
};

__global__ void k_cell_insert(const unsigned long long* __restrict__ ckey, const uint32_t* __restrict__ cstart,
                              int64_t m, CellSlot* __restrict__ slots, int log2cap, uint32_t mask,
                              int* __restrict__ max_probe, unsigned int* __restrict__ status) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= m) return;
  const unsigned long long key = ckey[c];
  uint32_t h = hash_slot(key, log2cap);
  for (uint32_t p = 0; p <= mask; ++p) {
    const unsigned long long old = atomicCAS(&slots[h].key, GLIM_EMPTY_KEY, key);
    if (old == GLIM_EMPTY_KEY) {
      slots[h].start = cstart[c];
      slots[h].count = cstart[c + 1] - cstart[c];
      atomicMax(max_probe, int(p + 1));
      return;
    }
    h = (h + 1u) & mask;
  }
  atomicOr(status, GLIM_DS_HASHFULL);
}

__global__ void k_gather_sorted(const float4* __restrict__ pts, const uint32_t* __restrict__ idx, int64_t n,
                                float4* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 p = pts[idx[i]];
  p.w = __uint_as_float(idx[i]);
  out[i] = p;
}

struct Cand {
  double d;
  int32_t i;
};

__device__ __forceinline__ bool cand_less(double da, int32_t ia, double db, int32_t ib) {
  return da < db || (da == db && ia < ib);
}

// The same order on the bit patterns of non-negative doubles (or +inf), which sort as
// unsigned integers: the top-k list compares with the integer units instead of FP64.
__device__ __forceinline__ bool key_less(unsigned long long da, int32_t ia, unsigned long long db, int32_t ib) {
  return da < db || (da == db && ia < ib);
}

template <int KMAX>
struct TopK {
  unsigned long long d[KMAX];  // FP64 squared distances as bit patterns (non-negative)
  int32_t i[KMAX];
  int k;
  int have;
  double wst;   // the k-th best distance once k candidates were seen, else +inf
  float wthr;   // FP32 bound: a candidate whose FP32 distance exceeds it cannot enter
  static constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;
  __device__ __forceinline__ void init(int kk) {
    k = kk;
    have = 0;
    wst = INFINITY;
    wthr = INFINITY;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      d[j] = INF_BITS;
      i[j] = 0x7FFFFFFF;
    }
  }
  __device__ __forceinline__ double dist(int j) const { return __longlong_as_double((long long)d[j]); }
  // insert (dc, ic) keeping d[0..k) sorted ascending by (distance, index)
  __device__ __forceinline__ void push(double dcd, int32_t ic) {
    const unsigned long long dc = (unsigned long long)__double_as_longlong(dcd);
    ++have;
#pragma unroll
    for (int j = KMAX - 1; j > 0; --j) {
      if (j < k) {
        if (key_less(dc, ic, d[j - 1], i[j - 1])) {
          d[j] = d[j - 1];
          i[j] = i[j - 1];
        } else if (key_less(dc, ic, d[j], i[j])) {
          d[j] = dc;
          i[j] = ic;
        }
      }
    }
    if (key_less(dc, ic, d[0], i[0])) {
      d[0] = dc;
      i[0] = ic;
    }
    if (have >= k) {
      unsigned long long w = d[0];
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j == k - 1) w = d[j];
      wst = __longlong_as_double((long long)w);
      // FP32 distances have a relative error below 4e-7 (three rounded differences, squares
      // and sums of non-negative terms), so any candidate with d64 <= wst has
      // d32 <= wst (1 + 1e-6); the bound is rounded up and +inf beyond the FP32 range
      const double t = wst * (1.0 + 1e-6);
      wthr = t < 3.0e38 ? __double2float_ru(t) : INFINITY;
    }
  }
  // offer a candidate at FP32 distance d32: the FP64 distance is formed only if it may enter
  __device__ __forceinline__ void offer(double qx, double qy, double qz, float qxf, float qyf, float qzf,
                                        const float4& p, int32_t pi) {
    const float fx = p.x - qxf, fy = p.y - qyf, fz = p.z - qzf;
    const float d32 = fx * fx + fy * fy + fz * fz;
    if (have >= k && d32 > wthr) return;
    const double dx = __dsub_rn(double(p.x), qx), dy = __dsub_rn(double(p.y), qy), dz = __dsub_rn(double(p.z), qz);
    const double dc = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (have < k || cand_less(dc, pi, wst, 0x7FFFFFFF)) push(dc, pi);
  }
};

struct GridArgs {
  const float4* sorted;      // points in cell order, w = original index bits
  const float4* pts;         // original order (warp scan, covariance)
  int64_t n;
  const CellSlot* slots;
  uint32_t mask;
  int log2cap;
  int max_probe;
  float inv_h;
  double h;
  int k;
  int reg_mode;
  float eps;
  float* cov6;
  float* normal3;
  int32_t* knn = nullptr;  // optional: the k neighbour indices of every point, nearest first
};

__device__ __forceinline__ bool find_cell(const GridArgs& a, unsigned long long key, uint32_t& start, uint32_t& count) {
  uint32_t h = hash_slot(key, a.log2cap);
  for (int p = 0; p < a.max_probe; ++p) {
    const unsigned long long k = a.slots[h].key;
    if (k == key) {
      start = a.slots[h].start;
      count = a.slots[h].count;
      return true;
    }
    if (k == GLIM_EMPTY_KEY) return false;
    h = (h + 1u) & a.mask;
  }
  return false;
}

// Eigenvector of the smallest eigenvalue of a symmetric 3x3 matrix (FP64).
__device__ __forceinline__ void smallest_eigvec(const double A[6], double n[3]) {
  const double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  double lam;
  if (p1 == 0.0) {
    lam = fmin(a00, fmin(a11, a22));
  } else {
    const double q = (a00 + a11 + a22) / 3.0;
    const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
    const double p = sqrt(p2 / 6.0);
    const double ip = 1.0 / p;
    const double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    double r = 0.5 * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02));
    r = fmin(1.0, fmax(-1.0, r));
    const double phi = acos(r) / 3.0;
    lam = q + 2.0 * p * cos(phi + 2.0943951023931954923);  // 2 pi / 3
  }
  const double r0[3] = {a00 - lam, a01, a02}, r1[3] = {a01, a11 - lam, a12}, r2[3] = {a02, a12, a22 - lam};
  double c[3][3];
  c[0][0] = r0[1] * r1[2] - r0[2] * r1[1]; c[0][1] = r0[2] * r1[0] - r0[0] * r1[2]; c[0][2] = r0[0] * r1[1] - r0[1] * r1[0];
  c[1][0] = r0[1] * r2[2] - r0[2] * r2[1]; c[1][1] = r0[2] * r2[0] - r0[0] * r2[2]; c[1][2] = r0[0] * r2[1] - r0[1] * r2[0];
  c[2][0] = r1[1] * r2[2] - r1[2] * r2[1]; c[2][1] = r1[2] * r2[0] - r1[0] * r2[2]; c[2][2] = r1[0] * r2[1] - r1[1] * r2[0];
  // the longest of the three cross products (the first on ties), selected without indexing
  double b0 = c[0][0], b1 = c[0][1], b2 = c[0][2];
  double bn = b0 * b0 + b1 * b1 + b2 * b2;
#pragma unroll
  for (int j = 1; j < 3; ++j) {
    const double nn = c[j][0] * c[j][0] + c[j][1] * c[j][1] + c[j][2] * c[j][2];
    if (nn > bn) {
      bn = nn;
      b0 = c[j][0];
      b1 = c[j][1];
      b2 = c[j][2];
    }
  }
  if (bn <= 0.0) {  // A - lam I has rank <= 1 (repeated smallest eigenvalue): any vector works
    n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
    return;
  }
  const double inv = 1.0 / sqrt(bn);
  n[0] = b0 * inv;
  n[1] = b1 * inv;
  n[2] = b2 * inv;
}

// Sample covariance (FP64, 1/k) of a query's k neighbours, its normal, and the outputs.
template <int KMAX>
__device__ __forceinline__ void finish_point(const GridArgs& a, int32_t self, double qx, double qy, double qz,
                                             const TopK<KMAX>& top) {
  double m[3] = {0, 0, 0};
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < a.k) {
      const float4 p = a.pts[top.i[j]];
      m[0] += p.x;
      m[1] += p.y;
      m[2] += p.z;
    }
  const double ik = 1.0 / double(a.k);
  m[0] *= ik; m[1] *= ik; m[2] *= ik;
  double C[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < a.k) {
      const float4 p = a.pts[top.i[j]];
      const double vx = p.x - m[0], vy = p.y - m[1], vz = p.z - m[2];
      C[0] += vx * vx; C[1] += vx * vy; C[2] += vx * vz;
      C[3] += vy * vy; C[4] += vy * vz; C[5] += vz * vz;
    }
#pragma unroll
  for (int c = 0; c < 6; ++c) C[c] *= ik;
  double nv[3];
  smallest_eigvec(C, nv);
  if (nv[0] * qx + nv[1] * qy + nv[2] * qz > 0.0) {
    nv[0] = -nv[0]; nv[1] = -nv[1]; nv[2] = -nv[2];
  }
  float* o = a.cov6 + 6 * int64_t(self);
  if (a.reg_mode == 0) {
    const double e = a.eps;
    o[0] = float(C[0] + e); o[1] = float(C[1]); o[2] = float(C[2]);
    o[3] = float(C[3] + e); o[4] = float(C[4]); o[5] = float(C[5] + e);
  } else {
    const double f = 1.0 - double(a.eps);
    o[0] = float(1.0 - f * nv[0] * nv[0]); o[1] = float(-f * nv[0] * nv[1]); o[2] = float(-f * nv[0] * nv[2]);
    o[3] = float(1.0 - f * nv[1] * nv[1]); o[4] = float(-f * nv[1] * nv[2]); o[5] = float(1.0 - f * nv[2] * nv[2]);
  }
  if (a.normal3) {
    float* nn = a.normal3 + 3 * int64_t(self);
    nn[0] = float(nv[0]); nn[1] = float(nv[1]); nn[2] = float(nv[2]);
  }
  if (a.knn) {
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < a.k) a.knn[int64_t(self) * a.k + j] = top.i[j];
  }
}

// Grid search, one thread per point (in cell order).  A query not settled after MAX_SHELL
// shells is appended to `unres` for the warp-per-query scan.
template <int KMAX>
__global__ void __launch_bounds__(128) k_knn_cov(const GridArgs a, int32_t* __restrict__ unres,
                                                 int* __restrict__ nunres) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const float4 qp = a.sorted[s];
  const int32_t self = int32_t(__float_as_uint(qp.w));
  const double qx = qp.x, qy = qp.y, qz = qp.z;
  TopK<KMAX> top;
  top.init(a.k);
  bool done = false;
  int cx, cy, cz;
  voxel_coord(qp.x, a.inv_h, cx);
  voxel_coord(qp.y, a.inv_h, cy);
  voxel_coord(qp.z, a.inv_h, cz);
  const double amax = fmax(fabs(qx), fmax(fabs(qy), fabs(qz)));
#pragma unroll 1
  for (int r = 0; r <= MAX_SHELL && !done; ++r) {
#pragma unroll 1
    for (int dx = -r; dx <= r; ++dx)
#pragma unroll 1
      for (int dy = -r; dy <= r; ++dy)
#pragma unroll 1
        for (int dz = -r; dz <= r; ++dz) {
          if (max(abs(dx), max(abs(dy), abs(dz))) != r) continue;
          const int x = cx + dx, y = cy + dy, z = cz + dz;
          if (x < -GLIM_KEY_BIAS || x >= GLIM_KEY_BIAS || y < -GLIM_KEY_BIAS || y >= GLIM_KEY_BIAS ||
              z < -GLIM_KEY_BIAS || z >= GLIM_KEY_BIAS)
            continue;
          uint32_t st, cnt;
          if (!find_cell(a, pack_key(x, y, z), st, cnt)) continue;
#pragma unroll 1
          for (uint32_t j = st; j < st + cnt; ++j) {
            const float4 p = a.sorted[j];
            top.offer(qx, qy, qz, qp.x, qp.y, qp.z, p, int32_t(__float_as_uint(p.w)));
          }
        }
    const double rad = double(r) * a.h - 1e-6 * (amax + double(r + 1) * a.h);
    if (top.have >= a.k && rad > 0.0 && top.wst <= rad * rad) done = true;
  }
  if (!done) {
    unres[atomicAdd(nunres, 1)] = self;
    return;
  }
  finish_point(a, self, qx, qy, qz, top);
}

// Exact scan of the whole frame for the listed queries, one warp per query: every lane keeps
// the k best of its stride of the points, then k rounds of a warp arg-min over the lanes'
// heads (distance, then index) give the k best of the frame in order.
template <int KMAX>
__global__ void __launch_bounds__(128) k_knn_warp_scan(const GridArgs a, const int32_t* __restrict__ list,
                                                       int count) {
  const int warp = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= count) return;  // whole warps leave together
  const int32_t self = list[warp];
  const float4 qp = a.pts[self];
  const double qx = qp.x, qy = qp.y, qz = qp.z;
  TopK<KMAX> mine;
  mine.init(a.k);
#pragma unroll 1
  for (int64_t j = lane; j < a.n; j += 32) mine.offer(qx, qy, qz, qp.x, qp.y, qp.z, a.pts[j], int32_t(j));
  TopK<KMAX> top;
  top.init(a.k);
  int head = 0;  // next unused entry of this lane's list
#pragma unroll 1
  for (int r = 0; r < a.k; ++r) {
    unsigned long long hd = TopK<KMAX>::INF_BITS;
    int32_t hi = 0x7FFFFFFF;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j == head && j < mine.have && j < a.k) {
        hd = mine.d[j];
        hi = mine.i[j];
      }
    unsigned long long bd = hd;
    int32_t bi = hi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (key_less(od, oi, bd, bi)) {
        bd = od;
        bi = oi;
      }
    }
    if (bd == hd && bi == hi) ++head;  // this lane supplied the winner (indices are unique)
    top.push(__longlong_as_double((long long)bd), bi);
  }
  if (lane == 0) finish_point(a, self, qx, qy, qz, top);
}

__global__ void k_bbox(const float4* __restrict__ pts, int64_t n, float* __restrict__ out /*6: min xyz, max xyz*/) {
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float4 p = pts[i];
    mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
    mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
  }
  for (int c = 0; c < 3; ++c) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
      mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    // float min/max through the ordered-int trick is not needed: values are finite; use a CAS loop
    for (int c = 0; c < 3; ++c) {
      unsigned int* a = reinterpret_cast<unsigned int*>(out + c);
      unsigned int old = *a, assumed;
      do {
        assumed = old;
        if (__uint_as_float(assumed) <= mn[c]) break;
        old = atomicCAS(a, assumed, __float_as_uint(mn[c]));
      } while (old != assumed);
      unsigned int* b = reinterpret_cast<unsigned int*>(out + 3 + c);
      old = *b;
      do {
        assumed = old;
        if (__uint_as_float(assumed) >= mx[c]) break;
        old = atomicCAS(b, assumed, __float_as_uint(mx[c]));
      } while (old != assumed);
    }
  }
}

__global__ void k_iota_i32(int32_t* __restrict__ a, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) a[i] = int32_t(i);
}

__global__ void k_check_finite(const float4* __restrict__ pts, int64_t n, unsigned int* __restrict__ status) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float4 p = pts[i];
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w))) atomicOr(status, GLIM_DS_NONFINITE);
  }
}

int log2_ceil64(int64_t x) {
  int l = 0;
  while ((int64_t(1) << l) < x) ++l;
  return l;
}

// The warp scan of `count` listed queries.
glim_status launch_warp_scan(glim_ctx* ctx, const GridArgs& a, const int32_t* list, int count) {
  if (count <= 0) return GLIM_OK;
  const int grid = ceil_div_i(int64_t(count) * 32, 128);
  if (a.k <= 16) k_knn_warp_scan<16><<<grid, 128, 0, ctx->stream>>>(a, list, count);
  else k_knn_warp_scan<32><<<grid, 128, 0, ctx->stream>>>(a, list, count);
  GLIM_LAUNCHED(ctx);
  return GLIM_OK;
}

// Every point by the warp scan (small frames, or keys out of the packable range).
glim_status knn_all_by_scan(glim_ctx* ctx, const GridArgs& a) {
  DevBuf<int32_t> list;
  GLIM_CUDA(ctx, list.alloc(std::max<int64_t>(a.n, 1), ctx->stream));
  k_iota_i32<<<ceil_div_i(std::max<int64_t>(a.n, 1), 256), 256, 0, ctx->stream>>>(list.p, a.n);
  GLIM_LAUNCHED(ctx);
  glim_status st = launch_warp_scan(ctx, a, list.p, int(a.n));
  if (st != GLIM_OK) return st;
  return take_device_status(ctx, "estimate_covariances");
}

}  // namespace

extern "C" glim_status glim_estimate_covariances(glim_ctx* ctx, const float* pts4, int64_t n, int32_t k,
                                                 int32_t reg_mode, float eps, float* cov6_out, float* normal3_out) {
  return glim_estimate_covariances_knn(ctx, pts4, n, k, reg_mode, eps, cov6_out, normal3_out, nullptr);
}

extern "C" glim_status glim_estimate_covariances_knn(glim_ctx* ctx, const float* pts4, int64_t n, int32_t k,
                                                     int32_t reg_mode, float eps, float* cov6_out,
                                                     float* normal3_out, int32_t* knn_out) {
  GLIM_RANGE("glim_estimate_covariances");
  if (!ctx) return GLIM_EINVAL;
  if (n < 0 || k < 3 || k > 32 || k > n || (reg_mode != 0 && reg_mode != 1) || !(eps >= 0.f) ||
      (n > 0 && (!pts4 || !cov6_out)))
    return set_error(ctx, GLIM_EINVAL, "estimate_covariances: bad arguments (n=%lld k=%d)", (long long)n, k);
  if (n > 0x7FFFFFFFll) return set_error(ctx, GLIM_EINVAL, "estimate_covariances: n too large");
  if (reinterpret_cast<uintptr_t>(pts4) & 15) return set_error(ctx, GLIM_EINVAL, "estimate_covariances: pts4 misaligned");
  DeviceGuard device_guard;
  GLIM_CUDA(ctx, device_guard.set(ctx->device));
  GridArgs a{};
  a.pts = reinterpret_cast<const float4*>(pts4);
  a.n = n;
  a.k = k;
  a.reg_mode = reg_mode;
  a.eps = eps;
  a.cov6 = cov6_out;
  a.normal3 = normal3_out;
  a.knn = knn_out;
  // reject non-finite input before any neighbour search (a NaN distance would never enter
  // the k-best list)
  k_check_finite<<<std::min(ceil_div_i(n, 256), 8 * ctx->num_sms), 256, 0, ctx->stream>>>(a.pts, n, ctx->d_status);
  GLIM_LAUNCHED(ctx);
  {
    glim_status st = take_device_status(ctx, "estimate_covariances");
    if (st != GLIM_OK) return st;
  }
  if (n <= 4096) return knn_all_by_scan(ctx, a);
  // cell size: start from the bounding box assuming points on surfaces, then adjust so that
  // an occupied cell holds about k/2 points
  DevBuf<float> bb;
  GLIM_CUDA(ctx, bb.alloc(6, ctx->stream));
  const float init[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  GLIM_CUDA(ctx, cudaMemcpyAsync(bb.p, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
  k_bbox<<<std::min(ceil_div_i(n, 256), 8 * ctx->num_sms), 256, 0, ctx->stream>>>(a.pts, n, bb.p);
  GLIM_LAUNCHED(ctx);
  float box[6];
  GLIM_CUDA(ctx, cudaMemcpyAsync(box, bb.p, sizeof(box), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int c = 0; c < 6; ++c)
    if (!std::isfinite(box[c])) return set_error(ctx, GLIM_EINVAL, "estimate_covariances: non-finite input");
  const double ext = std::max({double(box[3]) - box[0], double(box[4]) - box[1], double(box[5]) - box[2], 1e-6});
  double h = std::max(ext * std::sqrt(double(k) / double(n)), ext * 1e-5);
  SortedCells cells;
  for (int attempt = 0; attempt < 4; ++attempt) {
    glim_status st = sort_into_cells(ctx, pts4, n, float(1.0 / h), cells, false);
    if (st != GLIM_OK) return st;
    st = take_device_status(ctx, "estimate_covariances keys");
    if (st != GLIM_OK) return st;
    const double occ = double(n) / double(std::max<int64_t>(cells.m, 1));
    const double target = 0.5 * k;
    if (occ >= 0.25 * target && occ <= 4.0 * target) break;
    if (attempt == 3) break;
    h *= std::sqrt(target / occ);
  }
  const int64_t m = cells.m;
  uint32_t covered = 0;  // points with a cell key (keys outside the packable range have none)
  GLIM_CUDA(ctx, cudaMemcpyAsync(&covered, cells.cell_start.p + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (int64_t(covered) != n) return knn_all_by_scan(ctx, a);
  const int64_t cap = std::max<int64_t>(16, int64_t(1) << log2_ceil64(2 * m));
  DevBuf<CellSlot> slots;
  DevBuf<float4> sorted;
  DevBuf<int> maxp;
  GLIM_CUDA(ctx, slots.alloc(cap, ctx->stream));
  GLIM_CUDA(ctx, sorted.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, maxp.alloc(1, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(slots.p, 0xFF, cap * sizeof(CellSlot), ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(maxp.p, 0, sizeof(int), ctx->stream));
  const int l2 = log2_ceil64(cap);
  k_cell_insert<<<ceil_div_i(std::max<int64_t>(m, 1), 256), 256, 0, ctx->stream>>>(
      cells.cell_key.p, cells.cell_start.p, m, slots.p, l2, uint32_t(cap - 1), maxp.p, ctx->d_status);
  GLIM_LAUNCHED(ctx);
  k_gather_sorted<<<ceil_div_i(n, 256), 256, 0, ctx->stream>>>(a.pts, cells.idx_sorted.p, n, sorted.p);
  GLIM_LAUNCHED(ctx);
  int mp = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&mp, maxp.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  a.sorted = sorted.p;
  a.slots = slots.p;
  a.mask = uint32_t(cap - 1);
  a.log2cap = l2;
  a.max_probe = mp;
  a.inv_h = float(1.0 / h);
  a.h = h;
  DevBuf<int32_t> unres;
  DevBuf<int> nunres;
  GLIM_CUDA(ctx, unres.alloc(n, ctx->stream));
  GLIM_CUDA(ctx, nunres.alloc(1, ctx->stream));
  GLIM_CUDA(ctx, cudaMemsetAsync(nunres.p, 0, sizeof(int), ctx->stream));
  if (a.k <= 16) k_knn_cov<16><<<ceil_div_i(n, 128), 128, 0, ctx->stream>>>(a, unres.p, nunres.p);
  else k_knn_cov<32><<<ceil_div_i(n, 128), 128, 0, ctx->stream>>>(a, unres.p, nunres.p);
  GLIM_LAUNCHED(ctx);
  int nu = 0;
  GLIM_CUDA(ctx, cudaMemcpyAsync(&nu, nunres.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GLIM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  glim_status st = launch_warp_scan(ctx, a, unres.p, nu);
  if (st != GLIM_OK) return st;
  st = take_device_status(ctx, "estimate_covariances");
  if (st == GLIM_OK) ctx->err.clear();
  return st;
}
