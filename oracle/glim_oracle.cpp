// glim_oracle.cpp -- plain, slow FP64 CPU oracle of the matching-cost-factor
// linearization of GLIM (Koide et al., Sec. III-C, Eqs. (2)-(8)).
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg load this library.  It shares no code, header
// or constant generator with the CUDA path; it is its own definition of what
// that path computes, written for a reader to check against the paper by eye:
//
//   * voxelmaps are std::map<(x,y,z), accumulator>, one per resolution level
//     (Sec. III-C "Preprocessing": average of the points and covariances in
//     each voxel, r_l = r_0 * 2^(l-1));
//   * correspondences are one voxel per level, q = floor(p / r) (Sec. III-C
//     "Correspondence search"), with the surface-orientation test
//     (p_k - T_i^-1 t_j) . n_k > 0 => discard;
//   * the cost is Eq. (2)-(3), the Jacobians A_k, B_k are Eqs. (4)-(5) as
//     printed, and H, b are Eqs. (6)-(8) with the transposes read so that the
//     shapes agree (H_ii = sum A^T Omega A, b_i = sum A^T Omega d, ...);
//   * per-point covariances come from a brute-force k-nearest-neighbour search
//     and GICP plane regularisation (Segal et al. 2009, cited in Sec. III-C).
//
// Conventions where the paper is silent or inconsistent:
//   * source s = i (points), target t = j (voxelmap); the relative pose is
//     T_rel = T_t^-1 T_s (the one under which Eqs. (4)-(5) are the exact
//     derivatives), with right perturbations T <- T Exp(xi), xi = [omega; v];
//   * the voxel key is defined on FP32 arithmetic: R_f, t_f are the FP32
//     roundings of the FP64 relative pose, q_f is formed with three fused
//     multiply-adds per axis (in x, y, z order) and key = floor(q_f * inv_r_f),
//     inv_r_f = fp32(1 / r).  Everything after the key is FP64.
//   * canonical voxel id = rank of the key in lexicographic (x, y, z) order
//     among the occupied voxels of that level (std::map order); -1 = miss.
//
// This file must be compiled without FP contraction or fast-math
// (-ffp-contract=off), so that the FP32 key emulation is exact.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <queue>
#include <thread>
#include <vector>

namespace {

constexpr int ORC_OK = 0;
constexpr int ORC_EINVAL = -1;
constexpr int ORC_ERANGE = -5;
constexpr int ORC_ENOTPD = -6;
constexpr int64_t KEY_LIMIT = int64_t(1) << 20;  // keys must lie in [-2^20, 2^20)

struct Key3 {
  int32_t x, y, z;
  bool operator<(const Key3& o) const {
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};

struct Voxel {
  double sum_mu[3] = {0, 0, 0};
  double sum_C[6] = {0, 0, 0, 0, 0, 0};
  int64_t count = 0;
  double mean[3] = {0, 0, 0};
  double cov[6] = {0, 0, 0, 0, 0, 0};
  int32_t id = -1;
};

struct Level {
  double r = 0;
  float inv_r = 0;
  std::map<Key3, Voxel> map;
  std::vector<const Voxel*> by_id;
};

struct VMap {
  std::vector<Level> levels;
};

// ---------------------------------------------------------------- small linear algebra (FP64)
using M3 = std::array<std::array<double, 3>, 3>;
using V3 = std::array<double, 3>;

M3 sym_from6(const double* c) {
  M3 m;
  m[0] = {c[0], c[1], c[2]};
  m[1] = {c[1], c[3], c[4]};
  m[2] = {c[2], c[4], c[5]};
  return m;
}

M3 mul(const M3& a, const M3& b) {
  M3 r{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      r[i][j] = s;
    }
  return r;
}

M3 transpose(const M3& a) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r[i][j] = a[j][i];
  return r;
}

V3 mulv(const M3& a, const V3& v) {
  V3 r;
  for (int i = 0; i < 3; ++i) r[i] = a[i][0] * v[0] + a[i][1] * v[1] + a[i][2] * v[2];
  return r;
}

M3 hat(const V3& v) {  // (v)_x, the skew-symmetric matrix with hat(v) w = v x w
  M3 m;
  m[0] = {0.0, -v[2], v[1]};
  m[1] = {v[2], 0.0, -v[0]};
  m[2] = {-v[1], v[0], 0.0};
  return m;
}

// Inverse of a symmetric positive-definite 3x3 matrix by an LDL^T factorisation.
// Returns false if a pivot is not positive (the matrix is not PD).
bool spd_inverse(const M3& S, M3& inv) {
  double L[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double D[3];
  for (int j = 0; j < 3; ++j) {
    double d = S[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k] * D[k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    D[j] = d;
    for (int i = j + 1; i < 3; ++i) {
      double s = S[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k] * D[k];
      L[i][j] = s / d;
    }
  }
  // inverse = L^-T D^-1 L^-1; solve column by column
  for (int c = 0; c < 3; ++c) {
    double y[3], z[3], x[3];
    for (int i = 0; i < 3; ++i) {  // L y = e_c
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
      y[i] = s;
    }
    for (int i = 0; i < 3; ++i) z[i] = y[i] / D[i];
    for (int i = 2; i >= 0; --i) {  // L^T x = z
      double s = z[i];
      for (int k = i + 1; k < 3; ++k) s -= L[k][i] * x[k];
      x[i] = s;
    }
    for (int i = 0; i < 3; ++i) inv[i][c] = x[i];
  }
  return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (Jacobi 1846; as in
// Golub & Van Loan, Sec. 8.5).  On return, w holds eigenvalues and the columns of V
// the eigenvectors.
void jacobi_eigen(M3 A, double w[3], M3& V) {
  V = M3{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double scale = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2] + off;
    if (off <= 1e-34 * scale || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < 3; ++k) {
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) w[i] = A[i][i];
}

// ---------------------------------------------------------------- FP32 key emulation
// The correspondence key on the FP32 path: q_f = R_f mu + t_f with one fused
// multiply-add per term, starting from t_f and adding the x, y, z terms in order.
inline float fp32_transform_axis(const float Rrow[3], float t, float mx, float my, float mz) {
  return std::fmaf(Rrow[2], mz, std::fmaf(Rrow[1], my, std::fmaf(Rrow[0], mx, t)));
}

inline bool fp32_key(float coord, float inv_r, int32_t& key) {
  float prod = coord * inv_r;  // one IEEE round-to-nearest FP32 multiply
  float f = std::floor(prod);
  if (!std::isfinite(f) || f < -double(KEY_LIMIT) || f >= double(KEY_LIMIT)) return false;
  key = int32_t(f);
  return true;
}

// ---------------------------------------------------------------- frames, pairs, poses
struct Pose {
  M3 R;
  V3 t;
};

Pose pose_from12(const double* p) {
  Pose P;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) P.R[i][j] = p[4 * i + j];
    P.t[i] = p[4 * i + 3];
  }
  return P;
}

// T_rel = T_t^-1 T_s:  R = R_t^T R_s,  t = R_t^T (t_s - t_t)
Pose relative(const Pose& Ts, const Pose& Tt) {
  Pose r;
  M3 RtT = transpose(Tt.R);
  r.R = mul(RtT, Ts.R);
  V3 dt = {Ts.t[0] - Tt.t[0], Ts.t[1] - Tt.t[1], Ts.t[2] - Tt.t[2]};
  r.t = mulv(RtT, dt);
  return r;
}

}  // namespace

extern "C" {

typedef struct {
  const float* pts4;     // n x (x, y, z, w); w = per-point weight
  const float* cov6;     // n x (xx, xy, xz, yy, yz, zz)
  const float* normal3;  // n x 3, may be null (then surface validation keeps every point)
  int64_t n;
} orc_frame;

typedef struct {
  int32_t src, tgt;
} orc_pair;

typedef struct {
  int32_t validate_surface;  // apply the surface-orientation test
  int32_t omega_identity;    // test-only special case: Omega = I
  int32_t omega_grad_full;   // gradient: 1 = differentiate Omega too, 0 = Omega frozen
  int32_t nthreads;          // worker threads over pairs (>= 1)
} orc_opts;

int orc_abi_version() { return 1; }

// Covariance of point i from its k nearest neighbours nb (nearest first, the point itself
// included): mean and 1/k sample covariance in FP64, eigenvector n of the smallest eigenvalue
// (cyclic Jacobi), n oriented so that n . mu <= 0; reg_mode 0: C + eps I, reg_mode 1:
// C = I - (1 - eps) n n^T (GICP plane regularisation, Segal et al. 2009).
void point_covariance(const float* pts4, int64_t i, const std::vector<int64_t>& nb, int reg_mode, double eps,
                      double* cov6, double* normal3, int32_t* knn, uint8_t* near_tie) {
  const int k = int(nb.size());
  const double px = pts4[4 * i], py = pts4[4 * i + 1], pz = pts4[4 * i + 2];
  double m[3] = {0, 0, 0};
  for (int a = 0; a < k; ++a)
    for (int c = 0; c < 3; ++c) m[c] += pts4[4 * nb[a] + c];
  for (int c = 0; c < 3; ++c) m[c] /= k;
  M3 C{};
  for (int a = 0; a < k; ++a) {
    double v[3];
    for (int c = 0; c < 3; ++c) v[c] = pts4[4 * nb[a] + c] - m[c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) C[r][c] += v[r] * v[c];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) C[r][c] /= k;
  double w[3];
  M3 V;
  jacobi_eigen(C, w, V);
  int order[3] = {0, 1, 2};
  std::sort(order, order + 3, [&](int a, int b) { return w[a] < w[b]; });
  V3 nrm = {V[0][order[0]], V[1][order[0]], V[2][order[0]]};
  double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
  for (int c = 0; c < 3; ++c) nrm[c] /= nn;
  if (nrm[0] * px + nrm[1] * py + nrm[2] * pz > 0)
    for (int c = 0; c < 3; ++c) nrm[c] = -nrm[c];
  M3 out;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      if (reg_mode == 0)
        out[r][c] = C[r][c] + (r == c ? eps : 0.0);
      else
        out[r][c] = (r == c ? 1.0 : 0.0) - (1.0 - eps) * nrm[r] * nrm[c];
    }
  cov6[0] = out[0][0]; cov6[1] = out[0][1]; cov6[2] = out[0][2];
  cov6[3] = out[1][1]; cov6[4] = out[1][2]; cov6[5] = out[2][2];
  if (normal3)
    for (int c = 0; c < 3; ++c) normal3[c] = nrm[c];
  if (knn)
    for (int a = 0; a < k; ++a) knn[a] = int32_t(nb[a]);
  if (near_tie) *near_tie = (w[order[1]] - w[order[0]]) <= 1e-4 * std::fabs(w[order[2]]);
}

// ---------------------------------------------------------------- covariances (brute-force kNN)
// For each point: its k nearest neighbours (itself included; ties broken by
// (squared distance, index), distances in FP64), their sample covariance with
// 1/k normalisation, and
//   reg_mode 0: C = C_sample + eps * I
//   reg_mode 1: C = I - (1 - eps) n n^T, n = eigenvector of the smallest eigenvalue
// The normal n is oriented so that n . mu <= 0 (facing the sensor at the origin).
// near_tie[i] = 1 when the two smallest eigenvalues are within 1e-4 * largest.
int orc_estimate_covariances(const float* pts4, int64_t n, int k, int reg_mode, double eps,
                             double* cov6_out, double* normal3_out, int32_t* knn_out,
                             uint8_t* near_tie_out, int nthreads) {
  if (n < 0 || k < 3 || k > n || (reg_mode != 0 && reg_mode != 1)) return ORC_EINVAL;
  for (int64_t i = 0; i < 4 * n; ++i)
    if (!std::isfinite(pts4[i])) return ORC_EINVAL;
  auto work = [&](int64_t begin, int64_t end) {
    std::vector<std::pair<double, int64_t>> d(n);
    for (int64_t i = begin; i < end; ++i) {
      const double px = pts4[4 * i], py = pts4[4 * i + 1], pz = pts4[4 * i + 2];
      for (int64_t j = 0; j < n; ++j) {
        double dx = double(pts4[4 * j]) - px, dy = double(pts4[4 * j + 1]) - py,
               dz = double(pts4[4 * j + 2]) - pz;
        d[j] = {dx * dx + dy * dy + dz * dz, j};
      }
      std::partial_sort(d.begin(), d.begin() + k, d.end());
      std::vector<int64_t> nb(k);
      for (int a = 0; a < k; ++a) nb[a] = d[a].second;
      point_covariance(pts4, i, nb, reg_mode, eps, cov6_out + 6 * i, normal3_out ? normal3_out + 3 * i : nullptr,
                       knn_out ? knn_out + int64_t(k) * i : nullptr, near_tie_out ? near_tie_out + i : nullptr);
    }
  };
  int T = std::max(1, nthreads);
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t) th.emplace_back(work, n * t / T, n * (t + 1) / T);
  for (auto& x : th) x.join();
  return ORC_OK;
}

// The same for the listed query points only (nq indices into the frame): every query scans
// all n points, keeping the k smallest (squared distance in FP64, index) pairs.  Outputs are
// per query (nq x 6, nq x 3, nq x k, nq).  For parity tests on large frames.
int orc_covariances_at(const float* pts4, int64_t n, const int64_t* queries, int64_t nq, int k, int reg_mode,
                       double eps, double* cov6_out, double* normal3_out, int32_t* knn_out, uint8_t* near_tie_out,
                       int nthreads) {
  if (n < 0 || nq < 0 || k < 3 || k > n || (reg_mode != 0 && reg_mode != 1)) return ORC_EINVAL;
  for (int64_t q = 0; q < nq; ++q)
    if (queries[q] < 0 || queries[q] >= n) return ORC_EINVAL;
  auto work = [&](int64_t begin, int64_t end) {
    for (int64_t q = begin; q < end; ++q) {
      const int64_t i = queries[q];
      const double px = pts4[4 * i], py = pts4[4 * i + 1], pz = pts4[4 * i + 2];
      std::priority_queue<std::pair<double, int64_t>> best;  // the k best so far, worst on top
      for (int64_t j = 0; j < n; ++j) {
        double dx = double(pts4[4 * j]) - px, dy = double(pts4[4 * j + 1]) - py,
               dz = double(pts4[4 * j + 2]) - pz;
        const std::pair<double, int64_t> c{dx * dx + dy * dy + dz * dz, j};
        if (int(best.size()) < k) {
          best.push(c);
        } else if (c < best.top()) {
          best.pop();
          best.push(c);
        }
      }
      std::vector<int64_t> nb(k);
      for (int a = k - 1; a >= 0; --a) {
        nb[a] = best.top().second;
        best.pop();
      }
      point_covariance(pts4, i, nb, reg_mode, eps, cov6_out + 6 * q, normal3_out ? normal3_out + 3 * q : nullptr,
                       knn_out ? knn_out + int64_t(k) * q : nullptr, near_tie_out ? near_tie_out + q : nullptr);
    }
  };
  int T = std::max<int64_t>(1, std::min<int64_t>(nthreads, std::max<int64_t>(nq, 1)));
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t) th.emplace_back(work, nq * t / T, nq * (t + 1) / T);
  for (auto& x : th) x.join();
  return ORC_OK;
}

// ---------------------------------------------------------------- voxelmap (std::map)
// Voxel key of a raw (untransformed) point: floor(x * inv_r_f) per axis in FP32.
// Voxel statistics: mean of member means and mean of member covariances, in FP64.
void* orc_vmap_build(const float* pts4, const float* cov6, int64_t n, const double* resolutions,
                     int levels, int* status) {
  *status = ORC_OK;
  if (n < 0 || levels < 1 || levels > 8) {
    *status = ORC_EINVAL;
    return nullptr;
  }
  for (int64_t i = 0; i < 4 * n; ++i)
    if (!std::isfinite(pts4[i])) { *status = ORC_EINVAL; return nullptr; }
  for (int64_t i = 0; i < 6 * n; ++i)
    if (!std::isfinite(cov6[i])) { *status = ORC_EINVAL; return nullptr; }
  VMap* vm = new VMap;
  vm->levels.resize(levels);
  for (int l = 0; l < levels; ++l) {
    Level& L = vm->levels[l];
    if (!(resolutions[l] > 0.0)) { *status = ORC_EINVAL; delete vm; return nullptr; }
    L.r = resolutions[l];
    L.inv_r = float(1.0 / resolutions[l]);
    for (int64_t i = 0; i < n; ++i) {
      Key3 key;
      if (!fp32_key(pts4[4 * i], L.inv_r, key.x) || !fp32_key(pts4[4 * i + 1], L.inv_r, key.y) ||
          !fp32_key(pts4[4 * i + 2], L.inv_r, key.z)) {
        *status = ORC_ERANGE;
        delete vm;
        return nullptr;
      }
      Voxel& v = L.map[key];
      for (int c = 0; c < 3; ++c) v.sum_mu[c] += pts4[4 * i + c];
      for (int c = 0; c < 6; ++c) v.sum_C[c] += cov6[6 * i + c];
      v.count += 1;
    }
    int32_t id = 0;
    for (auto& kv : L.map) {
      Voxel& v = kv.second;
      for (int c = 0; c < 3; ++c) v.mean[c] = v.sum_mu[c] / double(v.count);
      for (int c = 0; c < 6; ++c) v.cov[c] = v.sum_C[c] / double(v.count);
      v.id = id++;
      L.by_id.push_back(&v);
    }
  }
  return vm;
}

int64_t orc_vmap_size(const void* h, int level) {
  const VMap* vm = static_cast<const VMap*>(h);
  if (level < 0 || level >= int(vm->levels.size())) return -1;
  return int64_t(vm->levels[level].map.size());
}

// Canonical (lexicographic key) order.
void orc_vmap_export(const void* h, int level, int32_t* keys3, double* mean3, double* cov6,
                     int64_t* count) {
  const VMap* vm = static_cast<const VMap*>(h);
  const Level& L = vm->levels[level];
  int64_t i = 0;
  for (auto& kv : L.map) {
    if (keys3) { keys3[3 * i] = kv.first.x; keys3[3 * i + 1] = kv.first.y; keys3[3 * i + 2] = kv.first.z; }
    if (mean3) for (int c = 0; c < 3; ++c) mean3[3 * i + c] = kv.second.mean[c];
    if (cov6) for (int c = 0; c < 6; ++c) cov6[6 * i + c] = kv.second.cov[c];
    if (count) count[i] = kv.second.count;
    ++i;
  }
}

void orc_vmap_free(void* h) { delete static_cast<VMap*>(h); }

}  // extern "C"

namespace {

// Correspondence of point k of the source under the FP32 key rule: voxel per level or null.
// Returns false if the surface test discards the point.
struct Corr {
  bool visible = true;
  const Voxel* vox[8] = {nullptr};
};

Corr correspond(const VMap& tgt, const float Rf[3][3], const float tf[3], const float vf[3],
                const float* mu4, const float* nrm3, bool validate) {
  Corr c;
  if (validate && nrm3) {
    // (p_k - T_s^-1 t_t) . n_k > 0  =>  the target viewpoint is behind the surface
    float dx = mu4[0] - vf[0], dy = mu4[1] - vf[1], dz = mu4[2] - vf[2];
    float s = nrm3[0] * dx;
    s = std::fmaf(nrm3[1], dy, s);
    s = std::fmaf(nrm3[2], dz, s);
    if (s > 0.0f) {
      c.visible = false;
      return c;
    }
  }
  float q[3];
  for (int a = 0; a < 3; ++a) q[a] = fp32_transform_axis(Rf[a], tf[a], mu4[0], mu4[1], mu4[2]);
  for (size_t l = 0; l < tgt.levels.size(); ++l) {
    const Level& L = tgt.levels[l];
    Key3 key;
    if (!fp32_key(q[0], L.inv_r, key.x) || !fp32_key(q[1], L.inv_r, key.y) ||
        !fp32_key(q[2], L.inv_r, key.z))
      continue;  // out of the key range: a miss
    auto it = L.map.find(key);
    if (it != L.map.end()) c.vox[l] = &it->second;
  }
  return c;
}

struct PairResult {
  double e = 0;
  double H[12][12] = {};
  double b[12] = {};
  long double eL = 0;
  long double HL[12][12] = {};
  long double bL[12] = {};
  int64_t inliers = 0;
  int64_t skipped = 0;
  double babs = 0;  // sum over terms of |w J^T Omega d|_2, a cancellation-free scale of b
};

struct PairCtx {
  Pose rel;
  float Rf[3][3], tf[3], vf[3];
};

PairCtx make_pair_ctx(const double* poses12, int s, int t) {
  PairCtx pc;
  pc.rel = relative(pose_from12(poses12 + 12 * s), pose_from12(poses12 + 12 * t));
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) pc.Rf[i][j] = float(pc.rel.R[i][j]);
    pc.tf[i] = float(pc.rel.t[i]);
  }
  // target viewpoint in the source frame: T_s^-1 t_t = -R^T t
  V3 v = mulv(transpose(pc.rel.R), pc.rel.t);
  for (int i = 0; i < 3; ++i) pc.vf[i] = float(-v[i]);
  return pc;
}

// One point-to-voxel term, Eq. (3), and its quadratic-factor contribution, Eqs. (4)-(8).
void accumulate_term(const Pose& T, const float* mu4, const float* cov6, const Voxel& vox,
                     bool omega_identity, PairResult& out) {
  const double w = mu4[3];
  V3 mu = {mu4[0], mu4[1], mu4[2]};
  double c6[6];
  for (int i = 0; i < 6; ++i) c6[i] = cov6[i];
  M3 C = sym_from6(c6);
  M3 Ct = sym_from6(vox.cov);
  M3 RCRt = mul(mul(T.R, C), transpose(T.R));
  M3 S;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = Ct[i][j] + RCRt[i][j];
  M3 Om;
  if (omega_identity) {
    Om = M3{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
  } else if (!spd_inverse(S, Om)) {
    out.skipped += 1;
    return;
  }
  V3 q = mulv(T.R, mu);
  for (int i = 0; i < 3; ++i) q[i] += T.t[i];
  V3 d = {vox.mean[0] - q[0], vox.mean[1] - q[1], vox.mean[2] - q[2]};
  // A_k = [R (mu)x, -R],  B_k = [-(T mu)x, I]   (3 x 6 each), J = [A_k, B_k] (3 x 12)
  double J[3][12];
  M3 Rmu = mul(T.R, hat(mu));
  M3 qx = hat(q);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      J[i][j] = Rmu[i][j];
      J[i][3 + j] = -T.R[i][j];
      J[i][6 + j] = -qx[i][j];
      J[i][9 + j] = (i == j) ? 1.0 : 0.0;
    }
  V3 Od = mulv(Om, d);
  double e = d[0] * Od[0] + d[1] * Od[1] + d[2] * Od[2];
  double OJ[3][12];
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 12; ++c) OJ[i][c] = Om[i][0] * J[0][c] + Om[i][1] * J[1][c] + Om[i][2] * J[2][c];
  out.e += w * e;
  out.eL += (long double)(w * e);
  double gsq = 0;
  for (int r = 0; r < 12; ++r) {
    for (int c = 0; c < 12; ++c) {
      double h = J[0][r] * OJ[0][c] + J[1][r] * OJ[1][c] + J[2][r] * OJ[2][c];
      out.H[r][c] += w * h;
      out.HL[r][c] += (long double)(w * h);
    }
    double g = J[0][r] * Od[0] + J[1][r] * Od[1] + J[2][r] * Od[2];
    out.b[r] += w * g;
    out.bL[r] += (long double)(w * g);
    gsq += (w * g) * (w * g);
  }
  out.babs += std::sqrt(gsq);
  out.inliers += 1;
}

template <class F>
void parallel_pairs(int npairs, int nthreads, F f) {
  int T = std::max(1, std::min(nthreads, npairs));
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t)
    th.emplace_back([&, t] {
      for (int p = t; p < npairs; p += T) f(p);
    });
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

// Linearize every (source, target) pair: e (npairs), H (npairs x 12 x 12, variables ordered
// [xi_s; xi_t], xi = [omega; v]), b (npairs x 12), inlier (point, level) hits (npairs).
// ids_out (nullable): per pair, n_src x levels canonical voxel ids (-1 = miss or discarded),
// concatenated over pairs in pair order.  ids_in (nullable): same layout; if given, these
// correspondences are used instead of the lookup (frozen correspondences).
// comp_out (nullable): per pair 1 + 144 + 12 values accumulated in long double, the
// oracle's own rounding reference, then the cancellation-free scale of b (sum over terms
// of |w J^T Omega d|_2): 158 values per pair.
int orc_linearize(const orc_frame* frames, int nframes, void* const* vmaps, const orc_pair* pairs,
                  int npairs, const double* poses12, const orc_opts* opts, double* e_out,
                  double* H_out, double* b_out, int64_t* inliers_out, int64_t* skipped_out,
                  int32_t* ids_out, const int32_t* ids_in, double* comp_out) {
  for (int p = 0; p < npairs; ++p) {
    if (pairs[p].src < 0 || pairs[p].src >= nframes || pairs[p].tgt < 0 || pairs[p].tgt >= nframes ||
        vmaps[pairs[p].tgt] == nullptr)
      return ORC_EINVAL;
  }
  std::vector<int64_t> id_off(npairs + 1, 0);
  for (int p = 0; p < npairs; ++p) {
    const VMap* vm = static_cast<const VMap*>(vmaps[pairs[p].tgt]);
    id_off[p + 1] = id_off[p] + frames[pairs[p].src].n * int64_t(vm->levels.size());
  }
  parallel_pairs(npairs, opts->nthreads, [&](int p) {
    const orc_frame& F = frames[pairs[p].src];
    const VMap& tgt = *static_cast<const VMap*>(vmaps[pairs[p].tgt]);
    const int L = int(tgt.levels.size());
    PairCtx pc = make_pair_ctx(poses12, pairs[p].src, pairs[p].tgt);
    PairResult res;
    for (int64_t k = 0; k < F.n; ++k) {
      const float* mu4 = F.pts4 + 4 * k;
      Corr c;
      if (ids_in) {
        for (int l = 0; l < L; ++l) {
          int32_t id = ids_in[id_off[p] + k * L + l];
          c.vox[l] = (id >= 0) ? tgt.levels[l].by_id[id] : nullptr;
        }
      } else {
        c = correspond(tgt, pc.Rf, pc.tf, pc.vf, mu4, F.normal3 ? F.normal3 + 3 * k : nullptr,
                       opts->validate_surface != 0);
      }
      for (int l = 0; l < L; ++l) {
        if (ids_out) ids_out[id_off[p] + k * L + l] = c.vox[l] ? c.vox[l]->id : -1;
        if (c.vox[l]) accumulate_term(pc.rel, mu4, F.cov6 + 6 * k, *c.vox[l], opts->omega_identity != 0, res);
      }
    }
    e_out[p] = res.e;
    for (int r = 0; r < 12; ++r) {
      for (int c = 0; c < 12; ++c) H_out[144 * p + 12 * r + c] = res.H[r][c];
      b_out[12 * p + r] = res.b[r];
    }
    if (inliers_out) inliers_out[p] = res.inliers;
    if (skipped_out) skipped_out[p] = res.skipped;
    if (comp_out) {
      double* o = comp_out + 158 * p;
      o[0] = double(res.eL);
      for (int r = 0; r < 12; ++r)
        for (int c = 0; c < 12; ++c) o[1 + 12 * r + c] = double(res.HL[r][c]);
      for (int r = 0; r < 12; ++r) o[145 + r] = double(res.bL[r]);
      o[157] = res.babs;
    }
  });
  return ORC_OK;
}

// Cost e (Eq. (2)) per pair at the given poses with frozen correspondences ids_in (layout as
// in orc_linearize).  If omega_poses12 is non-null, Omega is evaluated at those poses
// (Omega fixed at the linearization point); otherwise at poses12.
int orc_energy(const orc_frame* frames, int nframes, void* const* vmaps, const orc_pair* pairs,
               int npairs, const double* poses12, const double* omega_poses12,
               const int32_t* ids_in, const orc_opts* opts, double* e_out) {
  (void)nframes;
  int64_t off = 0;
  for (int p = 0; p < npairs; ++p) {
    const orc_frame& F = frames[pairs[p].src];
    const VMap& tgt = *static_cast<const VMap*>(vmaps[pairs[p].tgt]);
    const int L = int(tgt.levels.size());
    Pose T = relative(pose_from12(poses12 + 12 * pairs[p].src), pose_from12(poses12 + 12 * pairs[p].tgt));
    Pose TO = omega_poses12 ? relative(pose_from12(omega_poses12 + 12 * pairs[p].src),
                                       pose_from12(omega_poses12 + 12 * pairs[p].tgt))
                            : T;
    double e = 0;
    for (int64_t k = 0; k < F.n; ++k) {
      const float* mu4 = F.pts4 + 4 * k;
      V3 mu = {mu4[0], mu4[1], mu4[2]};
      double c6[6];
      for (int i = 0; i < 6; ++i) c6[i] = F.cov6[6 * k + i];
      M3 C = sym_from6(c6);
      for (int l = 0; l < L; ++l) {
        int32_t id = ids_in[off + k * L + l];
        if (id < 0) continue;
        const Voxel& v = *tgt.levels[l].by_id[id];
        M3 S = mul(mul(TO.R, C), transpose(TO.R));
        M3 Ct = sym_from6(v.cov);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) S[i][j] += Ct[i][j];
        M3 Om;
        if (opts->omega_identity) Om = M3{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
        else if (!spd_inverse(S, Om)) continue;
        V3 q = mulv(T.R, mu);
        V3 d = {v.mean[0] - q[0] - T.t[0], v.mean[1] - q[1] - T.t[1], v.mean[2] - q[2] - T.t[2]};
        V3 Od = mulv(Om, d);
        e += double(mu4[3]) * (d[0] * Od[0] + d[1] * Od[1] + d[2] * Od[2]);
      }
    }
    off += F.n * L;
    e_out[p] = e;
  }
  return ORC_OK;
}

// Gradient of E = sum over pairs of e (Eq. (2)), with the per-point weight w_k in the
// fourth lane of each point, with respect to:
//   dxi_out  (nframes x 6): right perturbation xi = [omega; v] of every frame pose,
//   dmu_out  (sum of frame sizes x 3, frames concatenated): source point coordinates,
//   dw_out   (sum of frame sizes): per-point weights.
// Correspondences are piecewise constant (zero gradient).  opts->omega_grad_full selects
// whether Omega = (C~ + R C R^T)^-1 is differentiated through R (1) or frozen (0).
int orc_gradient(const orc_frame* frames, int nframes, void* const* vmaps, const orc_pair* pairs,
                 int npairs, const double* poses12, const orc_opts* opts, double* dxi_out,
                 double* dmu_out, double* dw_out) {
  std::vector<int64_t> foff(nframes + 1, 0);
  for (int f = 0; f < nframes; ++f) foff[f + 1] = foff[f] + frames[f].n;
  std::fill(dxi_out, dxi_out + 6 * nframes, 0.0);
  std::fill(dmu_out, dmu_out + 3 * foff[nframes], 0.0);
  std::fill(dw_out, dw_out + foff[nframes], 0.0);
  for (int p = 0; p < npairs; ++p) {
    const int s = pairs[p].src, t = pairs[p].tgt;
    const orc_frame& F = frames[s];
    const VMap& tgt = *static_cast<const VMap*>(vmaps[t]);
    const int L = int(tgt.levels.size());
    PairCtx pc = make_pair_ctx(poses12, s, t);
    const Pose& T = pc.rel;
    for (int64_t k = 0; k < F.n; ++k) {
      const float* mu4 = F.pts4 + 4 * k;
      Corr c = correspond(tgt, pc.Rf, pc.tf, pc.vf, mu4, F.normal3 ? F.normal3 + 3 * k : nullptr,
                          opts->validate_surface != 0);
      const double w = mu4[3];
      V3 mu = {mu4[0], mu4[1], mu4[2]};
      double c6[6];
      for (int i = 0; i < 6; ++i) c6[i] = F.cov6[6 * k + i];
      M3 C = sym_from6(c6);
      M3 RCRt = mul(mul(T.R, C), transpose(T.R));
      V3 q = mulv(T.R, mu);
      for (int i = 0; i < 3; ++i) q[i] += T.t[i];
      for (int l = 0; l < L; ++l) {
        if (!c.vox[l]) continue;
        const Voxel& v = *c.vox[l];
        M3 S = sym_from6(v.cov);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) S[i][j] += RCRt[i][j];
        M3 Om;
        if (opts->omega_identity) Om = M3{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
        else if (!spd_inverse(S, Om)) continue;
        V3 d = {v.mean[0] - q[0], v.mean[1] - q[1], v.mean[2] - q[2]};
        V3 Od = mulv(Om, d);
        const double e = d[0] * Od[0] + d[1] * Od[1] + d[2] * Od[2];
        // dE/dd = 2 w Omega d;  d depends on xi through q (Eqs. (4)-(5)) and on mu through -R mu
        M3 A1 = mul(T.R, hat(mu));  // d d / d omega_s
        M3 qx = hat(q);
        for (int a = 0; a < 3; ++a) {
          double gs_w = 0, gs_v = 0, gt_w = 0, gt_v = 0;
          for (int i = 0; i < 3; ++i) {
            gs_w += A1[i][a] * Od[i];
            gs_v += -T.R[i][a] * Od[i];
            gt_w += -qx[i][a] * Od[i];
            gt_v += (i == a ? 1.0 : 0.0) * Od[i];
          }
          dxi_out[6 * s + a] += 2.0 * w * gs_w;
          dxi_out[6 * s + 3 + a] += 2.0 * w * gs_v;
          dxi_out[6 * t + a] += 2.0 * w * gt_w;
          dxi_out[6 * t + 3 + a] += 2.0 * w * gt_v;
        }
        if (opts->omega_grad_full && !opts->omega_identity) {
          // dE/dS = -w Omega d d^T Omega;  S depends on the rotations through R C R^T:
          //   dS/d omega_s,a = R (e_a x C - C e_a x) R^T
          //   dS/d omega_t,a = -(e_a x) R C R^T + R C R^T (e_a x)
          M3 G;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) G[i][j] = -w * Od[i] * Od[j];
          for (int a = 0; a < 3; ++a) {
            V3 ea = {0, 0, 0};
            ea[a] = 1.0;
            M3 E = hat(ea);
            M3 X = mul(E, C), Y = mul(C, E);
            M3 D;
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j) D[i][j] = X[i][j] - Y[i][j];
            M3 dSs = mul(mul(T.R, D), transpose(T.R));
            M3 P1 = mul(E, RCRt), P2 = mul(RCRt, E);
            double cs = 0, ct = 0;
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j) {
                cs += G[i][j] * dSs[i][j];
                ct += G[i][j] * (-P1[i][j] + P2[i][j]);
              }
            dxi_out[6 * s + a] += cs;
            dxi_out[6 * t + a] += ct;
          }
        }
        // dE/dmu = -2 w R^T Omega d ;  dE/dw = e
        V3 RtOd = mulv(transpose(T.R), Od);
        for (int i = 0; i < 3; ++i) dmu_out[3 * (foff[s] + k) + i] += -2.0 * w * RtOd[i];
        dw_out[foff[s] + k] += e;
      }
    }
  }
  return ORC_OK;
}

// Gauss-Newton step xi = -H^-1 b for a dim x dim system (dim 6 or 12) by Cholesky in FP64.
int orc_gn_solve(const double* H, const double* b, int dim, double* xi_out) {
  if (dim <= 0 || dim > 12) return ORC_EINVAL;
  double L[12][12] = {};
  for (int j = 0; j < dim; ++j) {
    double d = H[dim * j + j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !std::isfinite(d)) return ORC_ENOTPD;
    L[j][j] = std::sqrt(d);
    for (int i = j + 1; i < dim; ++i) {
      double s = H[dim * i + j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  double y[12];
  for (int i = 0; i < dim; ++i) {
    double s = -b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = dim - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < dim; ++k) s -= L[k][i] * xi_out[k];
    xi_out[i] = s / L[i][i];
  }
  return ORC_OK;
}

// One step of a small factor graph (Sec. V-A: the submaps of local mapping are optimised with
// all-to-all matching-cost factors by Levenberg-Marquardt).  Each factor p contributes its
// quadratic form over [xi_src; xi_tgt]: its 6 x 6 blocks are added to the blocks (src, src),
// (src, tgt), (tgt, src), (tgt, tgt) of the global H and its two 6-vectors to the entries of b.
// The variables of frame `fixed` (-1: none) are removed (the gauge of relative factors), the
// remaining diagonal is damped by (1 + lambda), and (H_ff + lambda diag(H_ff)) xi_f = -b_f is
// solved by Cholesky; xi of the fixed frame is zero.  Hg_out (6n x 6n) and bg_out (6n) receive
// the undamped assembled system (nullable).  ORC_ENOTPD if the reduced system is not positive
// definite.
int orc_graph_step(const int32_t* pair_frames, int npairs, int nframes, const double* H, const double* b,
                   int fixed, double lambda, double* xi_out, double* Hg_out, double* bg_out) {
  if (nframes < 1 || npairs < 0 || fixed < -1 || fixed >= nframes) return ORC_EINVAL;
  const int N = 6 * nframes;
  std::vector<double> Hg(size_t(N) * N, 0.0), bg(N, 0.0);
  for (int p = 0; p < npairs; ++p) {
    const int f[2] = {pair_frames[2 * p], pair_frames[2 * p + 1]};
    if (f[0] < 0 || f[0] >= nframes || f[1] < 0 || f[1] >= nframes) return ORC_EINVAL;
    for (int u = 0; u < 2; ++u) {
      for (int a = 0; a < 6; ++a) bg[6 * f[u] + a] += b[12 * p + 6 * u + a];
      for (int v = 0; v < 2; ++v)
        for (int a = 0; a < 6; ++a)
          for (int c = 0; c < 6; ++c)
            Hg[size_t(6 * f[u] + a) * N + 6 * f[v] + c] += H[144 * p + (6 * u + a) * 12 + 6 * v + c];
    }
  }
  if (Hg_out) std::memcpy(Hg_out, Hg.data(), Hg.size() * sizeof(double));
  if (bg_out) std::memcpy(bg_out, bg.data(), bg.size() * sizeof(double));
  std::vector<int> free_vars;
  for (int i = 0; i < N; ++i)
    if (fixed < 0 || i / 6 != fixed) free_vars.push_back(i);
  const int M = int(free_vars.size());
  std::vector<double> A(size_t(M) * M), L(size_t(M) * M, 0.0), y(M), x(M);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      double v = Hg[size_t(free_vars[i]) * N + free_vars[j]];
      if (i == j) v += lambda * v;
      A[size_t(i) * M + j] = v;
    }
  for (int j = 0; j < M; ++j) {  // A = L L^T
    double d = A[size_t(j) * M + j];
    for (int k = 0; k < j; ++k) d -= L[size_t(j) * M + k] * L[size_t(j) * M + k];
    if (!(d > 0.0) || !std::isfinite(d)) return ORC_ENOTPD;
    L[size_t(j) * M + j] = std::sqrt(d);
    for (int i = j + 1; i < M; ++i) {
      double t = A[size_t(i) * M + j];
      for (int k = 0; k < j; ++k) t -= L[size_t(i) * M + k] * L[size_t(j) * M + k];
      L[size_t(i) * M + j] = t / L[size_t(j) * M + j];
    }
  }
  for (int i = 0; i < M; ++i) {  // L y = -b_f
    double t = -bg[free_vars[i]];
    for (int k = 0; k < i; ++k) t -= L[size_t(i) * M + k] * y[k];
    y[i] = t / L[size_t(i) * M + i];
  }
  for (int i = M - 1; i >= 0; --i) {  // L^T x = y
    double t = y[i];
    for (int k = i + 1; k < M; ++k) t -= L[size_t(k) * M + i] * x[k];
    x[i] = t / L[size_t(i) * M + i];
  }
  for (int i = 0; i < N; ++i) xi_out[i] = 0.0;
  for (int i = 0; i < M; ++i) xi_out[free_vars[i]] = x[i];
  return ORC_OK;
}

// Overlap rate: fraction of source points with a voxel of the target at level ``level``
// under the relative pose (Sec. IV-B), surface test off.
double orc_overlap(const orc_frame* src, const void* vmap, const double* pose_s12,
                   const double* pose_t12, int level) {
  const VMap& tgt = *static_cast<const VMap*>(vmap);
  double poses[24];
  std::memcpy(poses, pose_s12, 12 * sizeof(double));
  std::memcpy(poses + 12, pose_t12, 12 * sizeof(double));
  PairCtx pc = make_pair_ctx(poses, 0, 1);
  int64_t hits = 0;
  for (int64_t k = 0; k < src->n; ++k) {
    Corr c = correspond(tgt, pc.Rf, pc.tf, pc.vf, src->pts4 + 4 * k, nullptr, false);
    if (c.vox[level]) ++hits;
  }
  return src->n ? double(hits) / double(src->n) : 0.0;
}

}  // extern "C"
