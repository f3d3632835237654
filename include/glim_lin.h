/* glim_lin.h -- C ABI of the B300 linearization library for GLIM matching-cost factors.
 *
 * The library evaluates the voxelized-GICP matching-cost factor of GLIM (Koide et al.,
 * "GLIM: 3D Range-Inertial Localization and Mapping with GPU-Accelerated Scan Matching
 * Factors", Sec. III-C) on one CUDA device:
 *
 *   e    = sum_l sum_k  w_k d_kl^T Omega_kl d_kl                       Eqs. (2)-(3)
 *   d_kl = mu~_l(k) - T_rel mu_k,   Omega_kl = (C~_l(k) + R C_k R^T)^-1
 *   A_k  = [R (mu_k)x, -R],  B_k = [-(T_rel mu_k)x, I]                 Eqs. (4)-(5)
 *   H    = sum [A B]^T Omega [A B],  b = sum [A B]^T Omega d           Eqs. (6)-(8)
 *
 * Conventions (the paper leaves them open or prints them inconsistently):
 *   - a factor pairs a SOURCE frame s (its points mu_k, covariances C_k) with a TARGET
 *     frame t (its voxelmap); T_rel = T_t^-1 T_s; poses are perturbed on the right,
 *     T <- T Exp(xi), xi = [omega; v] (rotation first).  With these, A_k and B_k above are
 *     the exact derivatives of d_k w.r.t. xi_s and xi_t.
 *   - H is 12 x 12 over [xi_s; xi_t], b has 12 entries; a unary factor (target fixed)
 *     uses the top-left 6 x 6 block of H and the first 6 entries of b.  With
 *     e(xi) ~ e + 2 b^T xi + xi^T H xi, the Gauss-Newton step is xi = -H^-1 b.
 *   - voxel key = floor(q * inv_r) per axis on the FP32 path: q is formed from the FP32
 *     rounding of T_rel with one fused multiply-add per term (t, then x, y, z), inv_r is
 *     the FP32 rounding of 1/r.  Keys must lie in [-2^20, 2^20).
 *   - a voxel holds the mean of its points and the mean of their covariances
 *     (Sec. III-C "Preprocessing"); level l uses resolution r_l (e.g. r_0 2^(l-1)).
 *   - surface validation (Sec. III-C "Correspondence search", Fig. 3): a source point is
 *     discarded when (mu_k - T_s^-1 t_t) . n_k > 0, evaluated in FP32 as
 *     s = n_x d_x; s = fma(n_y, d_y, s); s = fma(n_z, d_z, s) with d = mu_k - v.
 *
 * Memory and ownership: every array argument documented "device" is a pointer to memory
 * on the context's device, owned by the caller (for example a PyTorch tensor's storage),
 * contiguous in the layout stated.  "host" arguments are ordinary host memory.  Objects
 * returned through out-parameters (contexts, voxelmaps, plans) are owned by the library
 * and released with the matching destroy/free call.  Work is enqueued on the context's
 * stream; a call that returns host results synchronizes that stream first.
 *
 * Errors: no function throws or aborts.  Every call returns a glim_status; on failure
 * glim_last_error() describes it.  Device-side conditions (hash table full, key out of
 * range, non-finite input, bounded waits that gave up) are reported through status
 * words that the host reads, never by trapping the device.
 */
#ifndef GLIM_LIN_H
#define GLIM_LIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t glim_status;
#define GLIM_OK 0
#define GLIM_EINVAL -1    /* invalid argument or non-finite input */
#define GLIM_ENOMEM -2    /* device or pinned allocation failed */
#define GLIM_ECUDA -3     /* a CUDA runtime call failed */
#define GLIM_EHASHFULL -4 /* voxel hash table could not place a key */
#define GLIM_ERANGE -5    /* a voxel key lies outside [-2^20, 2^20) */
#define GLIM_ENOTPD -6    /* a Gauss-Newton system is not positive definite */
#define GLIM_ETIMEOUT -7  /* a bounded device wait gave up */

#define GLIM_MAX_LEVELS 4

/* A factor record: the linearization of one pair in GLIM_RECORD_DOUBLES doubles, for
 * exchange between processes (the per-pair {e, H, b} that a multi-GPU global step gathers to
 * the rank that assembles the system): [0] e; [1 .. 78] the upper triangle of the symmetric
 * H, row-major (H[0][0..11], H[1][1..11], ..., H[11][11]); [79 .. 90] b; [91] the inlier
 * count. */
#define GLIM_RECORD_DOUBLES 92

/* Accumulation modes of the per-point sums (precision of the partial sums of H, b, e). */
#define GLIM_ACC_FP32 0  /* FP32 everywhere, including the cross-block sum (naive) */
#define GLIM_ACC_KAHAN 1 /* FP32 with compensated (Kahan/Neumaier) per-thread and tree sums,
                            FP64 across blocks */
#define GLIM_ACC_FP64 2  /* FP32 per thread and per warp, FP64 across warps and blocks */

typedef struct glim_ctx glim_ctx;
typedef struct glim_vmap glim_vmap;
typedef struct glim_plan glim_plan;

/* A frame: n points of one scan or submap in its own coordinates (device pointers).
 *   pts4    n x float4 (x, y, z, w); w is the point's weight (1 for the paper's cost).
 *   cov6    n x 6 floats (xx, xy, xz, yy, yz, zz), the point covariance C_k.
 *   normal3 n x 3 floats, the surface normal n_k; NULL disables surface validation
 *           for points of this frame.  Each pointer must be 16-byte (pts4) or 8-byte
 *           (cov6) aligned. */
typedef struct {
  const float* pts4;
  const float* cov6;
  const float* normal3;
  int64_t n;
} glim_frame;

/* A factor: source frame index, target frame index, and the target's voxelmap. */
typedef struct {
  int32_t src_frame;
  int32_t tgt_frame;
  const glim_vmap* tgt;
} glim_pair;

/* Launch options of the linearization kernels.  Zero fields take defaults.
 *   validate_surface  1 = apply the surface-orientation test.
 *   accum_mode        GLIM_ACC_*.
 *   block             threads per block (64, 128 or 256, 64 for the per-lane dense-grid and
 *                     hash kernels only; default 256).
 *   pts_per_thread    points per thread per work item (1..256; default 16);
 *                     a work item (tile) covers block * pts_per_thread points of one pair.
 *   blocks_per_sm     resident blocks per SM of the persistent kernel (default: occupancy).
 *   persistent        1 (default) = one persistent kernel over an atomic work queue;
 *                     2 = one block per work item (hardware scheduling).
 *   kernel            0 (default) = the per-lane dense-grid kernel when every level of
 *                     every target map is a dense grid, the per-lane hash kernel when every
 *                     one is a hash table, else the general kernel; 1 = the general kernel
 *                     (any mix of dense grids and hash tables); 2 = the dense-grid kernel,
 *                     3 = the hash kernel (GLIM_EINVAL if a target level has the other
 *                     layout).  The per-lane kernels form a coarser level's key as the
 *                     level-0 key shifted right, so they also need every target map's
 *                     resolutions to double from level to level (r_l = r_0 2^l, the paper's
 *                     multi-resolution maps); other maps take the general kernel by default
 *                     and GLIM_EINVAL with 2 or 3.  All give the same results up to FP32
 *                     rounding order.
 *   reserved          must be 0. */
typedef struct {
  int32_t validate_surface;
  int32_t accum_mode;
  int32_t block;
  int32_t pts_per_thread;
  int32_t blocks_per_sm;
  int32_t persistent;
  int32_t kernel;
  int32_t reserved;
} glim_lin_opts;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, enqueuing work on `cuda_stream`
 * (a cudaStream_t; NULL = a new non-blocking stream owned by the context). */
glim_status glim_create(glim_ctx** out, int device, void* cuda_stream);
void glim_destroy(glim_ctx* ctx);
/* Text of the last error on this context (never NULL; empty after success). */
const char* glim_last_error(const glim_ctx* ctx);
/* Number of SMs of the context's device. */
int32_t glim_num_sms(const glim_ctx* ctx);
/* Number of kernels this context has launched since creation (for accounting). */
int64_t glim_kernel_launches(const glim_ctx* ctx);
/* Testing hook with no counterpart in the paper: the allocation n allocations from now
 * (0 = the next one) among all device and pinned host allocations of the library, in any
 * context and thread, fails once as if the device were out of memory, so that tests reach
 * every GLIM_ENOMEM path without exhausting a GPU.  n < 0 disables it (the default).  The
 * call that meets the failure returns GLIM_ENOMEM (GLIM_ECUDA where the failure surfaces
 * through a CUDA call's own status) and leaves its objects as they were. */
void glim_debug_fail_allocation(int64_t n);
/* Measured FP32 multiply-add throughput of the context's device in TFLOP/s (two flops per
 * FMA): eight independent register-resident FMA chains per thread, eight 256-thread blocks
 * per SM, `iters` x 128 FMAs per thread, best of three timed launches after a warm-up.  The
 * denominator of the FP32 roofline of the linearization kernel.  Synchronizes the stream. */
glim_status glim_fp32_fma_peak(glim_ctx* ctx, int32_t iters, double* tflops_out);
/* The same measurement with FP64 chains (`__fma_rn` on doubles): the device's FP64 FMA rate
 * in TFLOP/s.  B300's FP64 rate is a small fraction of its FP32 rate, so `iters` should be
 * correspondingly smaller.  Synchronizes the stream.  GLIM_EINVAL if iters < 1. */
glim_status glim_fp64_fma_peak(glim_ctx* ctx, int32_t iters, double* tflops_out);

/* ---------------------------------------------------------------- covariances */

/* Per-point covariance from the k nearest neighbours (Sec. III-C "Preprocessing";
 * Sec. IV-A): exact kNN over the frame, the point itself included, ties broken by
 * (squared distance in FP64, index); sample covariance with 1/k normalisation; then
 *   reg_mode 0: C = C_sample + eps I
 *   reg_mode 1: C = I - (1 - eps) n n^T (GICP plane regularisation), n = eigenvector of
 *               the smallest eigenvalue, oriented so that n . mu <= 0.
 * pts4 (device, n x float4), cov6_out (device, n x 6), normal3_out (device, n x 3, or
 * NULL).  3 <= k <= 32, k <= n. */
glim_status glim_estimate_covariances(glim_ctx* ctx, const float* pts4, int64_t n, int32_t k,
                                      int32_t reg_mode, float eps, float* cov6_out,
                                      float* normal3_out);

/* The same, also writing the neighbour sets: knn_out (device, n x k int32, or NULL) receives
 * the indices of every point's k nearest neighbours in (squared distance in FP64, index)
 * order, nearest first (the point itself included).  For inspection and parity tests. */
glim_status glim_estimate_covariances_knn(glim_ctx* ctx, const float* pts4, int64_t n, int32_t k,
                                          int32_t reg_mode, float eps, float* cov6_out,
                                          float* normal3_out, int32_t* knn_out);

/* ---------------------------------------------------------------- point order */

/* Permutation that orders a frame's points along a Z-order (Morton) curve of cubic cells of
 * size `cell` (metres): perm_out[i] is the index of the point placed at position i (device,
 * n int32).  Points with equal cells keep their relative order.  Applying it to a frame (as
 * voxel-grid downsampling or a scan-line order would) keeps neighbouring points together, so
 * the lanes of a warp read the same voxel records.  The linearization result does not depend
 * on the point order beyond floating-point rounding.  GLIM_ERANGE if a cell coordinate is
 * outside [-2^20, 2^20). */
glim_status glim_spatial_order(glim_ctx* ctx, const float* pts4, int64_t n, float cell,
                               int32_t* perm_out);

/* ---------------------------------------------------------------- voxelmaps */

/* Build the multi-resolution voxelmap of one frame (Sec. III-C "Preprocessing"): for each
 * level, the occupied voxels with the mean of their points and covariances, stored in a dense
 * grid or in hashed voxel blocks (see glim_build_voxelmap_ex).  pts4 / cov6 are device
 * arrays (n x float4, n x 6); resolutions is a host array of `levels` voxel sizes.
 * Returns GLIM_ERANGE if a key is outside [-2^20, 2^20), GLIM_EINVAL on non-finite input.
 * Synchronizes the stream.  The voxelmap keeps no reference to the input arrays. */
glim_status glim_build_voxelmap(glim_ctx* ctx, const float* pts4, const float* cov6, int64_t n,
                                const double* resolutions, int32_t levels, glim_vmap** out);
/* As glim_build_voxelmap, choosing the table layout of every level:
 *   layout 0 (default): a dense grid over the bounding box of the occupied keys whose cells
 *            hold the voxel records (48 bytes per cell) when the box has at most 256 cells
 *            per voxel plus 2^22 cells and needs at most 32 GiB, else hashed voxel blocks;
 *   layout 1: dense grid (GLIM_EINVAL if the bounding box exceeds the limit);
 *   layout 2: hashed voxel blocks: blocks of 2 x 2 x 2 voxels whose 8 cells hold the records,
 *            found through an open-addressing table of the block keys (linear probing, load
 *            <= 1/16), as voxel hashing stores voxel blocks.
 * Both layouts give identical correspondences and results; the dense grid resolves every
 * lookup, hit or miss, with one 48-byte read, the hashed layout with one table-entry read of
 * the block (one per probe) and one 48-byte read. */
glim_status glim_build_voxelmap_ex(glim_ctx* ctx, const float* pts4, const float* cov6, int64_t n,
                                   const double* resolutions, int32_t levels, int32_t layout,
                                   glim_vmap** out);
/* Free a voxelmap.  Waits for the device first, so that launches in flight on any stream that
 * read its tables complete.  Plans created on the map keep pointers to its tables: destroy
 * them before freeing the map. */
void glim_vmap_free(glim_vmap* vmap);
/* Incremental insertion (NEXT: submaps grow as frames are merged into them, Sec. V-A; the
 * voxel statistics are the running means of Sec. III-C).  Adds n map-frame points (pts4 /
 * cov6 laid out and aligned as for glim_build_voxelmap, device memory, borrowed) to every
 * level of vmap.  Per voxel the FP64 sums of the existing members and of the new points
 * are added and the means recomputed; the canonical ids are again the ranks of the keys,
 * so the result equals glim_build_voxelmap of all points ever inserted (keys, ids and
 * counts exactly; statistics up to the order of the FP64 additions).  layout as for
 * glim_build_voxelmap_ex (0 re-decides from the grown key box).  The device is
 * synchronised before the old tables are freed.  Plans created on vmap before the call
 * fail with GLIM_EINVAL afterwards (their table pointers are stale): create new ones.
 * On error vmap is unchanged: GLIM_EINVAL for bad arguments or non-finite input,
 * GLIM_ERANGE for a key outside [-2^20, 2^20), GLIM_EINVAL for layout 1 when the grown
 * box exceeds the dense limit, GLIM_ENOMEM. */
glim_status glim_vmap_insert(glim_ctx* ctx, glim_vmap* vmap, const float* pts4, const float* cov6,
                             int64_t n, int32_t layout);
/* Number of occupied voxels, capacity in cells (grid cells of a dense level, the cells of the
 * allocated blocks of a hashed level) and longest probe sequence of the block table (1 for a
 * dense level) of a level. */
glim_status glim_vmap_info(const glim_vmap* vmap, int32_t level, int64_t* n_voxels,
                           int64_t* capacity, int32_t* max_probe);
/* 1 if the level uses a dense index grid, 0 for a hash table, -1 for a bad argument. */
int32_t glim_vmap_is_dense(const glim_vmap* vmap, int32_t level);
/* Copy a level's voxels to device arrays in canonical order (lexicographic (x, y, z) key
 * order; the position is the canonical voxel id): keys3 (n_voxels x 3 int32), mean3
 * (n_voxels x 3), cov6 (n_voxels x 6), count (n_voxels int32).  Any output may be NULL. */
glim_status glim_vmap_export(glim_ctx* ctx, const glim_vmap* vmap, int32_t level, int32_t* keys3,
                             float* mean3, float* cov6, int32_t* count);

/* Canonical voxel id of every source point at every level of the target map under the
 * relative pose T_t^-1 T_s (host poses, 12 doubles [R|t] row-major each), or -1 for a
 * miss or a point discarded by surface validation.  ids_out: device, n x levels int32. */
glim_status glim_correspondences(glim_ctx* ctx, const glim_frame* src, const glim_vmap* tgt,
                                 const double* pose_s12, const double* pose_t12,
                                 int32_t validate_surface, int32_t* ids_out);

/* Overlap rate (Sec. IV-B): for every pair, the fraction of the source points that fall in
 * an occupied voxel of the target at `level` (surface validation off).  frames, pairs and
 * poses12 (nframes x 12 doubles) are host arrays; overlap_out is a device array of npairs
 * doubles.  One launch for all pairs. */
glim_status glim_overlap(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                         const glim_pair* pairs, int32_t npairs, const double* poses12,
                         int32_t level, double* overlap_out);

/* ---------------------------------------------------------------- linearization */

/* Linearize every factor of a batch in one pass (Sec. III-C "Linearization" and
 * "Implementation"): frames (host array of nframes descriptors), pairs (host array),
 * poses12 (host, nframes x 12 doubles).  Outputs e_out (npairs), H_out (npairs x 144,
 * row-major 12 x 12), b_out (npairs x 12), inliers_out (npairs, number of (point, level)
 * terms that entered the sums: correspondences whose S = C~ + R C R^T is positive definite;
 * may be NULL) are all host or all device arrays; with host outputs the
 * call synchronizes.  Builds a temporary plan; repeated linearizations of the same batch
 * should use glim_plan_*. */
glim_status glim_linearize_factors(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                   const glim_pair* pairs, int32_t npairs, const double* poses12,
                                   const glim_lin_opts* opts, double* e_out, double* H_out,
                                   double* b_out, int64_t* inliers_out);

/* Plain per-factor form, for comparison: one kernel launch per factor followed by a stream
 * synchronization and a copy of that factor's result, as a for-loop over factors would do.
 * Same arguments and results as glim_linearize_factors (FP32 accumulation). */
glim_status glim_linearize_factors_plain(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                         const glim_pair* pairs, int32_t npairs,
                                         const double* poses12, const glim_lin_opts* opts,
                                         double* e_out, double* H_out, double* b_out,
                                         int64_t* inliers_out);

/* For callers that cannot allocate device memory while they linearize: processes whose device
 * memory is reserved up front by another allocator, so that a cudaMalloc may fail or wait, and
 * real-time loops that must not block in the driver (cudaFree synchronizes the device).  The
 * paper has no counterpart; this is a service of the library.
 *
 * Same computation and arguments as glim_linearize_factors, except that e_out, H_out, b_out
 * and inliers_out (may be NULL) must be device arrays, and that the call allocates nothing:
 * its scratch (descriptors, work list, queue head, partial sums) is one statically sized array
 * of about 4.5 MB that every device loading this library holds until the process exits.
 * Limits: at most 256 frames, 256 pairs and 16384 work items of block * pts_per_thread points
 * (GLIM_EINVAL with a message naming the limit otherwise).  The first call on a device sets it
 * up (looks up that array's device address, fills a constant part of it and waits for that
 * fill, creates an event, and once per process page-locks the library's host staging block
 * with cudaHostRegister); make that first call before any stream capture.  The descriptors are
 * staged in that one host block, which every call rewrites, so a call made while the context's
 * stream is capturing returns GLIM_EINVAL without enqueuing anything.  Every call shares the
 * device array and overwrites it (the queue head is cleared on each call), so calls that
 * overlap on the GPU, from any stream or thread, race: issue them one after another.  The work
 * is enqueued on the context's stream.  The call does not wait for that stream, except that it
 * first waits until the previous call's upload of the staging block has been read, which is
 * ordered after only the work that preceded the previous call. */
glim_status glim_linearize_factors_noalloc(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                                           const glim_pair* pairs, int32_t npairs,
                                           const double* poses12, const glim_lin_opts* opts,
                                           double* e_out, double* H_out, double* b_out,
                                           int64_t* inliers_out);

/* A plan fixes a batch (frames, pairs, options) and owns its device work list, partial-sum
 * slots, a pinned staging block for the frame poses (nframes x 12 doubles, the only pose data
 * uploaded), the device pose block that a packing kernel forms from them (per pair T_rel =
 * T_t^-1 T_s in FP64, its FP32 rounding and the target viewpoint; the same bits as the host
 * arithmetic of the one-shot calls), a pinned output block (e, H, b, inliers), and a CUDA
 * graph of [upload, pose packing, queue reset, linearize, reduce, download].  The frames and
 * voxelmaps must stay alive and unchanged while the plan exists. */
glim_status glim_plan_create(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                             const glim_pair* pairs, int32_t npairs, const glim_lin_opts* opts,
                             glim_plan** out);
void glim_plan_destroy(glim_plan* plan);
/* Linearize at poses12 (host, nframes x 12 doubles): one upload, one graph launch, one
 * download.  Outputs as in glim_linearize_factors (host or device). */
glim_status glim_plan_linearize(glim_plan* plan, const double* poses12, double* e_out,
                                double* H_out, double* b_out, int64_t* inliers_out);
/* The same without the final host copy: runs the graph, synchronizes and returns pointers
 * into the plan's pinned host output block (e: npairs, H: npairs x 144, b: npairs x 12
 * doubles, inliers: npairs int64), valid until the plan's next launch or destruction. */
glim_status glim_plan_linearize_pinned(glim_plan* plan, const double* poses12, const double** e,
                                       const double** H, const double** b, const int64_t** inliers);
/* Device-resident use: glim_plan_set_poses uploads the frame poses and packs the pairs'
 * relative poses on the device (async);
 * glim_plan_launch enqueues queue reset, linearize and reduce (no copies, no sync) and
 * leaves the results in the plan's device output block, whose arrays
 * glim_plan_device_outputs returns (e: npairs doubles, H: npairs x 144, b: npairs x 12,
 * inliers: npairs int64). */
glim_status glim_plan_set_poses(glim_plan* plan, const double* poses12);
/* Copy the plan's current device pose block to the host (synchronizes): rt64_out (npairs x 12
 * doubles, [R row-major | t] of T_rel) and pose32_out (npairs x 16 floats: R, t, v, 0), either
 * may be NULL.  For inspection and tests of the pose packing. */
glim_status glim_plan_relative_poses(glim_plan* plan, double* rt64_out, float* pose32_out);
/* Correspondences as the plan's own kernel resolves them (Sec. III-C "Correspondence search":
 * one voxel per level, key floor(q * inv_r) on the FP32 path).  Runs the id-recording
 * instantiation of the linearization kernel that the plan uses (general, dense-grid or hash;
 * the same lookup and hit code, block size, tile and work queue, accumulation mode
 * GLIM_ACC_FP64) at poses12 (host, nframes x 12 doubles), and writes the canonical voxel id of
 * every source point at every level of its pair's target map, or -1 (a miss, a point
 * discarded by surface validation, a masked or non-finite point), to ids_out: device,
 * int32, per pair n_src x levels (point-major), pairs concatenated in order.  The e, H, b and
 * inlier counts of the same launch are copied to e_out, H_out, b_out, inliers_out (host
 * arrays as for glim_plan_linearize; each may be NULL).  For inspection and parity tests;
 * synchronizes.  GLIM_EINVAL for a null ids_out with pairs, or a plan whose maps changed. */
glim_status glim_plan_correspondence_ids(glim_plan* plan, const double* poses12, int32_t* ids_out,
                                         double* e_out, double* H_out, double* b_out,
                                         int64_t* inliers_out);
glim_status glim_plan_launch(glim_plan* plan);
glim_status glim_plan_device_outputs(glim_plan* plan, double** e, double** H, double** b,
                                     int64_t** inliers);
/* Device pointer to the plan's factor records (npairs x GLIM_RECORD_DOUBLES doubles, pair
 * order), written by every linearization of the plan together with its other outputs; valid
 * until the plan is destroyed.  H in every output of the library is exactly symmetric: its
 * record holds every entry. */
glim_status glim_plan_device_records(glim_plan* plan, double** rec);
/* Kernels enqueued per glim_plan_launch (queue reset excluded). */
int32_t glim_plan_kernels_per_launch(const glim_plan* plan);
/* Timing support: enqueue like glim_plan_launch but with direct launches (no graph), and
 * record two CUDA events on the context's stream immediately before and after the
 * linearization kernel, in timing slot `slot` (0 <= slot < 4096). */
glim_status glim_plan_launch_timed(glim_plan* plan, int32_t slot);
/* Wait for timing slots [0, nslots) and write each slot's linearization-kernel duration in
 * milliseconds to ms_out (host array of nslots floats). */
glim_status glim_plan_kernel_ms(glim_plan* plan, int32_t nslots, float* ms_out);
/* Autotuner: time every (block, pts_per_thread) candidate of the persistent kernel on this
 * plan's batch at poses12 with CUDA events (`iters` timed launches each, after one warm-up):
 * block 128 or 256 with 4, 8, 16, 32 or 64 points per thread, and per block size the points
 * per thread that make the batch's tiles about one resident wave of blocks;
 * keep the fastest in the plan, and write it to best_out (may be NULL).  On an error the
 * plan returns to its original configuration where that succeeds, and otherwise keeps the
 * last configuration that did: it stays launchable either way. */
glim_status glim_plan_autotune(glim_plan* plan, const double* poses12, int32_t iters,
                               glim_lin_opts* best_out, float* best_ms_out);
/* The options the plan currently uses. */
glim_status glim_plan_get_opts(const glim_plan* plan, glim_lin_opts* out);

/* ---------------------------------------------------------------- gradient */

/* Gradient of E = sum over pairs of e (Eq. (2), with the weights w_k) at poses12 (host),
 * correspondences held fixed (piecewise constant):
 *   dxi_out   device, nframes x 6 doubles: dE/dxi of every frame pose (right perturbation)
 *   dmu_out   device, the frames' points concatenated in frame order, 3 floats per point:
 *             dE/dmu_k
 *   dw_out    device, same concatenation, 1 float per point: dE/dw_k
 * omega_grad_full = 1 differentiates Omega = (C~ + R C R^T)^-1 through R as well;
 * 0 holds Omega fixed (then dE/dxi = 2 b).  dE/dmu_k = -2 w_k sum_l R^T Omega_kl d_kl and
 * dE/dw_k = sum_l d_kl^T Omega_kl d_kl.  Per-point outputs are written, not accumulated;
 * points of frames that are never a source get zeros.  Deterministic (no float atomics). */
glim_status glim_backward(glim_ctx* ctx, const glim_frame* frames, int32_t nframes,
                          const glim_pair* pairs, int32_t npairs, const double* poses12,
                          int32_t omega_grad_full, int32_t validate_surface, double* dxi_out,
                          float* dmu_out, float* dw_out);
/* The same gradient for the batch of a plan, so that repeated evaluations (an optimiser's
 * iterations, autograd) reuse the plan's descriptors; its validate_surface option applies
 * (its tile options do not: the gradient pass has its own work list of (source frame, point
 * tile) items that walk all pairs of their source).  The gradient scratch (host tables, one
 * slot of 9 sums per (item, pair), per-pair gradients; no per-(pair, point) storage) is
 * allocated at the first call and kept until glim_plan_destroy.  The frames' point arrays may be rewritten in
 * place between calls, by work ordered on the context stream (or after synchronizing it).
 * Outputs as for glim_backward, written by work enqueued on the context stream: the call does
 * not wait for it (the first call waits once, to build the gradient tables).  When poses12
 * equals the poses of the plan's last linearization or upload, the pose block on the device
 * is reused and the call does not wait for the stream at all; otherwise it first waits for
 * the stream's earlier work (the pinned pose staging block may still be in use). */
glim_status glim_plan_backward(glim_plan* plan, const double* poses12, int32_t omega_grad_full,
                               double* dxi_out, float* dmu_out, float* dw_out);

/* ---------------------------------------------------------------- Gauss-Newton step */

/* Gauss-Newton on the device for one frame with every other frame fixed (Sec. III-C: the
 * quadratic factors' Gauss-Newton step, xi = -H^-1 b, and the pose update T <- T Exp(xi)):
 * starting from poses12 (host, nframes x 12 doubles), `iters` times linearize the plan's
 * batch, sum the 6 x 6 systems of `frame` over the pairs in pair order (the source block
 * H[0:6, 0:6], b[0:6] of the pairs whose source it is, the target block H[6:12, 6:12],
 * b[6:12] of the pairs whose target it is), solve by Cholesky in FP64 and update the frame's
 * pose on the device, T <- T Exp(xi), xi = [omega; v], Exp(xi) = [Exp(omega) | V v]
 * (Rodrigues; V the left Jacobian of SO(3)).  No host round trip between iterations.
 * Writes the final poses to poses12_out (host, nframes x 12), the batch's total cost at each
 * linearization to cost_out (host, iters doubles, may be NULL) and GLIM_OK, or GLIM_ENOTPD
 * when a system was not positive definite (that iteration takes no step), to *status_out
 * (may be NULL).  The plan's device poses are the final ones afterwards; its outputs hold
 * the last linearization (at the poses before the last step).  Synchronizes.  GLIM_EINVAL
 * for a bad frame index, iters < 1 or a plan whose maps changed. */
glim_status glim_plan_gauss_newton(glim_plan* plan, const double* poses12, int32_t frame, int32_t iters,
                                   double* poses12_out, double* cost_out, int32_t* status_out);

/* Solve `count` systems H xi = -b by Cholesky in FP64 on the device (Sec. III-C: the
 * Gauss-Newton step of the quadratic factor).  System i uses the dim x dim block
 * H[i * stride_H + r * ldh + c] and b[i * stride_b + r]; xi_out is count x dim; status_out
 * (device, count int32, may be NULL) receives GLIM_OK or GLIM_ENOTPD per system.  All
 * pointers are device pointers.  1 <= dim <= 12.  Returns GLIM_ENOTPD if any system is not
 * positive definite (after synchronizing), else GLIM_OK. */
glim_status glim_gn_solve(glim_ctx* ctx, const double* H, int32_t ldh, int64_t stride_H,
                          const double* b, int64_t stride_b, int32_t dim, int64_t count,
                          double* xi_out, int32_t* status_out);

/* ---------------------------------------------------------------- small factor graphs */

/* One Gauss-Newton (lambda = 0) or Levenberg-Marquardt (lambda > 0) step of a graph of
 * matching-cost factors between nframes poses, on the device: the per-pair factors
 * (H: device, npairs x 144, over [xi_src; xi_tgt]; b: device, npairs x 12, as produced by the
 * linearization) are summed into the global system over all poses (pair_frames: host,
 * npairs x 2 (source, target) frame indices), frame `fixed_frame` (-1: none) is held fixed,
 * and (H_ff + lambda diag(H_ff)) xi_f = -b_f is solved by a dense FP64 Cholesky.  This is the
 * step of the all-to-all submap optimisation of local mapping (Sec. V-A).  xi_out: device,
 * nframes x 6 (zeros for the fixed frame); H_out (device, (6 nframes)^2) and b_out (device,
 * 6 nframes) receive the assembled, undamped global system (may be NULL).  1 <= nframes <= 128.
 * Returns GLIM_ENOTPD if the reduced system is not positive definite.  Synchronizes. */
glim_status glim_graph_step(glim_ctx* ctx, const int32_t* pair_frames, int32_t npairs,
                            int32_t nframes, const double* H, const double* b,
                            int32_t fixed_frame, double lambda, double* xi_out, double* H_out,
                            double* b_out);

#ifdef __cplusplus
}
#endif

#endif /* GLIM_LIN_H */
