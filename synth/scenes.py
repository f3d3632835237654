"""Seeded synthetic scenes and factor batches standing in for the paper's LiDAR data.

The paper evaluates on recorded datasets (Newer College, NTU VIRAL, and its own
flat-wall and cross-sensor recordings, Sec. VI); none is available here, so each
workload below is a synthetic scene of the same kind and scale:

* ``box_room``      -- one unary factor: 5k-point scan against a 20k-point scan of
                       a 10 x 8 x 3 m room (sigma 0.01 m, 1.0 m voxels).
* ``corridor``      -- odometry window: a 30k-point frame against 10 keyframes of
                       15k-40k points in a 60 m corridor with pillars every 5 m
                       (sigma 0.02 m, 0.5 m voxels), 10 binary factors.
* ``urban``         -- global step: 400 submaps of log-U[50k, 200k] points from a
                       street grid with buildings, poles and trunks (sigma 0.03 m),
                       4000 submap pairs (each submap to its 10 nearest),
                       0.5 / 1 / 2 m voxels.
* ``terrain``       -- precision / scale: a 1M-point scan against a 20M-point map of
                       sinusoidal terrain with box buildings (sigma 0.02 m, 0.25 m).

Points are drawn uniformly per unit surface area on axis-aligned rectangles,
vertical cylinders and a heightfield, restricted to a sensor range; occlusion is
not modelled.  Isotropic Gaussian noise is added in the world frame, then each
frame's points are expressed in that frame's own coordinates (mu = R^T (p - t)).
Poses are 3x4 row-major [R | t] in FP64.  This module only produces geometry and
poses; it computes no voxel, covariance or residual quantity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .rng import Stream


# ----------------------------------------------------------------------------- geometry helpers
def rot_axis_angle(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix about a unit axis (Rodrigues' formula)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def make_pose(R: np.ndarray, t) -> np.ndarray:
    T = np.zeros((3, 4), dtype=np.float64)
    T[:, :3] = R
    T[:, 3] = t
    return T


def to_local(p_world: np.ndarray, T: np.ndarray) -> np.ndarray:
    """World points into the frame of pose T (mu = R^T (p - t)), FP64."""
    return (p_world - T[:, 3]) @ T[:, :3]


def perturb_pose(T: np.ndarray, deg: float, dist: float, s: Stream) -> np.ndarray:
    """Rotate by ``deg`` about a random unit axis and shift by ``dist`` along a random direction."""
    axis = s.unit_vectors(1)[0]
    direction = s.unit_vectors(1)[0]
    R = T[:, :3] @ rot_axis_angle(axis, math.radians(deg))
    return make_pose(R, T[:, 3] + dist * direction)


# ----------------------------------------------------------------------------- primitives
@dataclass
class Rect:
    """Axis-aligned rectangle: coordinate ``axis`` fixed at ``value``; the other two axes span
    [lo[0], hi[0]] x [lo[1], hi[1]] (in increasing axis order)."""
    axis: int
    value: float
    lo: tuple
    hi: tuple

    def others(self):
        return [a for a in range(3) if a != self.axis]

    def clip(self, bmin, bmax):
        o = self.others()
        if not (bmin[self.axis] <= self.value <= bmax[self.axis]):
            return None
        lo = (max(self.lo[0], bmin[o[0]]), max(self.lo[1], bmin[o[1]]))
        hi = (min(self.hi[0], bmax[o[0]]), min(self.hi[1], bmax[o[1]]))
        if hi[0] <= lo[0] or hi[1] <= lo[1]:
            return None
        return Rect(self.axis, self.value, lo, hi)

    def area(self):
        return (self.hi[0] - self.lo[0]) * (self.hi[1] - self.lo[1])

    def sample(self, s: Stream, n: int) -> np.ndarray:
        o = self.others()
        p = np.empty((n, 3))
        p[:, self.axis] = self.value
        p[:, o[0]] = s.uniform(n, self.lo[0], self.hi[0])
        p[:, o[1]] = s.uniform(n, self.lo[1], self.hi[1])
        return p


@dataclass
class Cylinder:
    """Lateral surface of a vertical cylinder (axis along z)."""
    cx: float
    cy: float
    radius: float
    z0: float
    z1: float

    def clip(self, bmin, bmax):
        if (self.cx + self.radius < bmin[0] or self.cx - self.radius > bmax[0]
                or self.cy + self.radius < bmin[1] or self.cy - self.radius > bmax[1]
                or self.z1 < bmin[2] or self.z0 > bmax[2]):
            return None
        return self

    def area(self):
        return 2.0 * math.pi * self.radius * (self.z1 - self.z0)

    def sample(self, s: Stream, n: int) -> np.ndarray:
        th = s.uniform(n, 0.0, 2.0 * math.pi).astype(np.float32)  # FP32 trig: ~1e-8 m at these radii
        z = s.uniform(n, self.z0, self.z1)
        return np.stack([self.cx + self.radius * np.cos(th).astype(np.float64),
                         self.cy + self.radius * np.sin(th).astype(np.float64), z], 1)


def box_faces(x0, x1, y0, y1, z0, z1, roof=True, floor=False):
    f = [Rect(0, x0, (y0, z0), (y1, z1)), Rect(0, x1, (y0, z0), (y1, z1)),
         Rect(1, y0, (x0, z0), (x1, z1)), Rect(1, y1, (x0, z0), (x1, z1))]
    if roof:
        f.append(Rect(2, z1, (x0, y0), (x1, y1)))
    if floor:
        f.append(Rect(2, z0, (x0, y0), (x1, y1)))
    return f


def sample_scene(prims, n: int, s: Stream, center=None, radius=None) -> np.ndarray:
    """n points uniform per unit area over ``prims``; if ``center``/``radius`` are given,
    only surface within that sphere (sensor range) is sampled."""
    if center is not None:
        c = np.asarray(center, dtype=np.float64)
        bmin, bmax = c - radius, c + radius
        prims = [q for q in (p.clip(bmin, bmax) for p in prims) if q is not None]
    areas = np.array([p.area() for p in prims], dtype=np.float64)
    if len(prims) == 0 or areas.sum() <= 0:
        raise ValueError("no surface in range")
    cdf = np.cumsum(areas) / areas.sum()
    out = []
    have = 0
    while have < n:
        m = int((n - have) * 1.6) + 64
        which = np.minimum(np.searchsorted(cdf, s.uniform(m), side="right"), len(prims) - 1)
        pts = np.empty((m, 3))
        for i in np.unique(which):
            sel = which == i
            pts[sel] = prims[i].sample(s, int(sel.sum()))
        if center is not None:
            pts = pts[np.sum((pts - c) ** 2, axis=1) <= radius * radius]
        out.append(pts)
        have += len(pts)
    return np.concatenate(out)[:n]


def add_noise(p: np.ndarray, sigma: float, s: Stream) -> np.ndarray:
    if sigma == 0.0:
        return p
    return p + sigma * s.normal(p.size).reshape(p.shape)


# ----------------------------------------------------------------------------- workload container
@dataclass
class Workload:
    """A batch of factors: frames (points in their own coordinates), linearization poses,
    the (source, target) pair list and the voxel resolutions of the target maps."""
    name: str
    points: list                     # per frame: float32 (n, 3)
    poses: np.ndarray                # (nframes, 3, 4) FP64 linearization point
    poses_true: np.ndarray           # (nframes, 3, 4) FP64 ground truth
    pairs: np.ndarray                # (npairs, 2) int32: (source frame, target frame)
    resolutions: list                # voxel sizes, level 1..L
    weights: list = None             # optional per-frame float32 (n,) per-point weights
    meta: dict = field(default_factory=dict)

    @property
    def n_pair_points(self) -> int:
        return int(sum(len(self.points[s]) for s, _ in self.pairs))

    def targets(self):
        return sorted(set(int(t) for t in self.pairs[:, 1]))


# ----------------------------------------------------------------------------- configurations
def box_room(seed: int = 1, n_src: int = 5000, n_tgt: int = 20000, sigma: float = 0.01,
             perturb_deg: float = 5.0, perturb_m: float = 0.3) -> Workload:
    """One unary factor: a scan of a 10 x 8 x 3 m room against another scan of it.

    The target scan was taken near the room centre with a 17 degree yaw (so that no wall
    lies on a voxel face); the source scan 0.4 m away with a further 10 degree yaw.  The source's linearization pose is the true
    pose perturbed by ``perturb_deg`` / ``perturb_m``.
    """
    s = Stream(seed, "box_room")
    prims = box_faces(-5.0, 5.0, -4.0, 4.0, -1.5, 1.5, roof=True, floor=True)
    T_tgt = make_pose(rot_axis_angle([0, 0, 1], math.radians(17.0)), [0.23, -0.31, 0.07])
    T_src_true = make_pose(rot_axis_angle([0, 0, 1], math.radians(27.0)), [0.53, -0.56, 0.12])
    pw_t = add_noise(sample_scene(prims, n_tgt, s), sigma, s)
    pw_s = add_noise(sample_scene(prims, n_src, s), sigma, s)
    pts_t = to_local(pw_t, T_tgt).astype(np.float32)
    pts_s = to_local(pw_s, T_src_true).astype(np.float32)
    T_src_init = perturb_pose(T_src_true, perturb_deg, perturb_m, s)
    return Workload(
        name="box_room_unary_5k_vs_20k_1m",
        points=[pts_s, pts_t],
        poses=np.stack([T_src_init, T_tgt]),
        poses_true=np.stack([T_src_true, T_tgt]),
        pairs=np.array([[0, 1]], dtype=np.int32),
        resolutions=[1.0],
        meta=dict(sigma=sigma, seed=seed, perturb_deg=perturb_deg, perturb_m=perturb_m),
    )


def corridor_prims(length=60.0, half_w=1.5, height=3.0, pillar_every=5.0):
    prims = [Rect(2, 0.0, (0.0, -half_w), (length, half_w)),        # floor
             Rect(2, height, (0.0, -half_w), (length, half_w)),     # ceiling
             Rect(1, -half_w, (0.0, 0.0), (length, height)),        # right wall
             Rect(1, half_w, (0.0, 0.0), (length, height)),         # left wall
             Rect(0, 0.0, (-half_w, 0.0), (half_w, height)),        # end walls
             Rect(0, length, (-half_w, 0.0), (half_w, height))]
    k = 0
    x = pillar_every / 2.0
    while x < length:
        side = 1.0 if k % 2 == 0 else -1.0
        w, d = 0.4, 0.3
        yw = side * half_w
        yf = side * (half_w - d)
        prims.append(Rect(1, yf, (x - w / 2, 0.0), (x + w / 2, height)))      # pillar front
        ylo, yhi = min(yw, yf), max(yw, yf)
        prims.append(Rect(0, x - w / 2, (ylo, 0.0), (yhi, height)))           # pillar sides
        prims.append(Rect(0, x + w / 2, (ylo, 0.0), (yhi, height)))
        x += pillar_every
        k += 1
    return prims


def corridor(seed: int = 2, n_cur: int = 30000, kf_range=(15000, 40000), n_kf: int = 10,
             sigma: float = 0.02, sensor_range: float = 20.0, weights: bool = False) -> Workload:
    """Odometry window: the latest frame against ``n_kf`` keyframes in a corridor.

    Keyframe sensors sit every 4 m along the corridor axis; the latest frame is 3 m past
    the last keyframe.  Its linearization pose is the truth perturbed by 1 degree /
    0.1 m (an odometry prediction); keyframe poses are at the truth.  Frame 0 is the
    latest frame; pairs are (0, k) for every keyframe k.
    """
    s = Stream(seed, "corridor")
    prims = corridor_prims()
    xs = [6.0 + 4.0 * i for i in range(n_kf)] + [6.0 + 4.0 * (n_kf - 1) + 3.0]
    sizes = [int(v) for v in s.integers(n_kf, kf_range[0], kf_range[1] + 1)] + [n_cur]
    poses_true, pts = [], []
    for x, n in zip(xs, sizes):
        yaw = math.radians(float(s.uniform(1, -3.0, 3.0)[0]))
        T = make_pose(rot_axis_angle([0, 0, 1], yaw), [x, float(s.uniform(1, -0.3, 0.3)[0]), 1.5])
        pw = add_noise(sample_scene(prims, n, s, center=T[:, 3], radius=sensor_range), sigma, s)
        pts.append(to_local(pw, T).astype(np.float32))
        poses_true.append(T)
    # frame 0 = latest frame, frames 1..n_kf = keyframes
    order = [n_kf] + list(range(n_kf))
    pts = [pts[i] for i in order]
    poses_true = np.stack([poses_true[i] for i in order])
    poses = poses_true.copy()
    poses[0] = perturb_pose(poses_true[0], 1.0, 0.1, s)
    w = None
    if weights:
        w = [s.uniform(len(p), 0.5, 1.5).astype(np.float32) for p in pts]
    return Workload(
        name="corridor_odometry_30k_vs_10kf_0.5m",
        points=pts, poses=poses, poses_true=poses_true,
        pairs=np.array([[0, k] for k in range(1, n_kf + 1)], dtype=np.int32),
        resolutions=[0.5], weights=w,
        meta=dict(sigma=sigma, seed=seed, sizes=[len(p) for p in pts]),
    )


def urban_prims(seed: int, nx: int = 5, ny: int = 4, block: float = 60.0, street_half: float = 8.0):
    """Street grid: ground plane, building boxes in each block, poles along the streets and
    tree trunks on the pavements."""
    s = Stream(seed, "urban_layout")
    W, H = nx * block, ny * block
    prims = [Rect(2, 0.0, (-20.0, -20.0), (W + 20.0, H + 20.0))]
    for bx in range(nx):
        for by in range(ny):
            x0, y0 = bx * block + street_half, by * block + street_half
            x1, y1 = (bx + 1) * block - street_half, (by + 1) * block - street_half
            xm, ym = 0.5 * (x0 + x1) + s.uniform(1, -5, 5)[0], 0.5 * (y0 + y1) + s.uniform(1, -5, 5)[0]
            for (a0, a1) in ((x0, xm - 1.0), (xm + 1.0, x1)):
                for (b0, b1) in ((y0, ym - 1.0), (ym + 1.0, y1)):
                    h = float(s.uniform(1, 8.0, 30.0)[0])
                    prims += box_faces(a0, a1, b0, b1, 0.0, h, roof=False)
    # poles every 10 m along both sides of every street, trunks offset by 5 m
    for k in range(ny + 1):
        y = k * block
        for x in np.arange(0.0, W + 0.1, 10.0):
            for side in (-1.0, 1.0):
                prims.append(Cylinder(float(x), y + side * (street_half - 1.0), 0.12, 0.0, 6.0))
                prims.append(Cylinder(float(x) + 5.0, y + side * (street_half - 2.5), 0.3, 0.0, 4.0))
    for k in range(nx + 1):
        x = k * block
        for y in np.arange(0.0, H + 0.1, 10.0):
            for side in (-1.0, 1.0):
                prims.append(Cylinder(x + side * (street_half - 1.0), float(y), 0.12, 0.0, 6.0))
    return prims, W, H


def urban_trajectory(n: int, nx: int = 5, ny: int = 4, block: float = 60.0):
    """Serpentine drive along the horizontal streets, joined by the vertical ones; returns
    ``n`` equally spaced (x, y, yaw) samples."""
    W = nx * block
    way = []
    for k in range(ny + 1):
        y = k * block
        a, b = (0.0, W) if k % 2 == 0 else (W, 0.0)
        way.append((a, y))
        way.append((b, y))
    way = np.array(way)
    seg = np.diff(way, axis=0)
    seglen = np.linalg.norm(seg, axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seglen)])
    out = []
    for d in np.linspace(0.0, cum[-1], n):
        i = min(np.searchsorted(cum, d, side="right") - 1, len(seg) - 1)
        f = (d - cum[i]) / seglen[i]
        p = way[i] + f * seg[i]
        out.append((p[0], p[1], math.atan2(seg[i][1], seg[i][0])))
    return out


def urban(seed: int = 3, n_submaps: int = 400, n_range=(50000, 200000), neighbours: int = 10,
          sigma: float = 0.03, sensor_range: float = 35.0, resolutions=(0.5, 1.0, 2.0),
          point_scale: float = 1.0, keep: int = None) -> Workload:
    """Global step: submaps along a street trajectory, each paired with its nearest submaps.

    Submap sizes are log-uniform in ``n_range`` (times ``point_scale``); each submap is paired
    as source with its ``neighbours`` nearest submaps (by centre distance) as targets.  The
    linearization poses are the truth perturbed by 0.5 degree / 0.05 m, as in a global
    optimisation step that has not converged yet.  ``keep`` = N keeps only the first N submaps
    of the trajectory (same spacing, same sizes), paired among themselves: a smaller batch
    with the overlap statistics of the full one.
    """
    s = Stream(seed, "urban")
    prims, _, _ = urban_prims(seed)
    traj = urban_trajectory(n_submaps)
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    sizes = np.floor(np.exp(s.uniform(n_submaps, lo, hi)) * point_scale).astype(np.int64)
    if keep is not None:
        traj, sizes, n_submaps = traj[:keep], sizes[:keep], keep
    pts, poses_true = [], []
    for (x, y, yaw), n in zip(traj, sizes):
        T = make_pose(rot_axis_angle([0, 0, 1], yaw), [x, y, 1.8])
        pw = add_noise(sample_scene(prims, int(n), s, center=T[:, 3], radius=sensor_range), sigma, s)
        pts.append(to_local(pw, T).astype(np.float32))
        poses_true.append(T)
    poses_true = np.stack(poses_true)
    poses = np.stack([perturb_pose(T, 0.5, 0.05, s) for T in poses_true])
    c = poses_true[:, :, 3]
    d2 = np.sum((c[:, None, :] - c[None, :, :]) ** 2, axis=2)
    np.fill_diagonal(d2, np.inf)
    nb = np.argsort(d2, axis=1, kind="stable")[:, :neighbours]
    pairs = np.array([[i, int(j)] for i in range(n_submaps) for j in nb[i]], dtype=np.int32)
    return Workload(
        name=f"urban_global_{n_submaps}submaps_{len(pairs)}pairs_0.5-1-2m",
        points=pts, poses=poses, poses_true=poses_true, pairs=pairs,
        resolutions=list(resolutions),
        meta=dict(sigma=sigma, seed=seed, sizes=[int(v) for v in sizes]),
    )


_K1, _K2, _K3, _K4 = 2 * np.pi / 140.0, 2 * np.pi / 110.0, 2 * np.pi / 60.0, 2 * np.pi / 25.0


def _phase(a):
    """Phase reduced to [0, 2 pi) in FP64, then rounded to FP32 for a fast FP32 sine/cosine."""
    return np.mod(a, 2 * np.pi).astype(np.float32)


def terrain_height_and_slope(x, y):
    """Height of the sum-of-sinusoids terrain (amplitudes 0.4-3 m, wavelengths 25-140 m) and
    the area factor sqrt(1 + |grad z|^2), from one set of sines and cosines.  The trigonometry
    runs in FP32 on phases reduced in FP64 (the points are stored in FP32; the surface error
    is ~1e-7 m)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    a1 = _phase(_K1 * x + 0.3)
    b1 = _phase(_K2 * y)
    a2 = _phase(_K3 * (0.6 * x + 0.8 * y) + 1.1)
    a3 = _phase(_K4 * (0.9 * x - 0.4 * y))
    s1, c1, sb, cb = np.sin(a1), np.cos(a1), np.sin(b1), np.cos(b1)
    s2, c2 = np.sin(a2), np.cos(a2)
    s3, c3 = np.sin(a3), np.cos(a3)
    z = 3.0 * s1 * cb + 1.2 * s2 + 0.4 * c3
    gx = np.float32(3.0 * _K1) * c1 * cb + np.float32(1.2 * _K3 * 0.6) * c2 - np.float32(0.4 * _K4 * 0.9) * s3
    gy = np.float32(-3.0 * _K2) * s1 * sb + np.float32(1.2 * _K3 * 0.8) * c2 + np.float32(0.4 * _K4 * 0.4) * s3
    return z, np.sqrt(1.0 + gx * gx + gy * gy)


def terrain_height(x, y):
    return terrain_height_and_slope(x, y)[0]


def _terrain_points(s: Stream, n: int, cx: float, cy: float, radius: float, half: float,
                    buildings) -> np.ndarray:
    """Terrain surface (area-uniform by rejection on sqrt(1 + |grad|^2)) plus building walls
    and roofs, inside a disc of ``radius`` around (cx, cy) clipped to the square of
    half-width ``half``."""
    walls = []
    for (x0, x1, y0, y1, h) in buildings:
        z0 = float(terrain_height(np.array([0.5 * (x0 + x1)]), np.array([0.5 * (y0 + y1)]))[0]) - 1.0
        walls += box_faces(x0, x1, y0, y1, z0, z0 + h, roof=True)
    lo_x, hi_x = max(cx - radius, -half), min(cx + radius, half)
    lo_y, hi_y = max(cy - radius, -half), min(cy + radius, half)
    bmin = np.array([lo_x, lo_y, -1e9])
    bmax = np.array([hi_x, hi_y, 1e9])
    walls = [q for q in (w.clip(bmin, bmax) for w in walls) if q is not None]
    wall_area = sum(w.area() for w in walls)
    ground_area = math.pi * radius * radius if radius < half else (hi_x - lo_x) * (hi_y - lo_y)
    ground_area *= 1.05  # mean slope factor of this terrain
    frac_wall = wall_area / (wall_area + ground_area)
    n_wall = int(round(n * frac_wall))
    n_ground = n - n_wall
    out = []
    have = 0
    gmax = 1.6
    while have < n_ground:
        m = int((n_ground - have) * 1.7) + 64
        x = s.uniform(m, lo_x, hi_x)
        y = s.uniform(m, lo_y, hi_y)
        z, area = terrain_height_and_slope(x, y)
        keep = s.uniform(m) * gmax <= area
        keep &= (x - cx) ** 2 + (y - cy) ** 2 <= radius * radius
        out.append(np.stack([x[keep], y[keep], z[keep].astype(np.float64)], 1))
        have += int(keep.sum())
    g = np.concatenate(out)[:n_ground]
    if n_wall > 0:
        w = sample_scene(walls, n_wall, s)
        g = np.concatenate([g, w])
    return g


def terrain(seed: int = 5, n_src: int = 1_000_000, n_map: int = 20_000_000, sigma: float = 0.02,
            half: float = 250.0, src_radius: float = 60.0, resolution: float = 0.25) -> Workload:
    """Precision / scale stress: one scan against a large terrain map with buildings."""
    s = Stream(seed, "terrain")
    nb = 60
    bx = s.uniform(nb, -half + 20, half - 20)
    by = s.uniform(nb, -half + 20, half - 20)
    bw = s.uniform(nb, 8.0, 25.0)
    bd = s.uniform(nb, 8.0, 25.0)
    bh = s.uniform(nb, 6.0, 20.0)
    buildings = [(float(bx[i]), float(bx[i] + bw[i]), float(by[i]), float(by[i] + bd[i]), float(bh[i]))
                 for i in range(nb)]
    T_map = make_pose(np.eye(3), [0.0, 0.0, 0.0])
    pm = add_noise(_terrain_points(s, n_map, 0.0, 0.0, 2.0 * half, half, buildings), sigma, s)
    sx, sy = 40.0, -30.0
    sz = float(terrain_height(np.array([sx]), np.array([sy]))[0]) + 2.0
    T_src = make_pose(rot_axis_angle([0, 0, 1], math.radians(35.0)), [sx, sy, sz])
    ps = add_noise(_terrain_points(s, n_src, sx, sy, src_radius, half, buildings), sigma, s)
    pts_map = to_local(pm, T_map).astype(np.float32)
    pts_src = to_local(ps, T_src).astype(np.float32)
    T_init = perturb_pose(T_src, 1.0, 0.1, s)
    return Workload(
        name=f"terrain_{n_src // 1000}k_vs_{n_map // 1000}k_{resolution}m",
        points=[pts_src, pts_map], poses=np.stack([T_init, T_map]),
        poses_true=np.stack([T_src, T_map]),
        pairs=np.array([[0, 1]], dtype=np.int32), resolutions=[resolution],
        meta=dict(sigma=sigma, seed=seed),
    )
