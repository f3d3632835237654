"""Python handle on the FP64 CPU oracle (``glim_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.  It marshals numpy
arrays into the oracle's C functions and back; all arithmetic is in the C++ file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glim_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libglim_oracle.so")

ORC_OK, ORC_EINVAL, ORC_ERANGE, ORC_ENOTPD = 0, -1, -5, -6


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FP contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Frame(C.Structure):
    _fields_ = [("pts4", C.c_void_p), ("cov6", C.c_void_p), ("normal3", C.c_void_p), ("n", C.c_int64)]


class _Pair(C.Structure):
    _fields_ = [("src", C.c_int32), ("tgt", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("validate_surface", C.c_int32), ("omega_identity", C.c_int32),
                ("omega_grad_full", C.c_int32), ("nthreads", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_vmap_build.restype = C.c_void_p
        _lib.orc_vmap_build.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int,
                                        C.POINTER(C.c_int)]
        _lib.orc_vmap_size.restype = C.c_int64
        _lib.orc_vmap_size.argtypes = [C.c_void_p, C.c_int]
        _lib.orc_vmap_export.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 4
        _lib.orc_vmap_free.argtypes = [C.c_void_p]
        _lib.orc_estimate_covariances.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_double,
                                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        _lib.orc_covariances_at.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_double,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        _lib.orc_linearize.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                       C.c_void_p] + [C.c_void_p] * 8
        _lib.orc_energy.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_gradient.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_gn_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        _lib.orc_graph_step.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                        C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_overlap.restype = C.c_double
        _lib.orc_overlap.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def as_pts4(pts, weights=None) -> np.ndarray:
    """(n, 3) or (n, 4) -> contiguous float32 (n, 4) with the weight in the fourth lane."""
    pts = np.asarray(pts)
    out = np.ones((len(pts), 4), dtype=np.float32)
    out[:, :3] = pts[:, :3]
    if pts.shape[1] == 4:
        out[:, 3] = pts[:, 3]
    if weights is not None:
        out[:, 3] = weights
    return out


def estimate_covariances(pts, k: int = 10, reg_mode: int = 1, eps: float = 1e-3, nthreads: int = 0):
    """Brute-force kNN covariances; returns (cov6 f64, normals f64, knn int32, near_tie bool)."""
    p4 = as_pts4(pts)
    n = len(p4)
    cov = np.zeros((n, 6))
    nrm = np.zeros((n, 3))
    knn = np.zeros((n, k), dtype=np.int32)
    tie = np.zeros(n, dtype=np.uint8)
    st = lib().orc_estimate_covariances(_ptr(p4), n, k, reg_mode, eps, _ptr(cov), _ptr(nrm), _ptr(knn),
                                        _ptr(tie), nthreads or os.cpu_count())
    if st != ORC_OK:
        raise ValueError(f"orc_estimate_covariances failed: {st}")
    return cov, nrm, knn, tie.astype(bool)


def covariances_at(pts, queries, k: int = 10, reg_mode: int = 1, eps: float = 1e-3, nthreads: int = 0):
    """Brute-force kNN covariances of the listed query points only (each scans the whole frame);
    returns (cov6 f64 (nq, 6), normals (nq, 3), knn int32 (nq, k), near_tie bool (nq,))."""
    p4 = as_pts4(pts)
    qi = np.ascontiguousarray(queries, dtype=np.int64)
    nq = len(qi)
    cov = np.zeros((nq, 6))
    nrm = np.zeros((nq, 3))
    knn = np.zeros((nq, k), dtype=np.int32)
    tie = np.zeros(nq, dtype=np.uint8)
    st = lib().orc_covariances_at(_ptr(p4), len(p4), _ptr(qi), nq, k, reg_mode, eps, _ptr(cov), _ptr(nrm), _ptr(knn),
                                  _ptr(tie), nthreads or os.cpu_count())
    if st != ORC_OK:
        raise ValueError(f"orc_covariances_at failed: {st}")
    return cov, nrm, knn, tie.astype(bool)


class VMap:
    """std::map voxelmap of one frame at one or more resolutions."""

    def __init__(self, pts4, cov6, resolutions):
        self.pts4 = np.ascontiguousarray(pts4, dtype=np.float32)
        self.cov6 = np.ascontiguousarray(cov6, dtype=np.float32)
        self.resolutions = np.ascontiguousarray(resolutions, dtype=np.float64)
        st = C.c_int(0)
        self.h = lib().orc_vmap_build(_ptr(self.pts4), _ptr(self.cov6), len(self.pts4),
                                      _ptr(self.resolutions), len(self.resolutions), C.byref(st))
        self.status = st.value
        if not self.h:
            raise ValueError(f"orc_vmap_build failed: {st.value}")

    @property
    def levels(self):
        return len(self.resolutions)

    def size(self, level):
        return int(lib().orc_vmap_size(self.h, level))

    def export(self, level):
        m = self.size(level)
        keys = np.zeros((m, 3), dtype=np.int32)
        mean = np.zeros((m, 3))
        cov = np.zeros((m, 6))
        cnt = np.zeros(m, dtype=np.int64)
        lib().orc_vmap_export(self.h, level, _ptr(keys), _ptr(mean), _ptr(cov), _ptr(cnt))
        return dict(keys=keys, mean=mean, cov=cov, count=cnt)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_vmap_free(self.h)
            self.h = None


@dataclass
class Frame:
    pts4: np.ndarray
    cov6: np.ndarray
    normal3: np.ndarray = None


def _frames(frames):
    keep = []
    arr = (_Frame * len(frames))()
    for i, f in enumerate(frames):
        p = np.ascontiguousarray(f.pts4, dtype=np.float32)
        c = np.ascontiguousarray(f.cov6, dtype=np.float32)
        nrm = None if f.normal3 is None else np.ascontiguousarray(f.normal3, dtype=np.float32)
        keep += [p, c, nrm]
        arr[i] = _Frame(_ptr(p).value, _ptr(c).value, None if nrm is None else _ptr(nrm).value, len(p))
    return arr, keep


def _pairs(pairs):
    pairs = np.asarray(pairs, dtype=np.int32)
    arr = (_Pair * len(pairs))()
    for i, (s, t) in enumerate(pairs):
        arr[i] = _Pair(int(s), int(t))
    return arr


def _vmaps(vmaps):
    arr = (C.c_void_p * len(vmaps))()
    for i, v in enumerate(vmaps):
        arr[i] = None if v is None else v.h
    return arr


def _opts(validate=False, omega_identity=False, omega_grad_full=True, nthreads=1):
    return _Opts(int(validate), int(omega_identity), int(omega_grad_full), int(nthreads))


def _id_count(frames, vmaps, pairs):
    return sum(len(frames[s].pts4) * vmaps[t].levels for s, t in np.asarray(pairs))


def linearize(frames, vmaps, pairs, poses, validate=False, omega_identity=False, ids_in=None,
              want_ids=False, want_comp=False, nthreads=1):
    """e, H (12x12), b (12) per pair; ids (canonical voxel id per source point and level)."""
    pairs = np.asarray(pairs, dtype=np.int32)
    P = len(pairs)
    fr, keep = _frames(frames)
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1, 12)
    e = np.zeros(P)
    H = np.zeros((P, 12, 12))
    b = np.zeros((P, 12))
    inl = np.zeros(P, dtype=np.int64)
    skp = np.zeros(P, dtype=np.int64)
    nid = _id_count(frames, vmaps, pairs)
    ids = np.zeros(nid, dtype=np.int32) if want_ids else None
    if ids_in is not None:
        ids_in = np.ascontiguousarray(ids_in, dtype=np.int32)
        assert ids_in.size == nid
    comp = np.zeros((P, 158)) if want_comp else None
    opts = _opts(validate, omega_identity, True, nthreads)
    st = lib().orc_linearize(fr, len(frames), _vmaps(vmaps), _pairs(pairs), P, _ptr(poses), C.byref(opts),
                             _ptr(e), _ptr(H), _ptr(b), _ptr(inl), _ptr(skp), _ptr(ids), _ptr(ids_in),
                             _ptr(comp))
    if st != ORC_OK:
        raise ValueError(f"orc_linearize failed: {st}")
    out = dict(e=e, H=H, b=b, inliers=inl, skipped=skp)
    if want_ids:
        out["ids"] = ids
    if want_comp:
        out["comp_e"] = comp[:, 0]
        out["comp_H"] = comp[:, 1:145].reshape(P, 12, 12)
        out["comp_b"] = comp[:, 145:157]
        out["b_scale"] = comp[:, 157]
    return out


def energy(frames, vmaps, pairs, poses, ids_in, omega_poses=None, omega_identity=False):
    pairs = np.asarray(pairs, dtype=np.int32)
    fr, keep = _frames(frames)
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1, 12)
    op = None if omega_poses is None else np.ascontiguousarray(omega_poses, dtype=np.float64).reshape(-1, 12)
    ids_in = np.ascontiguousarray(ids_in, dtype=np.int32)
    e = np.zeros(len(pairs))
    opts = _opts(False, omega_identity)
    st = lib().orc_energy(fr, len(frames), _vmaps(vmaps), _pairs(pairs), len(pairs), _ptr(poses), _ptr(op),
                          _ptr(ids_in), C.byref(opts), _ptr(e))
    if st != ORC_OK:
        raise ValueError(f"orc_energy failed: {st}")
    return e


def gradient(frames, vmaps, pairs, poses, omega_grad_full=True, validate=False):
    """dE/dxi (nframes, 6), dE/dmu (list per frame of (n, 3)), dE/dw (list per frame of (n,))."""
    pairs = np.asarray(pairs, dtype=np.int32)
    fr, keep = _frames(frames)
    nf = len(frames)
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1, 12)
    ntot = sum(len(f.pts4) for f in frames)
    dxi = np.zeros((nf, 6))
    dmu = np.zeros((ntot, 3))
    dw = np.zeros(ntot)
    opts = _opts(validate, False, omega_grad_full)
    st = lib().orc_gradient(fr, nf, _vmaps(vmaps), _pairs(pairs), len(pairs), _ptr(poses), C.byref(opts),
                            _ptr(dxi), _ptr(dmu), _ptr(dw))
    if st != ORC_OK:
        raise ValueError(f"orc_gradient failed: {st}")
    offs = np.cumsum([0] + [len(f.pts4) for f in frames])
    return dxi, [dmu[offs[i]:offs[i + 1]] for i in range(nf)], [dw[offs[i]:offs[i + 1]] for i in range(nf)]


def gn_solve(H, b):
    H = np.ascontiguousarray(H, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    xi = np.zeros(len(b))
    st = lib().orc_gn_solve(_ptr(H), _ptr(b), len(b), _ptr(xi))
    if st != ORC_OK:
        raise np.linalg.LinAlgError(f"orc_gn_solve: {st}")
    return xi


def graph_step(pair_frames, nframes, H, b, fixed=0, lam=0.0):
    """Assembled global system and damped step of a factor graph: returns (xi (nframes, 6),
    H_glob (6n, 6n), b_glob (6n)); raises LinAlgError if the reduced system is not PD."""
    pf = np.ascontiguousarray(np.asarray(pair_frames, dtype=np.int32).reshape(-1, 2))
    H = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1, 144))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1, 12))
    xi = np.zeros((nframes, 6))
    Hg = np.zeros((6 * nframes, 6 * nframes))
    bg = np.zeros(6 * nframes)
    st = lib().orc_graph_step(_ptr(pf), len(pf), int(nframes), _ptr(H), _ptr(b), int(fixed), float(lam), _ptr(xi),
                              _ptr(Hg), _ptr(bg))
    if st == ORC_ENOTPD:
        raise np.linalg.LinAlgError("orc_graph_step: reduced system not positive definite")
    if st != ORC_OK:
        raise ValueError(f"orc_graph_step failed: {st}")
    return xi, Hg, bg


def overlap(frame: Frame, vmap: VMap, pose_s, pose_t, level=0):
    fr, keep = _frames([frame])
    ps = np.ascontiguousarray(pose_s, dtype=np.float64)
    pt = np.ascontiguousarray(pose_t, dtype=np.float64)
    return float(lib().orc_overlap(fr, vmap.h, _ptr(ps), _ptr(pt), level))


# ------------------------------------------------------------------ SE(3) helpers (test drivers)
def hat(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def so3_exp(w):
    th = np.linalg.norm(w)
    K = hat(w)
    if th < 1e-12:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K


def se3_exp(xi):
    """Exp of xi = [omega; v] as a 3x4 [R | t] (left Jacobian on the translation)."""
    w, v = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(w)
    K = hat(w)
    if th < 1e-12:
        V = np.eye(3) + 0.5 * K + K @ K / 6.0
    else:
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * K @ K
    T = np.zeros((3, 4))
    T[:, :3] = so3_exp(w)
    T[:, 3] = V @ v
    return T


def compose(A, B):
    T = np.zeros((3, 4))
    T[:, :3] = A[:, :3] @ B[:, :3]
    T[:, 3] = A[:, :3] @ B[:, 3] + A[:, 3]
    return T


def inverse(A):
    T = np.zeros((3, 4))
    T[:, :3] = A[:, :3].T
    T[:, 3] = -A[:, :3].T @ A[:, 3]
    return T


def retract(T, xi):
    """Right perturbation T <- T Exp(xi)."""
    return compose(T, se3_exp(xi))
