"""Python face of the linearization library: thin wrappers over the C ABI that take
PyTorch CUDA tensors (device memory) and numpy arrays (host poses).

Every computation happens in the CUDA library; this module only checks shapes and
dtypes, passes pointers and reports errors.  There is no CPU path.
"""
from __future__ import annotations

import atexit
import ctypes as C
import weakref

import numpy as np
import torch

from . import _abi

ACC_FP32, ACC_KAHAN, ACC_FP64 = _abi.ACC_FP32, _abi.ACC_KAHAN, _abi.ACC_FP64


class GlimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_abi.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _dev(t, dtype, shape1=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape1 is not None and (t.dim() != 2 or t.shape[1] != shape1):
        raise ValueError(f"{name} must have shape (n, {shape1}), got {tuple(t.shape)}")
    return t


def _poses(poses, nframes=None):
    P = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 12))
    if nframes is not None and len(P) != nframes:
        raise ValueError(f"expected {nframes} poses, got {len(P)}")
    return P


# Library objects still open at interpreter exit are released by an exit hook, plans and
# maps before the contexts they use: the interpreter's own teardown destroys objects in no
# fixed order, and it may do so after CUDA has started to shut down.
_LIVE = {"plans": weakref.WeakSet(), "maps": weakref.WeakSet(), "contexts": weakref.WeakSet()}


def _release_all():
    for kind, method in (("plans", "close"), ("maps", "free"), ("contexts", "close")):
        for obj in list(_LIVE[kind]):
            try:
                getattr(obj, method)()
            except Exception:
                pass


atexit.register(_release_all)


class Context:
    """A library context on one CUDA device, enqueuing on a torch stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream = None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.lib = _abi.load()
        self.device = device
        with torch.cuda.device(device):
            # the library works on its own stream; call() orders it against torch's current stream
            self.stream = stream or torch.cuda.Stream(device)
        h = C.c_void_p()
        st = self.lib.glim_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise GlimError(st, "glim_create failed")
        self.h = h
        _LIVE["contexts"].add(self)

    def check(self, st, what):
        if st != 0:
            raise GlimError(st, f"{what}: {self.lib.glim_last_error(self.h).decode()}")

    def call(self, what, fn, *args, ok=(0,)):
        """Run a library call on the context stream, after the work already queued on torch's
        current stream, and make torch's current stream wait for it."""
        cur = torch.cuda.current_stream(self.device)
        same = cur.cuda_stream == self.stream.cuda_stream
        if not same:
            self.stream.wait_stream(cur)
        st = fn(*args)
        if not same:
            cur.wait_stream(self.stream)
        if st not in ok:
            self.check(st, what)
        return st

    @property
    def num_sms(self):
        return int(self.lib.glim_num_sms(self.h))

    @property
    def kernel_launches(self):
        return int(self.lib.glim_kernel_launches(self.h))

    def fp32_fma_peak(self, iters=4096):
        """Measured FP32 FMA throughput of the device in TFLOP/s (FMA-chain kernel)."""
        out = C.c_double()
        self.call("fp32_fma_peak", self.lib.glim_fp32_fma_peak, self.h, int(iters), C.byref(out))
        return out.value

    def fp64_fma_peak(self, iters=128):
        """Measured FP64 FMA throughput of the device in TFLOP/s (the same FMA-chain kernel)."""
        out = C.c_double()
        self.call("fp64_fma_peak", self.lib.glim_fp64_fma_peak, self.h, int(iters), C.byref(out))
        return out.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.glim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_fail_allocation(n: int) -> None:
    """Testing hook: the library's allocation n allocations from now (0 = the next one) fails
    once as if the device were out of memory; n < 0 disables it.  Process-wide."""
    _abi.load().glim_debug_fail_allocation(int(n))


def to_pts4(points, weights=None, device="cuda"):
    """(n, 3) points (+ optional (n,) weights) -> contiguous float32 (n, 4) CUDA tensor."""
    p = torch.as_tensor(np.asarray(points, dtype=np.float32)) if not isinstance(points, torch.Tensor) else points
    out = torch.ones((p.shape[0], 4), dtype=torch.float32, device=device)
    out[:, :3] = p[:, :3].to(device=device, dtype=torch.float32)
    if weights is not None:
        w = torch.as_tensor(np.asarray(weights, dtype=np.float32)) if not isinstance(weights, torch.Tensor) else weights
        out[:, 3] = w.to(device=device, dtype=torch.float32)
    return out


def estimate_covariances(ctx: Context, pts4: torch.Tensor, k: int = 10, reg_mode: int = 1, eps: float = 1e-3,
                         normals: bool = True):
    """kNN covariances (n, 6) and normals (n, 3) of one frame."""
    _dev(pts4, torch.float32, 4, "pts4")
    n = pts4.shape[0]
    cov = torch.empty((n, 6), dtype=torch.float32, device=pts4.device)
    nrm = torch.empty((n, 3), dtype=torch.float32, device=pts4.device) if normals else None
    ctx.call("estimate_covariances", ctx.lib.glim_estimate_covariances, ctx.h, _ptr(pts4), n, k, reg_mode, eps, _ptr(cov), _ptr(nrm))
    return cov, nrm


def estimate_covariances_knn(ctx: Context, pts4: torch.Tensor, k: int = 10, reg_mode: int = 1, eps: float = 1e-3):
    """kNN covariances (n, 6), normals (n, 3) and the neighbour indices (n, k) int32, nearest
    first, of one frame."""
    _dev(pts4, torch.float32, 4, "pts4")
    n = pts4.shape[0]
    cov = torch.empty((n, 6), dtype=torch.float32, device=pts4.device)
    nrm = torch.empty((n, 3), dtype=torch.float32, device=pts4.device)
    knn = torch.empty((n, k), dtype=torch.int32, device=pts4.device)
    ctx.call("estimate_covariances_knn", ctx.lib.glim_estimate_covariances_knn, ctx.h, _ptr(pts4), n, k, reg_mode, eps,
             _ptr(cov), _ptr(nrm), _ptr(knn))
    return cov, nrm, knn


def spatial_order(ctx: Context, pts4: torch.Tensor, cell: float = 0.5) -> torch.Tensor:
    """Permutation (int64 CUDA tensor) ordering the points along a Z-order curve of cells."""
    _dev(pts4, torch.float32, 4, "pts4")
    perm = torch.empty(pts4.shape[0], dtype=torch.int32, device=pts4.device)
    ctx.call("spatial_order", ctx.lib.glim_spatial_order, ctx.h, _ptr(pts4), pts4.shape[0], float(cell), _ptr(perm))
    return perm.long()


# Number of VoxelMap.free calls so far: a plan re-checks its target maps before a launch
# only when a map was freed since its last check (a freed map's tables are gone).
_FREED_MAPS = 0


class VoxelMap:
    """Multi-resolution voxelmap of one frame (library-owned device tables)."""

    def __init__(self, ctx: Context, pts4: torch.Tensor, cov6: torch.Tensor, resolutions, layout: str = "auto"):
        """layout: "auto" (dense index grid when its box is small enough, else hash table),
        "dense" or "hash"."""
        _dev(pts4, torch.float32, 4, "pts4")
        _dev(cov6, torch.float32, 6, "cov6")
        if pts4.shape[0] != cov6.shape[0]:
            raise ValueError("pts4 and cov6 differ in length")
        self.ctx = ctx
        self.resolutions = [float(r) for r in resolutions]
        res = np.ascontiguousarray(self.resolutions, dtype=np.float64)
        h = C.c_void_p()
        lay = {"auto": 0, "dense": 1, "hash": 2}[layout]
        ctx.call("build_voxelmap", ctx.lib.glim_build_voxelmap_ex, ctx.h, _ptr(pts4), _ptr(cov6), pts4.shape[0],
                 _ptr(res), len(res), lay, C.byref(h))
        self.h = h
        _LIVE["maps"].add(self)

    @property
    def levels(self):
        return len(self.resolutions)

    def info(self, level):
        n, cap, mp = C.c_int64(), C.c_int64(), C.c_int32()
        self.ctx.call("vmap_info", self.ctx.lib.glim_vmap_info, self.h, level, C.byref(n), C.byref(cap), C.byref(mp))
        return dict(n_voxels=n.value, capacity=cap.value, max_probe=mp.value)

    def is_dense(self, level):
        return bool(self.ctx.lib.glim_vmap_is_dense(self.h, level))

    def insert(self, pts4: torch.Tensor, cov6: torch.Tensor, layout: str = "auto"):
        """Add map-frame points to every level (running FP64 sums per voxel, ids re-ranked);
        the result equals a build from all points inserted so far.  Plans created on this
        map before the call must be recreated."""
        _dev(pts4, torch.float32, 4, "pts4")
        _dev(cov6, torch.float32, 6, "cov6")
        if pts4.shape[0] != cov6.shape[0]:
            raise ValueError("pts4 and cov6 differ in length")
        lay = {"auto": 0, "dense": 1, "hash": 2}[layout]
        self.ctx.call("vmap_insert", self.ctx.lib.glim_vmap_insert, self.ctx.h, self.h, _ptr(pts4), _ptr(cov6),
                      pts4.shape[0], lay)
        return self

    def export(self, level):
        m = self.info(level)["n_voxels"]
        dev = torch.device("cuda", self.ctx.device)
        keys = torch.empty((m, 3), dtype=torch.int32, device=dev)
        mean = torch.empty((m, 3), dtype=torch.float32, device=dev)
        cov = torch.empty((m, 6), dtype=torch.float32, device=dev)
        cnt = torch.empty((m,), dtype=torch.int32, device=dev)
        self.ctx.call("vmap_export", self.ctx.lib.glim_vmap_export, self.ctx.h, self.h, level, _ptr(keys), _ptr(mean), _ptr(cov),
                                                     _ptr(cnt))
        return dict(keys=keys, mean=mean, cov=cov, count=cnt)

    def free(self):
        if getattr(self, "h", None):
            global _FREED_MAPS
            _FREED_MAPS += 1
            self.ctx.lib.glim_vmap_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class FrameData:
    """Device arrays of one frame: points (n, 4) with weights in the fourth lane, covariances
    (n, 6) and optional normals (n, 3)."""

    def __init__(self, pts4, cov6, normal3=None):
        self.pts4 = _dev(pts4, torch.float32, 4, "pts4")
        self.cov6 = _dev(cov6, torch.float32, 6, "cov6")
        self.normal3 = None if normal3 is None else _dev(normal3, torch.float32, 3, "normal3")

    @property
    def n(self):
        return self.pts4.shape[0]

    def c(self):
        return _abi.Frame(self.pts4.data_ptr(), self.cov6.data_ptr(),
                          None if self.normal3 is None else self.normal3.data_ptr(), self.n)


_FRAME_DTYPE = np.dtype([("pts4", "<u8"), ("cov6", "<u8"), ("normal3", "<u8"), ("n", "<i8")])  # glim_frame


def _frames(frames):
    """A packed glim_frame array (one numpy record per frame) and a pointer to it."""
    arr = np.zeros(max(len(frames), 1), dtype=_FRAME_DTYPE)
    if frames:
        arr[:len(frames)] = [(f.pts4.data_ptr(), f.cov6.data_ptr(), 0 if f.normal3 is None else f.normal3.data_ptr(),
                              f.n) for f in frames]
    ptr = arr.ctypes.data_as(C.POINTER(_abi.Frame))
    ptr._keep = arr
    return ptr


_PAIR_DTYPE = np.dtype([("src_frame", "<i4"), ("tgt_frame", "<i4"), ("tgt", "<u8")])  # glim_pair


def _pairs(pairs, vmaps):
    """pairs: (P, 2) (source, target); vmaps: per frame VoxelMap or None (target frames).
    Returns a pointer to a packed glim_pair array (built with numpy, not per pair) and P."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    P = len(pairs)
    handles = np.array([0 if vm is None else (vm.h.value or 0) for vm in vmaps], dtype=np.uint64)
    arr = np.zeros(max(P, 1), dtype=_PAIR_DTYPE)
    if P:
        t = pairs[:, 1]
        if ((t < 0) | (t >= len(vmaps))).any():
            raise ValueError("pair target outside the frame list")
        h = handles[t]
        missing = np.flatnonzero(h == 0)
        if len(missing):
            i = int(missing[0])
            raise ValueError(f"pair {i}: target frame {t[i]} has no voxelmap")
        arr["src_frame"][:P] = pairs[:, 0]
        arr["tgt_frame"][:P] = t
        arr["tgt"][:P] = h
    ptr = arr.ctypes.data_as(C.POINTER(_abi.Pair))
    ptr._keep = arr  # the array lives as long as the pointer
    return ptr, P


KERNELS = {"auto": 0, "general": 1, "dense": 2, "hash": 3}


def _opts(validate_surface=False, accum_mode=ACC_FP64, block=0, pts_per_thread=0, blocks_per_sm=0,
          persistent=0, kernel="auto"):
    """kernel: "auto" (the per-lane dense-grid or hash kernel when every target level has
    that layout, else the general kernel), "general", "dense" or "hash"."""
    o = _abi.LinOpts()
    o.kernel = KERNELS[kernel]
    o.validate_surface = int(validate_surface)
    o.accum_mode = int(accum_mode)
    o.block = int(block)
    o.pts_per_thread = int(pts_per_thread)
    o.blocks_per_sm = int(blocks_per_sm)
    o.persistent = int(persistent)
    return o


def _outputs(npairs, device):
    if device == "host":
        return (np.zeros(npairs), np.zeros((npairs, 12, 12)), np.zeros((npairs, 12)),
                np.zeros(npairs, dtype=np.int64))
    return (torch.empty(npairs, dtype=torch.float64, device=device),
            torch.empty((npairs, 12, 12), dtype=torch.float64, device=device),
            torch.empty((npairs, 12), dtype=torch.float64, device=device),
            torch.empty(npairs, dtype=torch.int64, device=device))


def linearize(ctx: Context, frames, vmaps, pairs, poses, out="host", plain=False, **opts):
    """e (P,), H (P, 12, 12), b (P, 12), inliers (P,) of every (source, target) pair at poses
    (nframes, 3, 4).  out = "host" (numpy) or a torch device (CUDA tensors)."""
    fr = _frames(frames)
    pr, P = _pairs(pairs, vmaps)
    Pz = _poses(poses, len(frames))
    o = _opts(**opts)
    e, H, b, inl = _outputs(P, out)
    fn = ctx.lib.glim_linearize_factors_plain if plain else ctx.lib.glim_linearize_factors
    ctx.call("linearize_factors_plain" if plain else "linearize_factors", fn, ctx.h, fr, len(frames), pr, P,
             _ptr(Pz), C.byref(o), _ptr(e), _ptr(H), _ptr(b), _ptr(inl))
    return e, H, b, inl


class Plan:
    """A fixed batch of factors: work list, serialized I/O blocks and CUDA graphs."""

    def __init__(self, ctx: Context, frames, vmaps, pairs, **opts):
        self.ctx = ctx
        self.frames = list(frames)
        self.vmaps = list(vmaps)
        fr = _frames(self.frames)
        pr, P = _pairs(pairs, self.vmaps)
        self.npairs = P
        self.nframes = len(self.frames)
        self._pairs_arr = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
        o = _opts(**opts)
        h = C.c_void_p()
        ctx.call("plan_create", ctx.lib.glim_plan_create, ctx.h, fr, self.nframes, pr, P, C.byref(o), C.byref(h))
        self.h = h
        _LIVE["plans"].add(self)
        self._host = _outputs(P, "host")
        self._freed_seen = _FREED_MAPS

    def _maps_alive(self):
        """Refuse to launch once a target map of the plan has been freed (its device tables
        no longer exist)."""
        if self._freed_seen != _FREED_MAPS:
            if any(m is not None and not getattr(m, "h", None) for m in self.vmaps):
                raise GlimError(-1, "a target voxelmap of this plan has been freed")
            self._freed_seen = _FREED_MAPS

    def linearize(self, poses, out=None, copy=True):
        """One upload, one graph launch, one download; returns host arrays (e, H, b, inliers).
        copy=False returns read-only views of the plan's pinned output block instead (no host
        copy), valid until the plan's next launch."""
        self._maps_alive()
        Pz = _poses(poses, self.nframes)
        if not copy and out is None:
            ptrs = [C.c_void_p() for _ in range(4)]
            self.ctx.call("plan_linearize_pinned", self.ctx.lib.glim_plan_linearize_pinned, self.h, _ptr(Pz),
                          *[C.byref(q) for q in ptrs])
            P = self.npairs
            views = []
            for q, shape, ct in zip(ptrs, [(P,), (P, 12, 12), (P, 12), (P,)],
                                    [C.c_double, C.c_double, C.c_double, C.c_int64]):
                a = np.ctypeslib.as_array(C.cast(q, C.POINTER(ct)), shape=shape) if P > 0 else np.zeros(shape)
                a.flags.writeable = False
                views.append(a)
            return tuple(views)
        e, H, b, inl = out if out is not None else self._host
        self.ctx.call("plan_linearize", self.ctx.lib.glim_plan_linearize, self.h, _ptr(Pz), _ptr(e), _ptr(H), _ptr(b), _ptr(inl))
        return e, H, b, inl

    def relative_poses(self):
        """The plan's current device pose block: (npairs, 3, 4) FP64 T_rel and (npairs, 16) FP32
        (R, t, target viewpoint, 0), as the kernels read them."""
        rt = np.empty((self.npairs, 12), np.float64)
        p32 = np.empty((self.npairs, 16), np.float32)
        self.ctx.call("plan_relative_poses", self.ctx.lib.glim_plan_relative_poses, self.h, _ptr(rt), _ptr(p32))
        T = np.empty((self.npairs, 3, 4), np.float64)
        T[:, :, :3] = rt[:, :9].reshape(-1, 3, 3)
        T[:, :, 3] = rt[:, 9:]
        return T, p32

    def correspondence_ids(self, poses):
        """Canonical voxel id of every (pair, source point, level) as the plan's own kernel
        resolves it (-1: miss), through the kernel's id-recording instantiation: an int32 CUDA
        tensor, per pair n_src x levels, pairs concatenated.  Also returns that launch's host
        (e, H, b, inliers)."""
        self._maps_alive()
        Pz = _poses(poses, self.nframes)
        lv = [self.vmaps[int(t)].levels for t in self._pairs_arr[:, 1]]
        n = sum(self.frames[int(s_)].n * l for s_, l in zip(self._pairs_arr[:, 0], lv))
        ids = torch.empty(max(n, 1), dtype=torch.int32, device=self.frames[0].pts4.device)
        e, H, b, inl = _outputs(self.npairs, "host")
        self.ctx.call("plan_correspondence_ids", self.ctx.lib.glim_plan_correspondence_ids, self.h, _ptr(Pz),
                      _ptr(ids), _ptr(e), _ptr(H), _ptr(b), _ptr(inl))
        return ids[:n], (e, H, b, inl)

    def set_poses(self, poses):
        self._maps_alive()
        Pz = _poses(poses, self.nframes)
        self.ctx.call("plan_set_poses", self.ctx.lib.glim_plan_set_poses, self.h, _ptr(Pz))

    def device_records(self):
        """The plan's factor records as a (npairs, 92) float64 CUDA tensor that shares the
        plan's device memory (no copy): [e, the upper triangle of H row by row (78), b (12),
        inliers] per pair, rewritten by every linearization of the plan.  Valid while the
        plan is open."""
        q = C.c_void_p()
        self.ctx.call("plan_device_records", self.ctx.lib.glim_plan_device_records, self.h, C.byref(q))
        return _device_view(q.value, (self.npairs, _abi.RECORD_DOUBLES), "<f8", self.frames[0].pts4.device)

    def device_outputs_alloc(self):
        """Device tensors (e, H, b, inliers) to pass as `out` to linearize."""
        return _outputs(self.npairs, self.frames[0].pts4.device)

    def backward(self, poses, omega_grad_full=True):
        """dE/dxi (nframes, 6) f64, dE/dmu (sum n, 3) f32, dE/dw (sum n,) f32 of the plan's
        batch."""
        self._maps_alive()
        Pz = _poses(poses, self.nframes)
        dev = self.frames[0].pts4.device
        ntot = sum(f.n for f in self.frames)
        dxi = torch.empty((self.nframes, 6), dtype=torch.float64, device=dev)
        dmu = torch.empty((ntot, 3), dtype=torch.float32, device=dev)
        dw = torch.empty((ntot,), dtype=torch.float32, device=dev)
        self.ctx.call("plan_backward", self.ctx.lib.glim_plan_backward, self.h, _ptr(Pz), int(omega_grad_full),
                      _ptr(dxi), _ptr(dmu), _ptr(dw))
        return dxi, dmu, dw

    def gauss_newton(self, poses, frame, iters=10):
        """Gauss-Newton on the device for `frame` with the other frames fixed: `iters`
        linearizations and steps without a host round trip.  Returns the final poses
        (nframes, 3, 4), the batch's total cost at each linearization (iters,) and the status
        (0, or the code for a system that was not positive definite)."""
        self._maps_alive()
        Pz = _poses(poses, self.nframes)
        out = np.empty_like(Pz)
        cost = np.empty(int(iters), np.float64)
        st = C.c_int32(0)
        self.ctx.call("plan_gauss_newton", self.ctx.lib.glim_plan_gauss_newton, self.h, _ptr(Pz), int(frame),
                      int(iters), _ptr(out), _ptr(cost), C.byref(st))
        return out.reshape(-1, 3, 4), cost, int(st.value)

    def launch(self):
        self._maps_alive()
        self.ctx.call("plan_launch", self.ctx.lib.glim_plan_launch, self.h)

    def launch_timed(self, slot):
        """Direct launches with CUDA events around the linearization kernel (timing slot)."""
        self._maps_alive()
        self.ctx.call("plan_launch_timed", self.ctx.lib.glim_plan_launch_timed, self.h, slot)

    def kernel_ms(self, nslots):
        out = (C.c_float * max(nslots, 1))()
        self.ctx.call("plan_kernel_ms", self.ctx.lib.glim_plan_kernel_ms, self.h, nslots, out)
        return np.array(out[:nslots], dtype=np.float64)

    @property
    def kernels_per_launch(self):
        return int(self.ctx.lib.glim_plan_kernels_per_launch(self.h))

    def device_outputs(self):
        """Views of the plan's device output block (valid until the next launch)."""
        e, H, b, inl = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        self.ctx.call("plan_device_outputs", self.ctx.lib.glim_plan_device_outputs, self.h, C.byref(e), C.byref(H), C.byref(b),
                                                             C.byref(inl))
        return e.value, H.value, b.value, inl.value

    def autotune(self, poses, iters=5):
        self._maps_alive()
        Pz = _poses(poses, self.nframes)
        o = _abi.LinOpts()
        ms = C.c_float()
        self.ctx.call("plan_autotune", self.ctx.lib.glim_plan_autotune, self.h, _ptr(Pz), iters, C.byref(o), C.byref(ms))
        return dict(block=o.block, pts_per_thread=o.pts_per_thread, ms=ms.value)

    def opts(self):
        o = _abi.LinOpts()
        self.ctx.call("plan_get_opts", self.ctx.lib.glim_plan_get_opts, self.h, C.byref(o))
        kernels = {v: k for k, v in KERNELS.items()}
        return dict(validate_surface=o.validate_surface, accum_mode=o.accum_mode, block=o.block,
                    pts_per_thread=o.pts_per_thread, blocks_per_sm=o.blocks_per_sm, persistent=o.persistent,
                    kernel=kernels[o.kernel])

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.glim_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def correspondences(ctx: Context, frame: FrameData, vmap: VoxelMap, pose_s, pose_t, validate_surface=False):
    """Canonical voxel id (n, levels) of every source point, -1 for a miss."""
    ids = torch.empty((frame.n, vmap.levels), dtype=torch.int32, device=frame.pts4.device)
    f = frame.c()
    ps = _poses(pose_s)
    pt = _poses(pose_t)
    ctx.call("correspondences", ctx.lib.glim_correspondences, ctx.h, C.byref(f), vmap.h, _ptr(ps), _ptr(pt), int(validate_surface),
                                           _ptr(ids))
    return ids


def overlap(ctx: Context, frames, vmaps, pairs, poses, level=0):
    fr = _frames(frames)
    pr, P = _pairs(pairs, vmaps)
    Pz = _poses(poses, len(frames))
    out = torch.empty(P, dtype=torch.float64, device=frames[0].pts4.device)
    ctx.call("overlap", ctx.lib.glim_overlap, ctx.h, fr, len(frames), pr, P, _ptr(Pz), level, _ptr(out))
    return out


def backward(ctx: Context, frames, vmaps, pairs, poses, omega_grad_full=True, validate_surface=False):
    """dE/dxi (nframes, 6) f64, dE/dmu (sum n, 3) f32, dE/dw (sum n,) f32 as CUDA tensors."""
    fr = _frames(frames)
    pr, P = _pairs(pairs, vmaps)
    Pz = _poses(poses, len(frames))
    dev = frames[0].pts4.device
    ntot = sum(f.n for f in frames)
    dxi = torch.empty((len(frames), 6), dtype=torch.float64, device=dev)
    dmu = torch.empty((ntot, 3), dtype=torch.float32, device=dev)
    dw = torch.empty((ntot,), dtype=torch.float32, device=dev)
    ctx.call("backward", ctx.lib.glim_backward, ctx.h, fr, len(frames), pr, P, _ptr(Pz), int(omega_grad_full),
                                    int(validate_surface), _ptr(dxi), _ptr(dmu), _ptr(dw))
    return dxi, dmu, dw


def gn_solve(ctx: Context, H: torch.Tensor, b: torch.Tensor, dim: int = None):
    """Solve H xi = -b per system; H (count, d, d) or (count, 12, 12) with dim 6 taking the
    top-left block; b (count, >= dim).  Returns xi (count, dim) and per-system status."""
    _dev(H, torch.float64, name="H")
    _dev(b, torch.float64, name="b")
    count = H.shape[0]
    ld = H.shape[-1]
    dim = dim or ld
    xi = torch.empty((count, dim), dtype=torch.float64, device=H.device)
    status = torch.empty(count, dtype=torch.int32, device=H.device)
    ctx.call("gn_solve", ctx.lib.glim_gn_solve, ctx.h, _ptr(H), ld, H.shape[-2] * ld, _ptr(b), b.shape[-1], dim,
             count, _ptr(xi), _ptr(status), ok=(0, -6))
    return xi, status


def shard_pairs(pairs, rank: int, world: int):
    """Partition a factor batch across `world` GPUs by source frame: the source frames, in
    order, are cut into `world` contiguous groups holding about the same number of pairs, and
    rank `rank` gets the indices of the pairs whose source is in its group.  Pairs are
    independent, so the ranks need no exchange until their (e, H, b) records are gathered;
    a rank must hold its source frames and the voxelmaps of their targets (see frames_needed).
    """
    pairs = np.asarray(pairs).reshape(-1, 2)
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    srcs = np.unique(pairs[:, 0])
    counts = np.array([(pairs[:, 0] == f).sum() for f in srcs])
    cum = np.cumsum(counts)
    total = cum[-1] if len(cum) else 0
    # group g holds the sources whose cumulative pair count falls in (g * total / world, ...]
    group = np.minimum((cum - 1) * world // max(total, 1), world - 1) if total else np.zeros(0, int)
    mine = set(srcs[group == rank].tolist())
    return np.array([i for i, (s_, _) in enumerate(pairs) if int(s_) in mine], dtype=np.int64)


class _DeviceArray:
    """Library-owned device memory described by the CUDA array interface, so that torch can
    view it without a copy (the library keeps ownership)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 2, "strides": None}


def _device_view(ptr, shape, typestr, device):
    if int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype=torch.float64, device=device)
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device=device)


_TRIU = np.triu_indices(12)


def pack_records(e, H, b, inliers):
    """Factor records (P, 92) of (e, H, b, inliers) in the library's record layout: e, the
    upper triangle of H row by row, b, the inlier count.  numpy in, numpy out; torch in,
    torch out (same device)."""
    if isinstance(e, torch.Tensor):
        P = e.shape[0]
        iu = torch.as_tensor(np.ravel_multi_index(_TRIU, (12, 12)), device=e.device)
        return torch.cat([e.reshape(P, 1).double(), H.reshape(P, 144).double()[:, iu], b.reshape(P, 12).double(),
                          inliers.reshape(P, 1).double()], dim=1)
    e = np.asarray(e, np.float64)
    P = len(e)
    H = np.asarray(H, np.float64).reshape(P, 12, 12)
    return np.concatenate([e.reshape(P, 1), H[:, _TRIU[0], _TRIU[1]], np.asarray(b, np.float64).reshape(P, 12),
                           np.asarray(inliers, np.float64).reshape(P, 1)], axis=1)


def unpack_records(rec):
    """(e, H (P, 12, 12) symmetric, b, inliers int64) of factor records (numpy or torch)."""
    is_t = isinstance(rec, torch.Tensor)
    r = rec.cpu().numpy() if is_t else np.asarray(rec, np.float64)
    P = r.shape[0]
    H = np.zeros((P, 12, 12))
    H[:, _TRIU[0], _TRIU[1]] = r[:, 1:79]
    H[:, _TRIU[1], _TRIU[0]] = r[:, 1:79]
    return r[:, 0].copy(), H, r[:, 79:91].copy(), np.rint(r[:, 91]).astype(np.int64)


def gather_records(rec, idx, npairs, group=None):
    """The exchange step of a factor batch sharded over ranks (shard_pairs): every rank holds
    the records `rec` (n_local, 92) of its pairs `idx` (global pair indices); one all-gather
    (torch.distributed: NCCL for CUDA tensors, gloo for CPU tensors) gives every rank the
    records of all `npairs` pairs in pair order, on rec's device.  A world of one returns the
    records placed in pair order."""
    import torch.distributed as dist
    rec_t = rec if isinstance(rec, torch.Tensor) else torch.as_tensor(np.asarray(rec, np.float64))
    dev = rec_t.device
    idx_t = torch.as_tensor(np.asarray(idx, np.int64), device=dev)
    if rec_t.shape[0] != idx_t.shape[0]:
        raise ValueError("records and pair indices differ in length")
    out = torch.zeros((npairs, rec_t.shape[1]), dtype=torch.float64, device=dev)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        out[idx_t] = rec_t.double()
        return out
    world = dist.get_world_size(group)
    n = torch.tensor([idx_t.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    m = int(max(int(c.item()) for c in counts))
    pad_r = torch.zeros((m, rec_t.shape[1]), dtype=torch.float64, device=dev)
    pad_r[:rec_t.shape[0]] = rec_t
    pad_i = torch.full((m,), -1, dtype=torch.int64, device=dev)
    pad_i[:idx_t.shape[0]] = idx_t
    all_r = [torch.empty_like(pad_r) for _ in range(world)]
    all_i = [torch.empty_like(pad_i) for _ in range(world)]
    dist.all_gather(all_r, pad_r, group=group)
    dist.all_gather(all_i, pad_i, group=group)
    for c, r_, i_ in zip(counts, all_r, all_i):
        k = int(c.item())
        out[i_[:k]] = r_[:k]
    return out


def frames_needed(pairs, idx):
    """Frames a rank must hold for the pairs `idx`: their sources and their targets."""
    pairs = np.asarray(pairs).reshape(-1, 2)
    sub = pairs[np.asarray(idx, dtype=np.int64)]
    return sorted(set(sub[:, 0].tolist()) | set(sub[:, 1].tolist()))


def graph_step(ctx: Context, pairs, nframes: int, H: torch.Tensor, b: torch.Tensor, fixed_frame: int = 0,
               lam: float = 0.0, want_system: bool = False):
    """Gauss-Newton / Levenberg-Marquardt step of a small factor graph (device): returns
    xi (nframes, 6) float64 CUDA tensor, and the assembled global (H, b) if want_system."""
    _dev(H, torch.float64, name="H")
    _dev(b, torch.float64, name="b")
    pf = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    xi = torch.empty((nframes, 6), dtype=torch.float64, device=H.device)
    Hg = torch.empty((6 * nframes, 6 * nframes), dtype=torch.float64, device=H.device) if want_system else None
    bg = torch.empty(6 * nframes, dtype=torch.float64, device=H.device) if want_system else None
    ctx.call("graph_step", ctx.lib.glim_graph_step, ctx.h, _ptr(pf), len(pf), nframes, _ptr(H), _ptr(b),
             int(fixed_frame), float(lam), _ptr(xi), _ptr(Hg), _ptr(bg))
    return (xi, Hg, bg) if want_system else xi
