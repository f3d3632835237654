"""The linearization entry point that allocates nothing (glim_linearize_factors_noalloc).

It serves callers that cannot allocate device memory while they linearize (device memory
reserved up front by another allocator, or real-time loops that must not block in the
driver).  Its results must match the regular entry point, call after call, although every
call reuses the same static scratch array.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def _setup(layout="auto"):
    import paper_2407_10344_b300 as G
    from paper_2407_10344_b300 import _abi
    ctx = G.Context(0)
    w = synth.corridor()
    dev = torch.device("cuda", 0)
    frames, maps = [], [None] * len(w.points)
    for i, p in enumerate(w.points):
        p4 = G.to_pts4(p, device=dev)
        cov, nrm = G.estimate_covariances(ctx, p4)
        frames.append(G.FrameData(p4, cov, nrm))
        if i > 0:
            maps[i] = G.VoxelMap(ctx, p4, cov, w.resolutions, layout=layout)
    torch.cuda.synchronize()
    return G, _abi, ctx, w, frames, maps


def _call_noalloc(G, _abi, ctx, w, frames, maps, pairs, kernel=0):
    fr = (_abi.Frame * len(frames))(*[f.c() for f in frames])
    pr = (_abi.Pair * len(pairs))(*[_abi.Pair(int(s), int(t), maps[int(t)].h.value) for s, t in pairs])
    poses = np.ascontiguousarray(w.poses.reshape(-1, 12))
    P = len(pairs)
    e = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    H = torch.full((P, 12, 12), float("nan"), dtype=torch.float64, device="cuda")
    b = torch.full((P, 12), float("nan"), dtype=torch.float64, device="cuda")
    inl = torch.full((P,), -1, dtype=torch.int64, device="cuda")
    opts = _abi.LinOpts()
    opts.kernel = kernel
    st = ctx.call("linearize_factors_noalloc", ctx.lib.glim_linearize_factors_noalloc, ctx.h, fr, len(frames), pr,
                  P, poses.ctypes.data_as(C.c_void_p), C.byref(opts), C.c_void_p(e.data_ptr()),
                  C.c_void_p(H.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(inl.data_ptr()))
    assert st == 0
    torch.cuda.synchronize()
    return e.cpu().numpy(), H.cpu().numpy(), b.cpu().numpy(), inl.cpu().numpy()


@pytest.mark.parametrize("layout", ["auto", "hash"])
def test_noalloc_matches_regular_entry_point_twice(layout):
    G, _abi, ctx, w, frames, maps = _setup(layout)
    ref = G.linearize(ctx, frames, maps, w.pairs, w.poses, out="cuda")
    ref = [x.cpu().numpy() for x in ref]
    lane_kernel = 2 if layout == "auto" else 3
    for kernel in (0, 0, 1, lane_kernel):  # two calls in a row share (and overwrite) the static scratch
        e, H, b, inl = _call_noalloc(G, _abi, ctx, w, frames, maps, w.pairs, kernel=kernel)
        assert np.array_equal(inl, ref[3])
        assert _rel(e, ref[0]) <= TOL and _rel(H, ref[1]) <= TOL and _rel(b, ref[2]) <= TOL
    other = 3 if layout == "auto" else 2  # the per-lane kernel of the other layout is refused
    with pytest.raises(G.GlimError, match="EINVAL"):
        _call_noalloc(G, _abi, ctx, w, frames, maps, w.pairs, kernel=other)
    # a different batch (fewer pairs) through the same scratch
    e, H, b, inl = _call_noalloc(G, _abi, ctx, w, frames, maps, w.pairs[3:5])
    assert np.array_equal(inl, ref[3][3:5])
    assert _rel(H, ref[1][3:5]) <= TOL


def test_noalloc_rejects_batches_beyond_its_limits():
    G, _abi, ctx, w, frames, maps = _setup()
    too_many = np.repeat(w.pairs, 26, axis=0)  # 260 pairs > 256
    with pytest.raises(G.GlimError, match="exceed the limits"):
        _call_noalloc(G, _abi, ctx, w, frames, maps, too_many)


def test_noalloc_refuses_stream_capture():
    """Every call stages its descriptors in one host block that the next call rewrites, so a
    call made while the context's stream captures a graph is refused (GLIM_EINVAL) and
    enqueues nothing; a call after the capture works as before."""
    G, _abi, ctx, w, frames, maps = _setup()
    ref = _call_noalloc(G, _abi, ctx, w, frames, maps, w.pairs)  # the set-up happens before any capture
    fr = (_abi.Frame * len(frames))(*[f.c() for f in frames])
    pr = (_abi.Pair * len(w.pairs))(*[_abi.Pair(int(s), int(t), maps[int(t)].h.value) for s, t in w.pairs])
    poses = np.ascontiguousarray(w.poses.reshape(-1, 12))
    P = len(w.pairs)
    shapes = [((P,), torch.float64), ((P * 144,), torch.float64), ((P * 12,), torch.float64), ((P,), torch.int64)]
    out = [torch.empty(n, dtype=dt, device="cuda") for n, dt in shapes]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(ctx.stream):
        g.capture_begin()
        try:
            st = ctx.lib.glim_linearize_factors_noalloc(ctx.h, fr, len(frames), pr, P, poses.ctypes.data_as(C.c_void_p),
                                                        None, *[C.c_void_p(t.data_ptr()) for t in out])
        finally:
            g.capture_end()
    assert st == -1
    assert b"capturing" in ctx.lib.glim_last_error(ctx.h)
    e, H, b, inl = _call_noalloc(G, _abi, ctx, w, frames, maps, w.pairs)
    assert np.array_equal(inl, ref[3]) and np.array_equal(H, ref[1])
