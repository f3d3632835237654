"""Correspondences as the linearization kernels themselves resolve them, bit-exact against
the oracle (Sec. III-C "Correspondence search": q = R mu + t on the FP32 path, key
floor(q * inv_r), exactly one voxel per level).

Every plan below runs the id-recording instantiation of the kernel it uses for e, H and b
(the per-lane dense-grid kernel, the per-lane hash kernel, or the general kernel with its
level-0 shift of the keys), in the plan's own launch configuration.  Its ids must equal the
oracle's for every (pair, point, level), and its e, H, b and inlier counts must be the same
bits as the production instantiation's, so that the ids are the ones the sums used.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    import paper_2407_10344_b300 as G
    return G


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


def _check_plan(G, ctx, frames, maps, pairs, poses, ref_ids, kernel, validate=False, block=0, ppt=0, ref=None):
    """The plan's kernel ids == the oracle's ids; the id-recording launch reproduces the
    production launch bit for bit.  Returns the kernel the plan ran and the hit fraction."""
    plan = G.Plan(ctx, frames, maps, pairs, kernel=kernel, validate_surface=validate, block=block,
                  pts_per_thread=ppt)
    ran = plan.opts()["kernel"]
    ids, (e1, H1, b1, inl1) = plan.correspondence_ids(poses)
    got = ids.cpu().numpy()
    assert got.shape == ref_ids.shape
    bad = np.flatnonzero(got != ref_ids)
    assert len(bad) == 0, (ran, len(bad), bad[:8], got[bad[:8]], ref_ids[bad[:8]])
    e0, H0, b0, inl0 = [np.array(x) for x in plan.linearize(poses)]
    assert np.array_equal(e0, e1) and np.array_equal(H0, H1) and np.array_equal(b0, b1)
    assert np.array_equal(inl0, inl1)
    if ref is not None:
        from gpu_helpers import rel_errors
        assert (inl0 == ref["inliers"]).all()
        assert max(m.max() for m in rel_errors(e0, H0, b0, ref)[:3]) <= TOL
    plan.close()
    return ran, float((got >= 0).mean())


# ---------------------------------------------------------------------------- face points
def test_kernel_ids_face_points(G, ctx):
    """Source points whose transformed coordinates sit within an ulp of a voxel face (the
    x coordinate of the target-frame point on a multiple of the voxel size), under a rotation
    that mixes all three axes: the FP32 transform decides the side, on every kernel."""
    res = 0.5
    Ts = synth.make_pose(synth.rot_axis_angle([0.6, -0.2, 0.7], 0.9), [1.3, -0.7, 0.4])
    Tt = np.eye(3, 4)
    s = synth.Stream(14, "faces")
    n = 5000
    face = np.stack([np.round(s.uniform(n, -4, 4) / res) * res, s.uniform(n, -4, 4), s.uniform(n, -4, 4)], 1)
    mu = ((face - Ts[:, 3]) @ Ts[:, :3]).astype(np.float32)
    tgt = np.concatenate([face, face + [res / 2, 0, 0], face - [res / 2, 0, 0]]).astype(np.float32)
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (len(tgt), 1))
    src4, scov = O.as_pts4(mu), cov[:n]
    of = [O.Frame(src4, scov), O.Frame(O.as_pts4(tgt), cov)]
    om = [None, O.VMap(of[1].pts4, of[1].cov6, [res])]
    poses = np.stack([Ts, Tt])
    pairs = np.array([[0, 1]], np.int32)
    ref = O.linearize(of, om, pairs, poses, want_ids=True, want_comp=True)
    frames = [G.FrameData(torch.as_tensor(f.pts4, device="cuda"), torch.as_tensor(f.cov6, device="cuda"))
              for f in of]
    seen = set()
    for layout in ("dense", "hash"):
        gm = [None, G.VoxelMap(ctx, frames[1].pts4, frames[1].cov6, [res], layout=layout)]
        for kernel, block, ppt in (("auto", 0, 0), ("general", 0, 0), ("auto", 128, 3)):
            ran, hit = _check_plan(G, ctx, frames, gm, pairs, poses, ref["ids"], kernel, block=block, ppt=ppt,
                                   ref=ref)
            seen.add(ran)
            assert hit > 0.3
    assert seen == {"dense", "hash", "general"}


# ---------------------------------------------------------------------------- key range edge
@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_kernel_ids_at_the_edge_of_the_key_range(G, ctx, layout):
    """Voxels at keys 2^20 - 1 and -2^20 (0.5 m; 1 m at level 1) and points one key beyond:
    the points inside resolve to their voxels and the ones beyond miss, as the oracle says,
    at the identity and after a shift that carries points across the boundary.  Every
    coordinate is a multiple of 1/16 m, so the FP32 transform is exact."""
    res = [0.5, 1.0]
    edge = 2 ** 20

    def cluster(k0):
        out = []
        for kx in (k0 - 1, k0):
            for ky in (-1, 0):
                for kz in (-1, 0):
                    c = np.array([kx + 0.5, ky + 0.5, kz + 0.5]) * res[0]
                    for a in ([0.125, 0.0625, 0.0625], [0.0625, -0.125, 0.0625]):
                        out += [c + a, c - np.array(a)]
        return np.array(out)

    beyond = np.array([[(edge + 0.5) * res[0], 0.125, 0.125], [(-edge - 0.5) * res[0], -0.1875, 0.3125]])
    src = np.concatenate([cluster(edge - 1), cluster(-edge + 1), beyond]).astype(np.float32)
    m = len(src) // 2 - 1
    pts = [src, src[:m], src[m:2 * m]]
    of = [O.Frame(O.as_pts4(p), np.tile(np.array([0.01, 0, 0, 0.01, 0, 0.01], np.float32), (len(p), 1)))
          for p in pts]
    om = [None, O.VMap(of[1].pts4, of[1].cov6, res), O.VMap(of[2].pts4, of[2].cov6, res)]
    gf = [G.FrameData(torch.as_tensor(f.pts4, device="cuda"), torch.as_tensor(f.cov6, device="cuda")) for f in of]
    gm = [None] + [G.VoxelMap(ctx, gf[i].pts4, gf[i].cov6, res, layout=layout) for i in (1, 2)]
    pairs = np.array([[0, 1], [0, 2]], np.int32)
    for shift in (0.0, 0.3125):
        poses = np.stack([np.eye(3, 4)] * 3)
        poses[0, 0, 3] = shift
        ref = O.linearize(of, om, pairs, poses, want_ids=True, want_comp=True)
        for kernel in ("auto", "general"):
            _check_plan(G, ctx, gf, gm, pairs, poses, ref["ids"], kernel, ref=ref)


# ---------------------------------------------------------------------------- probe chains
def _home_slot(bx, by, bz, log2cap):
    """Home slot of a block key in a hashed level's table, as the library lays the table out
    (the top log2cap bits of the 32-bit linear hash of the block key)."""
    h = (np.int64(bx) * 0xFFE6CC61 + np.int64(by) * 0xFC4A3B47 + np.int64(bz) * 0x27004D2D) & 0xFFFFFFFF
    return int(h) >> (32 - log2cap)


def test_kernel_ids_through_long_probe_chains(G, ctx):
    """Hashed voxel blocks whose keys share one home slot, so that finding them takes probe
    chains of up to nine entries, plus blocks absent from the map whose home slot is the same
    one (their lookups walk the chain to the first empty entry) and empty cells of present
    blocks: every kernel must resolve each (point, level) to the oracle's voxel or miss.  The
    block keys are chosen on the host for the table size the build picks (load <= 1/16)."""
    res = 1.0
    s = synth.Stream(21, "probe-chains")
    nblk = 12
    log2cap = int(np.ceil(np.log2(16 * nblk)))  # 16 * 12 = 192 -> 256 entries
    chain, absent, others = [], [], []
    target = None
    while len(chain) < 9 or len(absent) < 4 or len(others) < nblk - 9:
        b = tuple(int(v) for v in s.integers(3, -40, 40))
        if b in chain or b in absent or b in others:
            continue
        h = _home_slot(*b, log2cap)
        if target is None:
            target = h
        if h == target and len(chain) < 9:
            chain.append(b)
        elif h == target and len(absent) < 4:
            absent.append(b)
        elif h in ((target + 1) % 256, (target + 2) % 256) and len(others) < nblk - 9:
            others.append(b)  # present blocks whose home slots lie inside the chain
    present = chain + others
    # one voxel per present block, at a cell chosen by the stream; three points per voxel
    tgt, src = [], []
    for b in present:
        loc = s.integers(3, 0, 2)
        k = np.array(b) * 2 + loc
        c = (k + 0.5) * res
        tgt += [c + [0.1, 0.0, 0.0], c - [0.1, 0.0, 0.0], c + [0.0, 0.1, 0.05]]
        src.append(c + [0.05, -0.05, 0.05])                       # hit
        src.append((np.array(b) * 2 + (1 - loc) + 0.5) * res)  # empty cell of a present block
    for b in absent:
        src.append((np.array(b) * 2 + 0.5) * res)               # block not in the table
    tgt = np.array(tgt, np.float32)
    src = np.array(src, np.float32)
    cov = lambda n: np.tile(np.array([0.02, 0.001, 0, 0.03, 0.002, 0.01], np.float32), (n, 1))
    of = [O.Frame(O.as_pts4(src), cov(len(src))), O.Frame(O.as_pts4(tgt), cov(len(tgt)))]
    om = [None, O.VMap(of[1].pts4, of[1].cov6, [res])]
    poses = np.stack([np.eye(3, 4)] * 2)
    pairs = np.array([[0, 1]], np.int32)
    ref = O.linearize(of, om, pairs, poses, want_ids=True, want_comp=True)
    ids = ref["ids"]
    assert (ids[0::2][:len(present)] >= 0).all() and (ids[1:2 * len(present):2] < 0).all()
    assert (ids[2 * len(present):] < 0).all()
    gf = [G.FrameData(torch.as_tensor(f.pts4, device="cuda"), torch.as_tensor(f.cov6, device="cuda")) for f in of]
    gm = [None, G.VoxelMap(ctx, gf[1].pts4, gf[1].cov6, [res], layout="hash")]
    assert not gm[1].is_dense(0)
    assert gm[1].info(0)["max_probe"] >= 9
    seen = set()
    for kernel, block, ppt in (("auto", 0, 0), ("general", 0, 0), ("auto", 128, 1)):
        ran, _ = _check_plan(G, ctx, gf, gm, pairs, poses, ids, kernel, block=block, ppt=ppt, ref=ref)
        seen.add(ran)
    assert seen == {"hash", "general"}
    got = G.correspondences(ctx, gf[0], gm[1], poses[0], poses[1]).cpu().numpy()
    assert np.array_equal(got.reshape(ids.shape), ids)


# ---------------------------------------------------------------------------- scenes
@pytest.fixture(scope="module")
def room(ctx):
    from gpu_helpers import Prepared
    w = synth.box_room()
    w.resolutions = [0.5, 1.0, 2.0]
    return Prepared(ctx, w)


@pytest.fixture(scope="module")
def corridor(ctx):
    from gpu_helpers import Prepared
    return Prepared(ctx, synth.corridor())


def _hash_maps(G, ctx, P):
    return [None if m is None else G.VoxelMap(ctx, P.gframes[i].pts4, P.gframes[i].cov6, P.w.resolutions,
                                              layout="hash") for i, m in enumerate(P.gmaps)]


@pytest.mark.parametrize("validate", [False, True])
def test_kernel_ids_room_and_corridor(G, ctx, room, corridor, validate):
    """Box room (3 levels, unary factor) and corridor window (10 binary factors), surface
    validation on and off, on dense grids and on hash tables, per-lane and general kernels."""
    for P in (room, corridor):
        ref = P.oracle(validate=validate, want_ids=True)
        layouts = {"dense": P.gmaps, "hash": _hash_maps(G, ctx, P)}
        for name, maps in layouts.items():
            for kernel in ("auto", "general"):
                ran, hit = _check_plan(G, ctx, P.gframes, maps, P.w.pairs, P.w.poses, ref["ids"], kernel,
                                       validate=validate, ref=ref)
                assert ran == (name if kernel == "auto" else "general")
                assert hit > 0.2


@pytest.mark.parametrize("layout", ["auto", "hash"])
def test_kernel_ids_urban_submaps(G, ctx, layout):
    """The first 12 urban submaps at a fifth of the point density (0.5 / 1 / 2 m, 3 targets
    per source), with ragged tiles (block 128, 3 points per thread) and the default tiles."""
    from gpu_helpers import Prepared
    w = synth.urban(n_submaps=400, neighbours=3, point_scale=0.2, keep=12)
    P = Prepared(ctx, w, layout=layout)
    for validate in (False, True):
        ref = P.oracle(validate=validate, want_ids=True)
        for kernel, block, ppt in (("auto", 0, 0), ("auto", 128, 3), ("general", 0, 0)):
            _check_plan(G, ctx, P.gframes, P.gmaps, w.pairs, w.poses, ref["ids"], kernel, validate=validate,
                        block=block, ppt=ppt, ref=ref)


def test_kernel_ids_mixed_layouts_and_nonfinite(G, ctx, room):
    """A batch whose targets mix dense grids and hash tables runs the general kernel; a
    source point with a NaN coordinate resolves to -1 at every level."""
    w = room.w
    src = room.gframes[0]
    p4 = src.pts4.clone()
    p4[7, 1] = float("nan")
    p4[11, 0] = float("inf")
    fr = [G.FrameData(p4, src.cov6, src.normal3), room.gframes[1], room.gframes[1]]
    hm = G.VoxelMap(ctx, room.gframes[1].pts4, room.gframes[1].cov6, w.resolutions, layout="hash")
    maps = [None, room.gmaps[1], hm]
    pairs = np.array([[0, 1], [0, 2]], np.int32)
    poses = np.stack([w.poses[0], w.poses[1], w.poses[1]])
    of = [O.Frame(p4.cpu().numpy(), room.oframes[0].cov6, room.oframes[0].normal3), room.oframes[1], room.oframes[1]]
    om = [None, room.omaps[1], room.omaps[1]]
    ref = O.linearize(of, om, pairs, poses, want_ids=True, want_comp=True)
    ran, _ = _check_plan(G, ctx, fr, maps, pairs, poses, ref["ids"], "auto", ref=ref)
    assert ran == "general"
    L = len(w.resolutions)
    ids = ref["ids"].reshape(2, -1, L)
    assert (ids[:, 7] < 0).all() and (ids[:, 11] < 0).all()
