"""Parity of the CUDA path against the FP64 oracle (element by element on the same seeded
inputs): voxel keys and correspondence ids bit-exact, e / H / b within 1e-4 relative
(norm-wise, see gpu_helpers.rel_errors), covariances within 1e-4, gradients, the
Gauss-Newton step, the overlap rate, determinism and edge cases."""
import math

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


@pytest.fixture(scope="module", params=["auto", "hash"])
def urban_small(ctx, request):
    """Urban submaps at realistic spacing (the first 12 submaps of the 400-submap trajectory,
    at a fifth of the point density), with dense-grid and with hash-table voxelmaps."""
    from gpu_helpers import Prepared
    w = synth.urban(n_submaps=400, neighbours=3, point_scale=0.2, keep=12)
    P = Prepared(ctx, w, layout=request.param)
    t = int(w.pairs[0, 1])
    assert all(P.gmaps[t].is_dense(l) == (request.param == "auto") for l in range(3))
    return P


def _check(res, ref, tol=TOL):
    from gpu_helpers import numpy_of, rel_errors
    e, H, b, inl = [numpy_of(x) for x in res]
    ee, eH, eb = rel_errors(e, H, b, ref)
    assert (inl == ref["inliers"]).all(), (inl, ref["inliers"])
    assert ee.max() <= tol and eH.max() <= tol and eb.max() <= tol, (ee.max(), eH.max(), eb.max())
    return ee.max(), eH.max(), eb.max()


# ---------------------------------------------------------------------------- voxelmap
@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_voxelmap_matches_oracle(G, ctx, room, layout):
    g = room.gframes[1]
    gm, om = G.VoxelMap(ctx, g.pts4, g.cov6, room.w.resolutions, layout=layout), room.omaps[1]
    for l in range(om.levels):
        g = {k: v.cpu().numpy() for k, v in gm.export(l).items()}
        o = om.export(l)
        assert np.array_equal(g["keys"], o["keys"])          # canonical order, bit-exact keys
        assert np.array_equal(g["count"], o["count"])
        np.testing.assert_allclose(g["mean"], o["mean"], rtol=0, atol=2e-6 * max(1.0, np.abs(o["mean"]).max()))
        np.testing.assert_allclose(g["cov"], o["cov"], rtol=0, atol=2e-6 * np.abs(o["cov"]).max())
        info = gm.info(l)
        assert gm.is_dense(l) == (layout == "dense")
        assert info["capacity"] >= info["n_voxels"] and info["max_probe"] >= 1
        if layout == "hash":  # whole 2 x 2 x 2 blocks: at most 8 cells per voxel
            assert info["capacity"] % 8 == 0 and info["capacity"] <= 8 * info["n_voxels"]


def test_voxelmap_face_points_and_negative_coordinates(G, ctx):
    g = O.as_pts4(np.array([[0.25, 0.25, 0.25], [0.75, 0.5, 0.25], [-0.5, 0.125, 0.0], [-1.0, 0.0, -0.0],
                            [-1e-30, 2.0, -2.0]]))
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (len(g), 1))
    gm = G.VoxelMap(ctx, torch.as_tensor(g, device="cuda"), torch.as_tensor(cov, device="cuda"), [1.0, 0.5])
    om = O.VMap(g, cov, [1.0, 0.5])
    for l in range(2):
        assert np.array_equal(gm.export(l)["keys"].cpu().numpy(), om.export(l)["keys"])


def test_voxelmap_errors(G, ctx):
    cov = torch.tensor([[1, 0, 0, 1, 0, 1]] * 2, dtype=torch.float32, device="cuda")
    far = torch.tensor([[0, 0, 0, 1], [2.0 ** 21, 0, 0, 1]], dtype=torch.float32, device="cuda")
    with pytest.raises(G.GlimError, match="ERANGE"):
        G.VoxelMap(ctx, far, cov, [1.0])
    bad = torch.tensor([[0, 0, 0, 1], [float("nan"), 0, 0, 1]], dtype=torch.float32, device="cuda")
    with pytest.raises(G.GlimError, match="EINVAL"):
        G.VoxelMap(ctx, bad, cov, [1.0])
    # the context stays usable after the errors
    ok = G.VoxelMap(ctx, far[:1].clone(), cov[:1].clone(), [1.0])
    assert ok.info(0)["n_voxels"] == 1


# ---------------------------------------------------------------------------- correspondences
@pytest.mark.parametrize("validate", [False, True])
@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_correspondence_ids_bit_exact(G, ctx, room, validate, layout):
    w = room.w
    g = room.gframes[1]
    vm = G.VoxelMap(ctx, g.pts4, g.cov6, w.resolutions, layout=layout)
    gid = G.correspondences(ctx, room.gframes[0], vm, w.poses[0], w.poses[1], validate).cpu().numpy()
    ref = room.oracle(validate=validate, want_ids=True)
    assert np.array_equal(gid.reshape(-1), ref["ids"])
    assert (gid >= 0).mean() > 0.5


def test_correspondences_face_points(G, ctx):
    """Points whose transformed coordinates sit within an ulp of a voxel face."""
    res = 0.5
    Ts = synth.make_pose(synth.rot_axis_angle([0.6, -0.2, 0.7], 0.9), [1.3, -0.7, 0.4])
    Tt = np.eye(3, 4)
    s = synth.Stream(14, "faces")
    n = 5000
    face = np.stack([np.round(s.uniform(n, -4, 4) / res) * res, s.uniform(n, -4, 4), s.uniform(n, -4, 4)], 1)
    mu = ((face - Ts[:, 3]) @ Ts[:, :3]).astype(np.float32)
    tgt = np.concatenate([face, face + [res / 2, 0, 0], face - [res / 2, 0, 0]]).astype(np.float32)
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (len(tgt), 1))
    om = O.VMap(O.as_pts4(tgt), cov, [res])
    src4 = O.as_pts4(mu)
    scov = cov[:n]
    fr = G.FrameData(torch.as_tensor(src4, device="cuda"), torch.as_tensor(scov, device="cuda"))
    ref = O.linearize([O.Frame(src4, scov), O.Frame(O.as_pts4(tgt), cov)], [None, om], [[0, 1]],
                      np.stack([Ts, Tt]), want_ids=True)
    for layout in ("dense", "hash"):
        gm = G.VoxelMap(ctx, torch.as_tensor(O.as_pts4(tgt), device="cuda"), torch.as_tensor(cov, device="cuda"),
                        [res], layout=layout)
        gid = G.correspondences(ctx, fr, gm, Ts, Tt).cpu().numpy().reshape(-1)
        assert np.array_equal(gid, ref["ids"])


# ---------------------------------------------------------------------------- linearization
@pytest.mark.parametrize("acc", [0, 1, 2])
def test_linearize_room_all_accum_modes(G, ctx, room, acc):
    ref = room.oracle()
    res = G.linearize(ctx, room.gframes, room.gmaps, room.w.pairs, room.w.poses, accum_mode=acc)
    _check(res, ref)


@pytest.mark.parametrize("validate", [False, True])
def test_linearize_corridor_batched_plan(G, ctx, corridor, validate):
    ref = corridor.oracle(validate=validate)
    plan = G.Plan(ctx, corridor.gframes, corridor.gmaps, corridor.w.pairs, validate_surface=validate)
    for _ in range(2):  # first call captures the graph, second replays it
        res = plan.linearize(corridor.w.poses)
        _check(res, ref)
    plan.close()


def test_linearize_device_outputs_and_plain(G, ctx, corridor):
    ref = corridor.oracle()
    res_dev = G.linearize(ctx, corridor.gframes, corridor.gmaps, corridor.w.pairs, corridor.w.poses, out="cuda")
    _check(res_dev, ref)
    res_plain = G.linearize(ctx, corridor.gframes, corridor.gmaps, corridor.w.pairs, corridor.w.poses, plain=True)
    _check(res_plain, ref)


@pytest.mark.parametrize("block,ppt", [(128, 1), (128, 8), (256, 2), (256, 4)])
def test_linearize_urban_multilevel_tiles(G, ctx, urban_small, block, ppt):
    ref = urban_small.oracle(validate=True)
    res = G.linearize(ctx, urban_small.gframes, urban_small.gmaps, urban_small.w.pairs, urban_small.w.poses,
                      validate_surface=True, block=block, pts_per_thread=ppt)
    _check(res, ref)


def test_linearize_grid_variant_and_autotune(G, ctx, urban_small):
    w = urban_small.w
    ref = urban_small.oracle()
    res = G.linearize(ctx, urban_small.gframes, urban_small.gmaps, w.pairs, w.poses, persistent=2)
    _check(res, ref)
    plan = G.Plan(ctx, urban_small.gframes, urban_small.gmaps, w.pairs)
    best = plan.autotune(w.poses, iters=2)
    assert best["block"] in (64, 128, 256) and 1 <= best["pts_per_thread"] <= 256 and best["ms"] > 0
    _check(plan.linearize(w.poses), ref)


def test_deterministic_and_partitioned(G, ctx, urban_small):
    """Two runs are bit-identical, and splitting the pair list into parts run one after the
    other reproduces the full run bit for bit (the multi-GPU partitioning)."""
    w = urban_small.w
    r1 = G.linearize(ctx, urban_small.gframes, urban_small.gmaps, w.pairs, w.poses)
    r2 = G.linearize(ctx, urban_small.gframes, urban_small.gmaps, w.pairs, w.poses)
    for a, b in zip(r1, r2):
        assert np.array_equal(a, b)
    parts = np.array_split(np.arange(len(w.pairs)), 3)
    cat = [G.linearize(ctx, urban_small.gframes, urban_small.gmaps, w.pairs[idx], w.poses) for idx in parts]
    for j in range(4):
        assert np.array_equal(np.concatenate([c[j] for c in cat]), r1[j])


def test_edge_cases_empty_ragged_and_misses(G, ctx, room):
    """Empty source frame, a source smaller than one tile, a ragged tail, and a pair whose
    points all miss (poses far apart)."""
    dev = torch.device("cuda")
    src = room.gframes[0]
    empty = G.FrameData(torch.zeros((0, 4), device=dev), torch.zeros((0, 6), device=dev))
    tiny = G.FrameData(src.pts4[:37].clone(), src.cov6[:37].clone())
    ragged = G.FrameData(src.pts4[:1025 + 3].clone(), src.cov6[:1025 + 3].clone())
    frames = [empty, tiny, ragged, room.gframes[1]]
    oframes = [O.Frame(f.pts4.cpu().numpy(), f.cov6.cpu().numpy()) for f in frames]
    gmaps = [None, None, None, room.gmaps[1]]
    omaps = [None, None, None, room.omaps[1]]
    pairs = np.array([[0, 3], [1, 3], [2, 3], [2, 3]], np.int32)
    poses = np.stack([room.w.poses[0]] * 3 + [room.w.poses[1]])
    far = poses.copy()
    far[2, :, 3] += 500.0
    for P in (poses, far):
        ref = O.linearize(oframes, omaps, pairs, P, want_comp=True)
        res = G.linearize(ctx, frames, gmaps, pairs, P)
        assert res[0][0] == 0 and not res[1][0].any() and res[3][0] == 0
        if P is far:
            assert res[3][2] == 0 and res[0][2] == 0
        ok = ref["e"] > 0
        from gpu_helpers import rel_errors
        ee, eH, eb = rel_errors(res[0][ok], res[1][ok], res[2][ok], {k: v[ok] for k, v in ref.items()})
        assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL
        assert np.array_equal(res[3], ref["inliers"])


@pytest.mark.parametrize("kernel", ["general", "dense"])
@pytest.mark.parametrize("validate", [False, True])
def test_dense_grid_kernel_and_general_kernel(G, ctx, room, kernel, validate):
    """The dense-grid kernel (chosen automatically when every target level is a dense grid)
    and the general kernel both match the oracle on the same dense maps, across every
    accumulation mode, one block per item and the persistent queue."""
    assert all(room.gmaps[1].is_dense(l) for l in range(len(room.w.resolutions)))
    ref = room.oracle(validate=validate)
    for acc in (G.ACC_FP32, G.ACC_KAHAN, G.ACC_FP64):
        for persistent, block, ppt in ((1, 128, 64), (2, 256, 3)):
            res = G.linearize(ctx, room.gframes, room.gmaps, room.w.pairs, room.w.poses, kernel=kernel,
                              validate_surface=validate, accum_mode=acc, persistent=persistent, block=block,
                              pts_per_thread=ppt)
            _check(res, ref)
    plan = G.Plan(ctx, room.gframes, room.gmaps, room.w.pairs, kernel="auto")
    assert plan.opts()["kernel"] == "dense"


@pytest.mark.parametrize("kernel", ["dense", "general"])
def test_degenerate_covariances_and_zero_weights(G, ctx, room, kernel):
    """Degenerate cases of the cost: source points whose covariance is zero, so that S = C~ +
    R C R^T is singular wherever the voxel covariance is zero too (the term is skipped, the
    hit is no inlier), voxels with zero covariance, points of weight zero (they add nothing
    and still count) and of negative weight, against the oracle."""
    dev = torch.device("cuda")
    src, tgt = room.gframes[0], room.gframes[1]
    n = src.n
    sel = torch.arange(n, device=dev)
    cov_s = src.cov6.clone()
    cov_s[sel % 7 == 0] = 0.0                      # zero source covariances
    p4 = src.pts4.clone()
    p4[sel % 11 == 0, 3] = 0.0                     # zero weights
    p4[sel % 13 == 0, 3] = 2.5                     # some non-unit ones
    p4[sel % 17 == 0, 3] = -0.5                    # and negative ones (the sums take w as given)
    cov_t = tgt.cov6.clone()
    cov_t[torch.arange(tgt.n, device=dev) % 5 == 0] = 0.0   # zero covariances in some voxels' means
    frames = [G.FrameData(p4, cov_s), G.FrameData(tgt.pts4, cov_t)]
    vm = G.VoxelMap(ctx, tgt.pts4, cov_t, room.w.resolutions)
    oframes = [O.Frame(p4.cpu().numpy(), cov_s.cpu().numpy()), O.Frame(tgt.pts4.cpu().numpy(), cov_t.cpu().numpy())]
    om = O.VMap(oframes[1].pts4, oframes[1].cov6, room.w.resolutions)
    ref = O.linearize(oframes, [None, om], room.w.pairs, room.w.poses, want_comp=True)
    _check(G.linearize(ctx, frames, [None, vm], room.w.pairs, room.w.poses, kernel=kernel), ref)
    # every source covariance and every voxel covariance zero: every S is singular, every term
    # is skipped (and is no inlier), although the correspondences exist
    z = G.FrameData(p4, torch.zeros_like(cov_s))
    vz = G.VoxelMap(ctx, tgt.pts4, torch.zeros_like(cov_t), room.w.resolutions)
    e, H, b, inl = G.linearize(ctx, [z, G.FrameData(tgt.pts4, torch.zeros_like(cov_t))], [None, vz], room.w.pairs,
                               room.w.poses, kernel=kernel)
    assert inl[0] == 0 and e[0] == 0.0 and not np.any(H) and not np.any(b)
    ids = G.correspondences(ctx, z, vz, room.w.poses[0], room.w.poses[1]).cpu().numpy()
    assert (ids >= 0).sum() > 0


def test_plan_linearize_pinned_views(G, ctx, corridor):
    """The zero-copy form returns the same numbers as the copying form, as read-only views
    of the plan's pinned block that the next launch overwrites."""
    w = corridor.w
    plan = G.Plan(ctx, corridor.gframes, corridor.gmaps, w.pairs)
    ref = [np.array(x) for x in plan.linearize(w.poses)]
    views = plan.linearize(w.poses, copy=False)
    for a, b in zip(views, ref):
        assert np.array_equal(a, b)
    assert not views[1].flags.writeable
    moved = w.poses.copy()
    moved[0, :, 3] += 0.05
    e2 = np.array(plan.linearize(moved, copy=False)[0])
    assert np.array_equal(views[0], e2) and not np.array_equal(e2, ref[0])


@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_lane_kernels_mixed_levels_ragged_and_nonfinite(G, ctx, layout):
    """One batch whose target maps have 3, 1 and 2 levels (absent levels read an empty record
    or probe an empty table), sources of 1, 37, and 130 * 64 + 5 points (ragged tiles, lanes
    past the end), a source point at NaN and one at 1e30 (misses), against the oracle, with
    the per-lane kernel of the layout and with the general kernel."""
    w = synth.corridor(n_kf=3, n_cur=9000, kf_range=(6000, 9000))
    dev = torch.device("cuda")
    res_of = {1: [0.5, 1.0, 2.0], 2: [1.0], 3: [0.5, 1.0]}
    gframes, oframes, gmaps, omaps = [], [], [], []
    for i, p in enumerate(w.points):
        p = np.asarray(p, np.float32).copy()
        if i == 0:
            p = p[:130 * 64 + 5]
            p[7] = np.nan
            p[8] = 1e30
        p4 = G.to_pts4(p, device=dev)
        good = torch.isfinite(p4).all(1) & (p4.abs() < 1e20).all(1)
        cov = torch.zeros((len(p4), 6), dtype=torch.float32, device=dev)
        cg, _ = G.estimate_covariances(ctx, p4[good].contiguous())
        cov[good] = cg
        cov[~good] = torch.tensor([1, 0, 0, 1, 0, 1], dtype=torch.float32, device=dev)
        gframes.append(G.FrameData(p4, cov))
        oframes.append(O.Frame(p4.cpu().numpy(), cov.cpu().numpy()))
        gmaps.append(G.VoxelMap(ctx, p4, cov, res_of[i], layout=layout) if i in res_of else None)
        omaps.append(O.VMap(oframes[i].pts4, oframes[i].cov6, res_of[i]) if i in res_of else None)
    # small sources: single points and a 37-point prefix of frame 0
    for n in (1, 37):
        gframes.append(G.FrameData(gframes[0].pts4[:n].clone(), gframes[0].cov6[:n].clone()))
        oframes.append(O.Frame(oframes[0].pts4[:n].copy(), oframes[0].cov6[:n].copy()))
        gmaps.append(None)
        omaps.append(None)
    poses = np.concatenate([w.poses, w.poses[:1], w.poses[:1]])
    pairs = np.array([[0, 1], [0, 2], [0, 3], [4, 1], [5, 3], [5, 2], [1, 2], [3, 1]], np.int32)
    assert all(gmaps[t].is_dense(l) == (layout == "dense") for t in (1, 2, 3) for l in range(len(res_of[t])))
    ref = O.linearize(oframes, omaps, pairs, poses, want_comp=True)
    for kernel in (layout, "general"):
        for block, ppt in ((128, 64), (256, 1), (128, 5)):
            res = G.linearize(ctx, gframes, gmaps, pairs, poses, kernel=kernel, block=block, pts_per_thread=ppt)
            from gpu_helpers import numpy_of, rel_errors
            e, H, b, inl = [numpy_of(x) for x in res]
            assert np.array_equal(inl, ref["inliers"])
            ok = ref["e"] > 0
            ee, eH, eb = rel_errors(e[ok], H[ok], b[ok], {k: v[ok] for k, v in ref.items()})
            assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL, (kernel, block, ppt)


@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_four_level_maps(G, ctx, layout):
    """Maps of four levels (0.25 / 0.5 / 1 / 2 m; the kernels' largest level count): the
    per-lane and general linearization, their correspondence ids, and the gradient (the
    pipelined per-lane kernel) against the oracle, with surface validation."""
    from gpu_helpers import rel_errors
    w = synth.corridor(n_kf=3, n_cur=8000, kf_range=(5000, 7000), weights=True)
    w.resolutions = [0.25, 0.5, 1.0, 2.0]
    from gpu_helpers import Prepared
    P = Prepared(ctx, w, layout=layout)
    assert all(P.gmaps[t].levels == 4 for t in set(int(t) for t in w.pairs[:, 1]))
    ref = P.oracle(validate=True, want_ids=True)
    for kernel in ("auto", "general"):
        plan = G.Plan(ctx, P.gframes, P.gmaps, w.pairs, kernel=kernel, validate_surface=True)
        e, H, b, inl = [np.array(x) for x in plan.linearize(w.poses)]
        assert np.array_equal(inl, ref["inliers"])
        ee, eH, eb = rel_errors(e, H, b, ref)
        assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL, (kernel, ee.max(), eH.max(), eb.max())
        ids, _ = plan.correspondence_ids(w.poses)
        assert np.array_equal(ids.cpu().numpy(), ref["ids"])
        if kernel == "auto":
            assert plan.opts()["kernel"] == layout
            dxi, dmu, dw = plan.backward(w.poses)
            odxi, odmu, odw = O.gradient(P.oframes, P.omaps, w.pairs, w.poses, validate=True)
            assert np.linalg.norm(dxi.cpu().numpy() - odxi) <= TOL * np.linalg.norm(odxi)
            odmu_all = np.concatenate(odmu)
            assert np.linalg.norm(dmu.cpu().numpy() - odmu_all) <= TOL * np.linalg.norm(odmu_all)
        plan.close()


@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_resolutions_not_doubling_run_the_general_kernel(G, ctx, layout):
    """The per-lane kernels take a coarser level's key as the level-0 key shifted right, which
    is exact only when the resolutions double per level.  Maps of 0.5 / 0.75 / 1.6 m run the
    general kernel (which forms every level's key by its own product), forcing a per-lane
    kernel is refused, and the result matches the oracle, correspondence ids included."""
    from gpu_helpers import Prepared
    w = synth.corridor(n_kf=3, n_cur=8000, kf_range=(5000, 7000))
    w.resolutions = [0.5, 0.75, 1.6]
    P = Prepared(ctx, w, layout=layout)
    ref = P.oracle(validate=True, want_ids=True)
    plan = G.Plan(ctx, P.gframes, P.gmaps, w.pairs, validate_surface=True)
    assert plan.opts()["kernel"] == "general"
    _check(plan.linearize(w.poses), ref)
    ids, _ = plan.correspondence_ids(w.poses)
    assert np.array_equal(ids.cpu().numpy(), ref["ids"])
    plan.close()
    with pytest.raises(G.GlimError, match="EINVAL"):
        G.linearize(ctx, P.gframes, P.gmaps, w.pairs, w.poses, kernel=layout)


@pytest.mark.parametrize("validate", [False, True])
def test_hash_kernel_and_general_kernel_on_hash_maps(G, ctx, room, validate):
    """Hash-table maps: the per-lane hash kernel (chosen automatically) and the general kernel
    match the oracle across accumulation modes and launch shapes; each per-lane kernel is
    refused on the other layout, and a batch mixing layouts runs on the general kernel."""
    g = room.gframes[1]
    hm = G.VoxelMap(ctx, g.pts4, g.cov6, room.w.resolutions, layout="hash")
    ref = room.oracle(validate=validate)
    for kernel in ("hash", "general"):
        for acc in (G.ACC_FP32, G.ACC_KAHAN, G.ACC_FP64):
            for persistent, block, ppt in ((1, 128, 64), (2, 256, 3)):
                _check(G.linearize(ctx, room.gframes, [None, hm], room.w.pairs, room.w.poses, kernel=kernel,
                                   validate_surface=validate, accum_mode=acc, persistent=persistent, block=block,
                                   pts_per_thread=ppt), ref)
    assert G.Plan(ctx, room.gframes, [None, hm], room.w.pairs).opts()["kernel"] == "hash"
    with pytest.raises(G.GlimError, match="EINVAL"):
        G.linearize(ctx, room.gframes, [None, hm], room.w.pairs, room.w.poses, kernel="dense")
    with pytest.raises(G.GlimError, match="EINVAL"):
        G.linearize(ctx, room.gframes, room.gmaps, room.w.pairs, room.w.poses, kernel="hash")
    # one dense and one hash target in the same batch
    pairs = np.array([[0, 1], [0, 2]], np.int32)
    frames = room.gframes + [room.gframes[1]]
    poses = np.concatenate([room.w.poses, room.w.poses[1:2]])
    plan = G.Plan(ctx, frames, [None, room.gmaps[1], hm], pairs)
    assert plan.opts()["kernel"] == "general"
    e, H, b, inl = plan.linearize(poses)
    for q in range(2):
        _check((e[q:q + 1], H[q:q + 1], b[q:q + 1], inl[q:q + 1]), room.oracle())


def test_invalid_arguments(G, ctx, room):
    with pytest.raises(G.GlimError, match="EINVAL"):
        G.linearize(ctx, room.gframes, room.gmaps, [[0, 1]], room.w.poses, block=96)
    with pytest.raises(ValueError):
        G.linearize(ctx, room.gframes, room.gmaps, [[0, 0]], room.w.poses)  # frame 0 has no voxelmap
    plan = G.Plan(ctx, room.gframes, room.gmaps, room.w.pairs)
    for frame, iters in ((-1, 2), (len(room.gframes), 2), (0, 0)):
        with pytest.raises(G.GlimError, match="EINVAL"):
            plan.gauss_newton(room.w.poses, frame, iters)
    plan.close()


# ---------------------------------------------------------------------------- covariances
def test_covariances_match_bruteforce_oracle(G, ctx):
    w = synth.corridor(n_cur=6000, kf_range=(5000, 5001), n_kf=1)
    for pts in w.points:
        p4 = G.to_pts4(pts, device="cuda")
        cov, nrm = G.estimate_covariances(ctx, p4, k=10)
        c64, n64, _, tie = O.estimate_covariances(pts, k=10)
        cov, nrm = cov.cpu().numpy().astype(np.float64), nrm.cpu().numpy().astype(np.float64)
        # points whose two smallest eigenvalues are within 1e-4 of the largest have no stable
        # normal; they are left out of the comparison and must stay rare (none in these frames)
        assert tie.sum() <= 0.001 * len(pts), int(tie.sum())
        ok = ~tie
        Cg = cov[:, [0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(-1, 3, 3)
        Co = c64[:, [0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(-1, 3, 3)
        rel = np.linalg.norm((Cg - Co).reshape(len(Cg), -1), axis=1) / np.linalg.norm(Co.reshape(len(Co), -1), axis=1)
        assert rel[ok].max() <= 1e-4
        assert np.abs(nrm[ok] - n64[ok]).max() <= 1e-4
        # raw covariance mode
        cov0, _ = G.estimate_covariances(ctx, p4, k=7, reg_mode=0, eps=1e-6)
        c0, _, _, _ = O.estimate_covariances(pts, k=7, reg_mode=0, eps=1e-6)
        np.testing.assert_allclose(cov0.cpu().numpy(), c0, rtol=1e-4, atol=1e-6 * np.abs(c0).max())


def test_covariances_small_cloud_bruteforce_path(G, ctx):
    pts = synth.box_room(n_src=300, n_tgt=300).points[0]
    cov, _ = G.estimate_covariances(ctx, G.to_pts4(pts, device="cuda"), k=5, reg_mode=0, eps=0.0)
    c0, _, _, _ = O.estimate_covariances(pts, k=5, reg_mode=0, eps=0.0)
    np.testing.assert_allclose(cov.cpu().numpy(), c0, rtol=1e-4, atol=1e-7 * np.abs(c0).max())


# ---------------------------------------------------------------------------- gradient
@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("layout", ["auto", "hash"])
def test_backward_matches_oracle_gradient(G, ctx, full, layout):
    from gpu_helpers import Prepared
    P = Prepared(ctx, synth.corridor(n_cur=4000, kf_range=(3000, 5000), n_kf=3, weights=True), layout=layout)
    assert all(P.gmaps[t].is_dense(0) == (layout == "auto") for t in set(int(t) for t in P.w.pairs[:, 1]))
    w = P.w
    dxi, dmu, dw = G.backward(ctx, P.gframes, P.gmaps, w.pairs, w.poses, omega_grad_full=full)
    odxi, odmu, odw = O.gradient(P.oframes, P.omaps, w.pairs, w.poses, omega_grad_full=full)
    dxi = dxi.cpu().numpy()
    assert np.linalg.norm(dxi - odxi) <= 1e-4 * np.linalg.norm(odxi)
    odmu_all = np.concatenate(odmu)
    odw_all = np.concatenate(odw)
    assert np.linalg.norm(dmu.cpu().numpy() - odmu_all) <= 1e-4 * np.linalg.norm(odmu_all)
    assert np.linalg.norm(dw.cpu().numpy() - odw_all) <= 1e-4 * np.linalg.norm(odw_all)


@pytest.mark.parametrize("full,n_kf,n_cur", [(True, 4, 6000), (False, 4, 6000), (True, 18, 1_300_000)])
def test_backward_pipelined_and_general_kernels_agree(G, ctx, full, n_kf, n_cur):
    """The gradient pass of a batch whose target maps are all dense grids, or all hashed, runs
    the pipelined per-lane kernel; a batch that mixes the layouts runs the general kernel.  On
    the same voxels (the maps of one batch built in both layouts) the three give the same
    gradient up to FP32 rounding, with three levels and surface validation.  With 18 keyframes
    and a 1.3M-point current frame the batch has enough tiles for one group per frame, which
    the 16-pair limit of a group splits in two."""
    from gpu_helpers import Prepared
    w = synth.corridor(n_cur=n_cur, kf_range=(3000, 5000), n_kf=n_kf, weights=True)
    w.resolutions = [0.5, 1.0, 2.0]
    P = Prepared(ctx, w)
    targets = sorted(set(int(t) for t in w.pairs[:, 1]))
    layouts = {"dense": ["dense"] * len(targets), "hash": ["hash"] * len(targets),
               "mixed": ["dense" if i % 2 else "hash" for i in range(len(targets))]}
    res = {}
    for name, lay in layouts.items():
        maps = [None] * len(w.points)
        for t, l in zip(targets, lay):
            maps[t] = G.VoxelMap(ctx, P.gframes[t].pts4, P.gframes[t].cov6, w.resolutions, layout=l)
        plan = G.Plan(ctx, P.gframes, maps, w.pairs, validate_surface=True)
        res[name] = [x.double().cpu().numpy() for x in plan.backward(w.poses, omega_grad_full=full)]
        plan.close()
    for name in ("dense", "hash"):
        for a, b in zip(res[name], res["mixed"]):
            assert np.linalg.norm(a - b) <= 2e-6 * np.linalg.norm(b), (name, np.linalg.norm(a - b) / np.linalg.norm(b))
    for a, b in zip(res["dense"], res["hash"]):  # same kernel code, same lookups: same bits
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------- Gauss-Newton
def test_gn_solve_matches_oracle_and_flags_singular(G, ctx, room):
    res = G.linearize(ctx, room.gframes, room.gmaps, room.w.pairs, room.w.poses, out="cuda")
    xi, st = G.gn_solve(ctx, res[1], res[2], dim=6)
    H, b = res[1].cpu().numpy()[0], res[2].cpu().numpy()[0]
    np.testing.assert_allclose(xi.cpu().numpy()[0], O.gn_solve(H[:6, :6], b[:6]), rtol=1e-9, atol=1e-12)
    assert st.cpu().numpy()[0] == 0
    # the full 12 x 12 binary H has the 6-dimensional gauge null space: not positive definite
    _, st12 = G.gn_solve(ctx, res[1], res[2], dim=12)
    assert st12.cpu().numpy()[0] == -6


def test_gauss_newton_recovers_pose(G, ctx):
    from gpu_helpers import Prepared
    P = Prepared(ctx, synth.box_room(sigma=0.0))
    poses = P.w.poses.copy()
    plan = G.Plan(ctx, P.gframes, P.gmaps, P.w.pairs)
    for _ in range(10):
        e, H, b, _ = plan.linearize(poses)
        xi, st = G.gn_solve(ctx, torch.as_tensor(H, device="cuda"), torch.as_tensor(b, device="cuda"), dim=6)
        poses[0] = O.retract(poses[0], xi.cpu().numpy()[0])
    D = O.compose(O.inverse(P.w.poses_true[0]), poses[0])
    ang = math.degrees(math.acos(min(1.0, (np.trace(D[:, :3]) - 1) / 2)))
    assert ang < 0.05 and np.linalg.norm(D[:, 3]) < 0.005
    # parity at the optimum, where b is the difference of large cancelling terms: the b error
    # is taken against the cancellation-free scale sum |w J^T Omega d|
    from gpu_helpers import rel_errors
    e, H, b, inl = plan.linearize(poses)
    ref = O.linearize(P.oframes, P.omaps, P.w.pairs, poses, want_comp=True)
    assert np.linalg.norm(ref["b"][:, :6]) < 1e-2 * ref["b_scale"].max()
    ee, eH, eb = rel_errors(e, H, b, ref)
    assert (np.asarray(inl) == ref["inliers"]).all()
    assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL, (ee.max(), eH.max(), eb.max())


def test_corridor_parity_after_gauss_newton(G, ctx, corridor):
    """The odometry window after Gauss-Newton on the current frame (the keyframes fixed): the
    frame's 6 x 6 system is the sum of the source blocks of its 10 binary factors, solved on
    the device; at the optimum, where b is the difference of large cancelling terms, the batch
    still matches the oracle (P7, b against the cancellation-free scale)."""
    from gpu_helpers import rel_errors
    P = corridor
    w = P.w
    assert (w.pairs[:, 0] == 0).all()
    plan = G.Plan(ctx, P.gframes, P.gmaps, w.pairs)
    poses = w.poses.copy()
    e0 = None
    for _ in range(6):
        e, H, b, _ = plan.linearize(poses)
        e0 = e.sum() if e0 is None else e0
        Hs = torch.as_tensor(H.sum(axis=0)[None], device="cuda")
        bs = torch.as_tensor(b.sum(axis=0)[None], device="cuda")
        xi, st = G.gn_solve(ctx, Hs, bs, dim=6)
        assert st.cpu().numpy()[0] == 0
        poses[0] = O.retract(poses[0], xi.cpu().numpy()[0])
    e, H, b, inl = plan.linearize(poses)
    assert e.sum() < e0
    ref = P.oracle(poses=poses)
    ref0 = P.oracle()
    # the frame's gradient has shrunk (its factors' source blocks largely cancel now)
    assert np.linalg.norm(ref["b"][:, :6].sum(axis=0)) < 0.1 * np.linalg.norm(ref0["b"][:, :6].sum(axis=0))
    ee, eH, eb = rel_errors(e, H, b, ref)
    assert np.array_equal(np.asarray(inl), ref["inliers"])
    assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL, (ee.max(), eH.max(), eb.max())


def test_gauss_newton_on_the_device_matches_the_host_loop(G, ctx, corridor):
    """glim_plan_gauss_newton (linearize, per-frame 6 x 6 system, Cholesky, T <- T Exp(xi),
    all on the device) against the same iterations driven from the host (device Cholesky,
    pose update in FP64 on the host): the box room's unary factor and the odometry window's
    current frame against 10 fixed keyframes.  The poses agree to FP64 rounding (the update's
    sine and cosine come from different libraries), the costs to 1e-9; a frame of no pair has
    a zero system and takes no step."""
    from gpu_helpers import Prepared
    P = Prepared(ctx, synth.box_room(sigma=0.0))
    for prep, iters in ((P, 10), (corridor, 6)):
        w = prep.w
        plan = G.Plan(ctx, prep.gframes, prep.gmaps, w.pairs)
        poses = w.poses.copy()
        costs = []
        for _ in range(iters):
            e, H, b, _ = plan.linearize(poses)
            costs.append(float(np.sum(e)))
            Hs = torch.as_tensor(H[w.pairs[:, 0] == 0].sum(axis=0)[None], device="cuda")
            bs = torch.as_tensor(b[w.pairs[:, 0] == 0].sum(axis=0)[None], device="cuda")
            xi, st = G.gn_solve(ctx, Hs, bs, dim=6)
            poses[0] = O.retract(poses[0], xi.cpu().numpy()[0])
        out, cost, status = plan.gauss_newton(w.poses, 0, iters)
        assert status == 0
        out2, cost2, _ = plan.gauss_newton(w.poses, 0, iters)  # the cached loop, replayed
        assert np.array_equal(out2, out) and np.array_equal(cost2, cost)
        assert np.abs(out - poses).max() <= 1e-9, np.abs(out - poses).max()
        assert np.array_equal(out[1:], w.poses[1:])
        np.testing.assert_allclose(cost, costs, rtol=1e-9)
        # the plan's device poses are the final ones: a gradient at those poses uploads nothing
        # and equals the one-shot gradient there
        g_plan = plan.backward(out)
        g_one = G.backward(ctx, prep.gframes, prep.gmaps, w.pairs, out)
        for a, b_ in zip(g_plan, g_one):
            assert torch.equal(a, b_)
        plan.close()
    # a frame that is in no pair: its system is zero, no step is taken
    w = P.w
    frames = P.gframes + [P.gframes[0]]
    plan = G.Plan(ctx, frames, P.gmaps + [None], w.pairs)
    poses = np.concatenate([w.poses, w.poses[:1]])
    out, cost, status = plan.gauss_newton(poses, 2, 2)
    assert status == -6 and np.array_equal(out, poses)  # GLIM_ENOTPD
    plan.close()


# ---------------------------------------------------------------------------- overlap
def test_overlap_matches_oracle(G, ctx, corridor):
    w = corridor.w
    for level in range(len(w.resolutions)):
        ov = G.overlap(ctx, corridor.gframes, corridor.gmaps, w.pairs, w.poses, level=level).cpu().numpy()
        for p, (s, t) in enumerate(w.pairs):
            ref = O.overlap(corridor.oframes[s], corridor.omaps[t], w.poses[s], w.poses[t], level=level)
            assert ov[p] == pytest.approx(ref, abs=0)


# ---------------------------------------------------------------------------- point order
def test_spatial_order_is_a_stable_morton_sort(G, ctx):
    pts = synth.corridor(n_cur=5000, kf_range=(100, 101), n_kf=1).points[0]
    p4 = G.to_pts4(pts, device="cuda")
    perm = G.spatial_order(ctx, p4, 0.5).cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(len(pts)))
    k = np.floor(pts.astype(np.float32) * np.float32(2.0)).astype(np.int64) + (1 << 20)

    def spread(v):
        out = np.zeros_like(v)
        for b in range(21):
            out |= ((v >> b) & 1) << (3 * b)
        return out

    code = (spread(k[:, 0]) << 2) | (spread(k[:, 1]) << 1) | spread(k[:, 2])
    c = code[perm]
    assert (np.diff(c) >= 0).all()
    ties = np.diff(c) == 0
    assert (np.diff(perm)[ties] > 0).all()  # stable within a cell


def test_linearize_independent_of_point_order(G, ctx, corridor):
    """Reordering the source points changes e, H, b only by rounding."""
    ref = corridor.oracle()
    src = corridor.gframes[0]
    perm = G.spatial_order(ctx, src.pts4, 0.5)
    fr = [G.FrameData(src.pts4[perm].contiguous(), src.cov6[perm].contiguous(),
                      src.normal3[perm].contiguous())] + corridor.gframes[1:]
    _check(G.linearize(ctx, fr, corridor.gmaps, corridor.w.pairs, corridor.w.poses), ref)


# ---------------------------------------------------------------------------- autograd
@pytest.mark.parametrize("full", [True, False])
def test_autograd_function_against_fd(G, ctx, full):
    """GlimFactorFn on an odometry-window batch with per-point weights: the backward pass
    matches central finite differences (h = 1e-6, FP64 oracle energy with the correspondences
    and, for the frozen mode, Omega held at the linearization point) on a 500-point subset,
    and the oracle's analytic gradient on all points."""
    from gpu_helpers import Prepared
    from paper_2407_10344_b300.autograd import FactorProblem, retract
    P = Prepared(ctx, synth.corridor(n_cur=4000, kf_range=(3000, 5000), n_kf=3, weights=True))
    w = P.w
    prob = FactorProblem(ctx, P.gframes, P.gmaps, w.pairs, w.poses, omega_grad_full=full)
    pts, wts = prob.points()
    pts = pts.clone().requires_grad_(True)
    wts = wts.clone().requires_grad_(True)
    xi = torch.zeros((len(w.points), 6), dtype=torch.float64, device="cuda", requires_grad=True)
    E = prob.energy(xi, pts, wts)
    E.backward()
    ref = P.oracle(want_ids=True)
    assert abs(E.item() - ref["e"].sum()) <= 1e-4 * ref["e"].sum()
    # analytic oracle gradient
    odxi, odmu, odw = O.gradient(P.oframes, P.omaps, w.pairs, w.poses, omega_grad_full=full)
    gxi = xi.grad.cpu().numpy()
    assert np.linalg.norm(gxi - odxi) <= 1e-4 * np.linalg.norm(odxi)
    n0 = len(w.points[0])
    gmu = pts.grad.cpu().numpy()
    assert np.linalg.norm(gmu[:n0] - odmu[0]) <= 1e-4 * np.linalg.norm(odmu[0])
    assert np.linalg.norm(wts.grad.cpu().numpy()[:n0] - odw[0]) <= 1e-4 * np.linalg.norm(odw[0])
    # central FD of the FP64 energy (frozen correspondences) on pose increments of two frames
    ids = ref["ids"]

    def E_fd(x):
        poses = np.stack([retract(w.poses[f], x[6 * f:6 * f + 6]) for f in range(len(w.points))])
        return O.energy(P.oframes, P.omaps, w.pairs, poses, ids, omega_poses=None if full else w.poses).sum()

    h = 1e-6
    for f in (0, 2):
        for a in range(6):
            x = np.zeros(6 * len(w.points))
            x[6 * f + a] = h
            fd = (E_fd(x) - E_fd(-x)) / (2 * h)
            assert abs(fd - gxi[f, a]) <= 1e-4 * np.abs(gxi).max(), (f, a, fd, gxi[f, a])
    # FD of points and weights on a 500-point subset of the source frame: the terms of point k
    # depend only on point k, so each derivative is taken on a one-point frame with that
    # point's frozen correspondences
    sel = synth.Stream(7, "subset").integers(500, 0, n0)
    L = len(w.resolutions)
    ids_pp = ids.reshape(len(w.pairs), n0, L)
    grads = np.concatenate([gmu[:n0], wts.grad.cpu().numpy()[:n0, None]], 1)
    worst = 0.0
    for k in sel:
        one_ids = ids_pp[:, k, :].reshape(-1)
        for a in range(4):
            def Ep(hv):
                p = P.oframes[0].pts4[k:k + 1].copy()
                p[0, a] = np.float32(np.float64(p[0, a]) + hv)
                fr = [O.Frame(p, P.oframes[0].cov6[k:k + 1], P.oframes[0].normal3[k:k + 1])] + P.oframes[1:]
                return O.energy(fr, P.omaps, w.pairs, w.poses, one_ids).sum()
            hv = 1e-3 if a < 3 else 1e-2
            fd = (Ep(hv) - Ep(-hv)) / (2 * hv)
            worst = max(worst, abs(fd - grads[k, a]) / max(1.0, abs(grads[k, a])))
    assert worst <= 2e-3


@pytest.mark.parametrize("full", [False, True])
def test_plan_backward_equals_one_shot_and_reuses_scratch(G, ctx, full):
    """glim_plan_backward on a plan gives the one-shot glim_backward's gradient bit for bit,
    again on a second call with the kept scratch, and on a plan with other linearization tiles
    (the gradient pass has its own work list)."""
    from gpu_helpers import Prepared
    P = Prepared(ctx, synth.corridor(n_cur=4000, kf_range=(3000, 5000), n_kf=3, weights=True))
    w = P.w
    one = G.backward(ctx, P.gframes, P.gmaps, w.pairs, w.poses, omega_grad_full=full)
    plan = G.Plan(ctx, P.gframes, P.gmaps, w.pairs, block=256, pts_per_thread=1)
    for _ in range(2):  # the second call finds the poses on the device and uploads nothing
        got = plan.backward(w.poses, omega_grad_full=full)
        for a, b in zip(one, got):
            assert torch.equal(a, b)
    # a linearization at other poses, then gradients at the first poses and at the other ones:
    # each call uploads the poses it was given when the device holds different ones
    poses2 = w.poses.copy()
    poses2[0, :, 3] += np.array([0.05, -0.03, 0.02])
    one2 = G.backward(ctx, P.gframes, P.gmaps, w.pairs, poses2, omega_grad_full=full)
    plan.linearize(poses2)
    for poses, ref in ((w.poses, one), (poses2, one2), (poses2, one2)):
        got = plan.backward(poses, omega_grad_full=full)
        for a, b in zip(ref, got):
            assert torch.equal(a, b)
    assert not torch.equal(one[0], one2[0])
    other = G.Plan(ctx, P.gframes, P.gmaps, w.pairs, block=128, pts_per_thread=16)
    for a, b in zip(one, other.backward(w.poses, omega_grad_full=full)):
        assert torch.equal(a, b)


def test_autograd_interleaved_evaluations(G, ctx):
    """Two evaluations at different points before the first one's backward: the gradient is
    the first evaluation's (its gradient pass read the shared point buffer before the second
    evaluation rewrote it)."""
    from gpu_helpers import Prepared
    from paper_2407_10344_b300.autograd import FactorProblem
    P = Prepared(ctx, synth.corridor(n_cur=4000, kf_range=(3000, 5000), n_kf=3, weights=True))
    w = P.w

    def grads(prob, pts, wts, second=None):
        p1 = pts.clone().requires_grad_(True)
        w1 = wts.clone().requires_grad_(True)
        xi = torch.zeros((len(w.points), 6), dtype=torch.float64, device="cuda", requires_grad=True)
        E = prob.energy(xi, p1, w1)
        if second is not None:
            prob.energy(xi.detach(), second, wts)
        E.backward()
        return E.item(), xi.grad.clone(), p1.grad.clone(), w1.grad.clone()

    prob = FactorProblem(ctx, P.gframes, P.gmaps, w.pairs, w.poses)
    pts, wts = prob.points()
    ref = grads(FactorProblem(ctx, P.gframes, P.gmaps, w.pairs, w.poses), pts, wts)
    got = grads(prob, pts, wts, second=pts + 0.05)
    assert got[0] == ref[0]
    for a, b in zip(got[1:], ref[1:]):
        assert torch.equal(a, b)


# ---------------------------------------------------------------------------- small factor graph
def test_graph_step_assembly_and_solve_against_oracle(G, ctx):
    """glim_graph_step (device assembly + damped FP64 Cholesky) against the oracle's
    orc_graph_step on a random graph, for a fixed frame and plain GN, a fixed frame with LM
    damping, and no fixed frame with damping."""
    s = synth.Stream(77, "graph")
    n, P = 7, 18
    pairs = []
    while len(pairs) < P:
        a, b_ = s.integers(2, 0, n)
        if a != b_:
            pairs.append((int(a), int(b_)))
    Hs, bs = [], []
    for _ in range(P):
        J = s.normal(12 * 40).reshape(40, 12)
        Hs.append(J.T @ J)
        bs.append(s.normal(12))
    H = torch.as_tensor(np.stack(Hs), device="cuda")
    b = torch.as_tensor(np.stack(bs), device="cuda")
    for fixed, lam in ((0, 0.0), (3, 1e-3), (-1, 0.5)):
        xi, Hg, bg = G.graph_step(ctx, pairs, n, H, b, fixed_frame=fixed, lam=lam, want_system=True)
        oxi, oHg, obg = O.graph_step(pairs, n, Hs, bs, fixed=fixed, lam=lam)
        np.testing.assert_allclose(Hg.cpu().numpy(), oHg, rtol=1e-14, atol=1e-12)
        np.testing.assert_allclose(bg.cpu().numpy(), obg, rtol=1e-14, atol=1e-12)
        np.testing.assert_allclose(xi.cpu().numpy(), oxi, rtol=1e-9, atol=1e-9 * np.abs(oxi).max())
    # relative-pose factors alone leave the gauge free: not positive definite without a fixed frame
    with pytest.raises(G.GlimError, match="ENOTPD"):
        gh = torch.zeros((1, 144), dtype=torch.float64, device="cuda")
        G.graph_step(ctx, [(0, 1)], 2, gh.view(1, 12, 12), torch.zeros((1, 12), dtype=torch.float64, device="cuda"),
                     fixed_frame=-1)


def test_local_mapping_all_to_all_converges(G, ctx):
    """All-to-all factors between 5 corridor keyframes with perturbed poses (frame 0 fixed):
    device Gauss-Newton steps of the whole graph recover the true relative poses."""
    from gpu_helpers import Prepared
    from paper_2407_10344_b300.autograd import retract
    w = synth.corridor(n_kf=5, n_cur=20000, kf_range=(20000, 25000))
    kf = list(range(1, 6))
    pairs = np.array([[i, j] for i in kf for j in kf if i != j], np.int32)
    w.pairs = pairs
    P = Prepared(ctx, w)
    s = synth.Stream(5, "lm")
    poses = w.poses_true.copy()
    for f in kf[1:]:
        poses[f] = synth.perturb_pose(poses[f], 0.5, 0.05, s)
    plan = G.Plan(ctx, P.gframes, P.gmaps, pairs)
    idx = {f: i for i, f in enumerate(kf)}
    local_pairs = [(idx[a], idx[b_]) for a, b_ in pairs]
    costs = []
    for _ in range(8):
        e, H, b, _ = plan.linearize(poses)
        costs.append(e.sum())
        xi = G.graph_step(ctx, local_pairs, len(kf), torch.as_tensor(H, device="cuda"),
                          torch.as_tensor(b, device="cuda"), fixed_frame=0).cpu().numpy()
        for f in kf:
            poses[f] = retract(poses[f], xi[idx[f]])
    assert costs[-1] < costs[0]
    for f in kf[1:]:
        D = O.compose(O.inverse(O.compose(O.inverse(w.poses_true[kf[0]]), w.poses_true[f])),
                      O.compose(O.inverse(poses[kf[0]]), poses[f]))
        ang = math.degrees(math.acos(min(1.0, (np.trace(D[:, :3]) - 1) / 2)))
        assert ang < 0.05 and np.linalg.norm(D[:, 3]) < 0.01, (f, ang, np.linalg.norm(D[:, 3]))
    # every factor of the converged graph agrees with the oracle at the final poses
    from gpu_helpers import rel_errors
    e, H, b, inl = plan.linearize(poses)
    ref = O.linearize(P.oframes, P.omaps, pairs, poses, want_comp=True)
    ee, eH, eb = rel_errors(e, H, b, ref)
    assert (np.asarray(inl) == ref["inliers"]).all()
    assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL, (ee.max(), eH.max(), eb.max())


# ---------------------------------------------------------------------------- FMA rates
def test_fma_peaks_are_plausible(G, ctx):
    """The FMA-chain kernels give the FP32 roofline's denominator and the FP64 rate: both
    positive and below the nominal rate of the device (128 FP32 lanes per SM at the maximum
    clock), FP64 far below FP32."""
    fp32 = ctx.fp32_fma_peak(iters=1024)
    fp64 = ctx.fp64_fma_peak(iters=16)
    nominal = ctx.num_sms * 128 * 2 * 2.1e9 / 1e12
    assert 0.3 * nominal < fp32 <= 1.02 * nominal, (fp32, nominal)
    assert 0.0 < fp64 < 0.5 * fp32, (fp64, fp32)
    with pytest.raises(G.GlimError, match="EINVAL"):
        ctx.fp64_fma_peak(iters=0)


def test_process_exit_with_open_objects():
    """A script that ends with a context, voxelmaps and a plan (with pinned output views)
    still open exits cleanly: the binding releases them before the interpreter tears down."""
    import subprocess
    import sys
    import os
    code = (
        "import numpy as np, torch, synth\n"
        "import paper_2407_10344_b300 as G\n"
        "from gpu_helpers import Prepared\n"
        "ctx = G.Context(0)\n"
        "P = Prepared(ctx, synth.box_room())\n"
        "plan = G.Plan(ctx, P.gframes, P.gmaps, P.w.pairs)\n"
        "e, H, b, inl = plan.linearize(P.w.poses, copy=False)\n"
        "print(float(e[0]) > 0)\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([root, os.path.join(root, "tests")]))
    r = subprocess.run([sys.executable, "-X", "faulthandler", "-c", code], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    assert r.stdout.strip().endswith("True")


def test_plan_pose_packing_bits(G, ctx, corridor):
    """The plan forms every pair's relative pose on the device from the uploaded frame poses:
    T_rel = T_t^-1 T_s in FP64 with each product and sum rounded on its own, in a fixed order,
    then rounded to FP32 with the target viewpoint v = -R^T t.  numpy's float64 arithmetic in
    the same order gives the same bits."""
    w = corridor.w
    s = synth.Stream(21, "pose-bits")
    poses = np.stack([synth.perturb_pose(T, 3.0, 0.4, s) for T in w.poses])
    plan = G.Plan(ctx, corridor.gframes, corridor.gmaps, w.pairs)
    plan.set_poses(poses)
    T, p32 = plan.relative_poses()
    for q, (si, ti) in enumerate(w.pairs):
        S, Tt = poses[si], poses[ti]
        R = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                v = 0.0
                for k in range(3):
                    v = v + Tt[k, i] * S[k, j]
                R[i, j] = v
        dt = S[:, 3] - Tt[:, 3]
        tr = np.array([(Tt[0, i] * dt[0] + Tt[1, i] * dt[1]) + Tt[2, i] * dt[2] for i in range(3)])
        assert np.array_equal(T[q, :, :3], R) and np.array_equal(T[q, :, 3], tr), q
        v = np.zeros(3)
        for i in range(3):
            acc = 0.0
            for k in range(3):
                acc = acc + R[k, i] * tr[k]
            v[i] = -acc
        want = np.concatenate([R.reshape(-1), tr, v, [0.0]]).astype(np.float32)
        assert np.array_equal(p32[q], want), q
    # the packed poses are the ones linearized: the plan equals the one-shot call, whose
    # relative poses are formed on the host
    o = plan.opts()
    e1, H1, b1, i1 = plan.linearize(poses)
    e2, H2, b2, i2 = G.linearize(ctx, corridor.gframes, corridor.gmaps, w.pairs, poses, block=o["block"],
                                 pts_per_thread=o["pts_per_thread"], accum_mode=o["accum_mode"])
    for a, b_ in ((e1, e2), (H1, H2), (b1, b2), (i1, i2)):
        assert np.array_equal(np.asarray(a), np.asarray(b_))


# ---------------------------------------------------------------------------- key range edge
@pytest.mark.parametrize("layout", ["dense", "hash"])
def test_keys_at_the_edge_of_the_key_range(G, ctx, layout):
    """Voxels at the largest and smallest valid keys (2^20 - 1 and -2^20 at 0.5 m, and their
    level-1 keys at 1 m) and source points one key beyond them: the points inside hit their
    voxels, the ones beyond miss, with ids bit-exact and e, H, b within the tolerance, at the
    identity and after a shift that carries points across the boundary.

    Near |x| = 2^20 r a binary32 coordinate has a spacing of r / 8, so every coordinate, voxel
    mean and the shift are placed on multiples of 1/16 m: then the transform, the FP32 voxel
    means and the differences d are exact and only the residual arithmetic rounds."""
    res = [0.5, 1.0]
    edge = 2 ** 20

    def cluster(k0):  # 4 points symmetric about the centre of each voxel with x keys k0 - 1, k0
        out = []
        for kx in (k0 - 1, k0):
            for ky in (-1, 0):
                for kz in (-1, 0):
                    c = np.array([kx + 0.5, ky + 0.5, kz + 0.5]) * res[0]
                    for a in ([0.125, 0.0625, 0.0625], [0.0625, -0.125, 0.0625]):
                        out += [c + a, c - np.array(a)]
        return np.array(out)  # FP64

    beyond = np.array([[(edge + 0.5) * res[0], 0.125, 0.125], [(-edge - 0.5) * res[0], -0.1875, 0.3125]])
    src64 = np.concatenate([cluster(edge - 1), cluster(-edge + 1), beyond])
    src = src64.astype(np.float32)
    assert np.array_equal(src.astype(np.float64), src64)  # every coordinate is a binary32 value
    m = len(src) // 2 - 1
    tA, tB = src[:m], src[m:2 * m]
    n = len(src)

    def cov(k):
        return np.tile(np.array([0.01, 0, 0, 0.01, 0, 0.01], np.float32), (k, 1))

    pts = [src, tA, tB]
    of = [O.Frame(O.as_pts4(p), cov(len(p))) for p in pts]
    om = [None, O.VMap(of[1].pts4, of[1].cov6, res), O.VMap(of[2].pts4, of[2].cov6, res)]
    gf = [G.FrameData(torch.as_tensor(f.pts4, device="cuda"), torch.as_tensor(f.cov6, device="cuda")) for f in of]
    gm = [None] + [G.VoxelMap(ctx, gf[i].pts4, gf[i].cov6, res, layout=layout) for i in (1, 2)]
    for i in (1, 2):
        for l in range(2):
            assert gm[i].is_dense(l) == (layout == "dense")
            assert np.array_equal(gm[i].export(l)["keys"].cpu().numpy(), om[i].export(l)["keys"])
    assert om[1].export(0)["keys"][:, 0].max() == edge - 1 and om[2].export(0)["keys"][:, 0].min() == -edge
    pairs = np.array([[0, 1], [0, 2]], np.int32)
    for shift in (0.0, 0.3125):
        poses = np.stack([np.eye(3, 4)] * 3)
        poses[0, 0, 3] = shift
        ref = O.linearize(of, om, pairs, poses, want_ids=True, want_comp=True)
        got = G.linearize(ctx, gf, gm, pairs, poses, kernel="auto")
        _check(got, ref)
        gid = np.concatenate([G.correspondences(ctx, gf[0], gm[t], poses[0], poses[t]).cpu().numpy().reshape(-1)
                              for t in (1, 2)])
        assert np.array_equal(gid, ref["ids"])
        ids = gid.reshape(2, n, 2)
        if shift == 0.0:  # every point inside the range hits at both levels; the two beyond miss
            assert (ids[0, :m] >= 0).all() and (ids[1, m:2 * m] >= 0).all()
            assert (ids[:, n - 2:] < 0).all()
        else:  # the shift moves the last x-voxel of A past 2^20 - 1 at level 0
            assert (ids[0, :m, 0] < 0).any() and (ids[0, :m, 0] >= 0).any()


# ---------------------------------------------------------------------------- C-level guards
def test_plan_on_a_map_freed_through_the_c_abi_is_refused(G, ctx, corridor):
    """A plan whose target map was freed with glim_vmap_free (bypassing the Python binding's
    own guard) returns GLIM_EINVAL from its launch entry points instead of reading freed
    tables; a plan on live maps is unaffected, and the caller's current device is kept."""
    import ctypes as C
    w = corridor.w
    t = int(w.pairs[0, 1])
    g = corridor.gframes[t]
    vm = G.VoxelMap(ctx, g.pts4, g.cov6, w.resolutions)
    maps = list(corridor.gmaps)
    maps[t] = vm
    plan = G.Plan(ctx, corridor.gframes, maps, w.pairs)
    other = G.Plan(ctx, corridor.gframes, corridor.gmaps, w.pairs)
    plan.linearize(w.poses)
    ctx.lib.glim_vmap_free(vm.h)  # the C call alone: the binding does not see it
    poses = np.ascontiguousarray(w.poses.reshape(-1, 12))
    assert ctx.lib.glim_plan_launch(plan.h) == -1
    assert ctx.lib.glim_plan_set_poses(plan.h, poses.ctypes.data_as(C.c_void_p)) in (0, -1)
    assert ctx.lib.glim_plan_launch_timed(plan.h, 0) == -1
    e, H, b, inl = other.linearize(w.poses)
    assert np.isfinite(H).all() and (inl > 0).all()
    vm.h = None  # already freed
    plan.close()
    other.close()
    assert torch.cuda.current_device() == 0


def test_factor_records_and_symmetric_H(G, ctx, corridor):
    """Every linearization of a plan also writes one 92-double record per pair (e, the upper
    triangle of H, b, inliers): it equals the packing of the plan's own outputs bit for bit,
    H is exactly symmetric, and unpacking the records gives those outputs back; gathering the
    records of a split pair list (world of one) puts them back in pair order."""
    w = corridor.w
    plan = G.Plan(ctx, corridor.gframes, corridor.gmaps, w.pairs)
    e, H, b, inl = [np.array(x) for x in plan.linearize(w.poses)]
    rec = plan.device_records()
    assert rec.shape == (len(w.pairs), 92) and rec.is_cuda
    assert np.array_equal(H, np.transpose(H, (0, 2, 1)))
    assert np.array_equal(rec.cpu().numpy(), G.pack_records(e, H, b, inl))
    e2, H2, b2, inl2 = G.unpack_records(rec)
    assert np.array_equal(e2, e) and np.array_equal(H2, H) and np.array_equal(b2, b) and np.array_equal(inl2, inl)
    idx = np.arange(len(w.pairs))[::-1].copy()
    full = G.gather_records(rec[torch.as_tensor(idx, device=rec.device)], idx, len(w.pairs))
    assert torch.equal(full, rec)
    plan.close()
