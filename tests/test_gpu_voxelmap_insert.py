"""Incremental voxelmap insertion (a submap that grows as frames are merged into it,
Sec. V-A): a map built from a first chunk of points and grown by insertions must equal the
oracle's voxelmap of all points (keys and counts bit-exact, statistics to FP32 rounding), and
linearizing against it must match the oracle on the union.  Also: layout changes as the key
box grows, errors leave the map unchanged, plans made before an insertion refuse to run."""
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


def _assert_same_map(gm, om, levels):
    for l in range(levels):
        g = {k: v.cpu().numpy() for k, v in gm.export(l).items()}
        o = om.export(l)
        assert np.array_equal(g["keys"], o["keys"])
        assert np.array_equal(g["count"], o["count"])
        np.testing.assert_allclose(g["mean"], o["mean"], rtol=0, atol=2e-6 * max(1.0, np.abs(o["mean"]).max()))
        np.testing.assert_allclose(g["cov"], o["cov"], rtol=0, atol=2e-6 * np.abs(o["cov"]).max())


@pytest.mark.parametrize("layout", ["auto", "hash"])
def test_insert_equals_build_of_all_points(G, ctx, room, layout):
    g = room.gframes[1]
    n = g.n
    cuts = [0, n // 3, n // 3, n // 3 + 7, n]             # ragged chunks, one of them empty
    gm = G.VoxelMap(ctx, g.pts4[:cuts[1]].contiguous(), g.cov6[:cuts[1]].contiguous(), room.w.resolutions,
                    layout=layout)
    for a, b in zip(cuts[1:-1], cuts[2:]):
        gm.insert(g.pts4[a:b].contiguous(), g.cov6[a:b].contiguous(), layout=layout)
    _assert_same_map(gm, room.omaps[1], len(room.w.resolutions))
    full = G.VoxelMap(ctx, g.pts4, g.cov6, room.w.resolutions, layout=layout)
    for l in range(len(room.w.resolutions)):
        assert gm.is_dense(l) == full.is_dense(l)
        assert gm.info(l)["n_voxels"] == full.info(l)["n_voxels"]
    # linearization against the grown map matches the oracle on the union
    from gpu_helpers import numpy_of, rel_errors
    maps = list(room.gmaps)
    maps[1] = gm
    res = G.linearize(ctx, room.gframes, maps, room.w.pairs, room.w.poses)
    ref = room.oracle()
    e, H, b, inl = [numpy_of(x) for x in res]
    ee, eH, eb = rel_errors(e, H, b, ref)
    assert (inl == ref["inliers"]).all()
    assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL, (ee.max(), eH.max(), eb.max())


def test_submap_grows_from_frames_in_map_coordinates(G, ctx):
    """Keyframes transformed to the map frame and inserted one by one (the submap of Sec. V-A)
    equal the oracle's map of their concatenation."""
    w = synth.corridor(n_kf=4, n_cur=5000, kf_range=(8000, 12000))
    res = [0.5, 1.0]
    dev = torch.device("cuda", ctx.device)
    pts_all, cov_all = [], []
    gm = None
    for f in range(1, 5):
        T = np.asarray(w.poses_true[f], np.float64)
        p = w.points[f] @ T[:, :3].T + T[:, 3]
        p4 = G.to_pts4(p.astype(np.float32), device=dev)
        cov, _ = G.estimate_covariances(ctx, p4, k=10)
        pts_all.append(p4)
        cov_all.append(cov)
        if gm is None:
            gm = G.VoxelMap(ctx, p4, cov, res)
        else:
            gm.insert(p4, cov)
    P = torch.cat(pts_all).cpu().numpy()
    Cv = torch.cat(cov_all).cpu().numpy()
    _assert_same_map(gm, O.VMap(P, Cv, res), len(res))


def test_insert_layout_switch_errors_and_stale_plans(G, ctx, room):
    g = room.gframes[1]
    res = room.w.resolutions
    gm = G.VoxelMap(ctx, g.pts4, g.cov6, res)
    assert all(gm.is_dense(l) for l in range(len(res)))
    before = [{k: v.cpu().numpy() for k, v in gm.export(l).items()} for l in range(len(res))]

    def unchanged():
        for l in range(len(res)):
            now = {k: v.cpu().numpy() for k, v in gm.export(l).items()}
            for k in before[l]:
                assert np.array_equal(now[k], before[l][k])

    cov1 = torch.tensor([[0.01, 0, 0, 0.01, 0, 0.01]], dtype=torch.float32, device="cuda")
    # a key outside [-2^20, 2^20) and a non-finite covariance are rejected; the map is unchanged
    with pytest.raises(G.GlimError, match="ERANGE"):
        gm.insert(torch.tensor([[2.0 ** 20, 0, 0, 1]], dtype=torch.float32, device="cuda"), cov1)
    with pytest.raises(G.GlimError, match="EINVAL"):
        gm.insert(torch.tensor([[0, 0, 0, 1]], dtype=torch.float32, device="cuda"),
                  torch.tensor([[float("inf"), 0, 0, 1, 0, 1]], dtype=torch.float32, device="cuda"))
    # a far point makes the key box too large for a dense grid: "dense" is refused ...
    far = torch.tensor([[40000.0, -30000.0, 20000.0, 1.0]], dtype=torch.float32, device="cuda")
    with pytest.raises(G.GlimError, match="EINVAL"):
        gm.insert(far, cov1, layout="dense")
    unchanged()
    # ... a plan made now goes stale with the next insertion ...
    plan = G.Plan(ctx, room.gframes, [None, gm], room.w.pairs)
    plan.linearize(room.w.poses)
    gm.insert(far, cov1)                                # "auto" falls back to the hash table
    assert not any(gm.is_dense(l) for l in range(len(res)))
    with pytest.raises(G.GlimError, match="EINVAL"):
        plan.linearize(room.w.poses)
    # ... and the grown map equals the oracle's map of all points
    allp = np.concatenate([g.pts4.cpu().numpy(), far.cpu().numpy()])
    allc = np.concatenate([g.cov6.cpu().numpy(), cov1.cpu().numpy()])
    _assert_same_map(gm, O.VMap(allp, allc, res), len(res))
    # a fresh plan runs and agrees with the oracle on the original pairs (the far voxel is never hit)
    e, H, b, inl = G.Plan(ctx, room.gframes, [None, gm], room.w.pairs).linearize(room.w.poses)
    ref = O.linearize(room.oframes, [None, O.VMap(allp, allc, res)], room.w.pairs, room.w.poses, want_comp=True)
    from gpu_helpers import rel_errors
    ee, eH, eb = rel_errors(e, H, b, ref)
    assert (np.asarray(inl) == ref["inliers"]).all()
    assert ee.max() <= TOL and eH.max() <= TOL and eb.max() <= TOL


def test_insert_into_empty_map(G, ctx, room):
    g = room.gframes[1]
    res = room.w.resolutions
    empty = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    gm = G.VoxelMap(ctx, empty, torch.empty((0, 6), dtype=torch.float32, device="cuda"), res)
    assert gm.info(0)["n_voxels"] == 0
    gm.insert(g.pts4, g.cov6)
    _assert_same_map(gm, room.omaps[1], len(res))


def test_plan_refuses_to_launch_on_a_freed_map(G, ctx, room):
    """A plan whose target map has been freed raises instead of launching on tables that no
    longer exist; the other plans of the context are unaffected."""
    g = room.gframes[1]
    vm = G.VoxelMap(ctx, g.pts4, g.cov6, room.w.resolutions)
    other = G.Plan(ctx, room.gframes, room.gmaps, room.w.pairs)
    plan = G.Plan(ctx, room.gframes, [None, vm], room.w.pairs)
    first = plan.linearize(room.w.poses)
    ref = [np.asarray(x).copy() for x in other.linearize(room.w.poses)]
    vm.free()
    for call in (lambda: plan.linearize(room.w.poses), plan.launch, lambda: plan.set_poses(room.w.poses)):
        with pytest.raises(G.GlimError, match="freed"):
            call()
    for a, b in zip(other.linearize(room.w.poses), ref):
        assert np.array_equal(np.asarray(a), b)
    assert np.array_equal(np.asarray(first[3]), ref[3])
    plan.close()
    other.close()
