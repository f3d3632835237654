"""Parity at the benchmark's full sizes, in the launch configuration the benchmark times.

* Urban global step (400 submaps of log-U[50k, 200k] points, 4000 pairs, 0.5 / 1 / 2 m): the
  whole batch runs as one plan (dense-grid kernel, block 64, 64 points per thread, FP64
  cross-block sums, Z-ordered points, persistent work queue); a seeded sample of pairs is
  recomputed by the oracle one pair at a time on the same float32 inputs, and each sampled
  pair must match (inliers exactly, e / H / b within 1e-4, and the correspondence ids that the
  kernel's id-recording instantiation resolved, in the same launch configuration, bit for
  bit).  The plain relative error of b, |b - b*| / |b*|, is bounded as well.  The same step
  on hashed voxel blocks gives the same bits for all 4000 pairs (e, H, b, ids and the gradient);
  the gradient of the sampled pairs matches the oracle's analytic gradient; with surface
  validation, sampled pairs match the oracle too.
* Odometry window at its full size (30k-point frame, 10 keyframes, per-point weights): the
  gradient of the batch against the oracle's analytic gradient.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    import paper_2407_10344_b300 as G
    return G


@pytest.fixture(scope="module")
def ctx(G):
    return G.Context(0)


def test_urban_global_step_full_size_sampled_pairs(G, ctx):
    from gpu_helpers import b_rel_plain, rel_errors
    w = synth.urban(n_submaps=400)
    dev = torch.device("cuda", ctx.device)
    frames, maps = [], [None] * len(w.points)
    targets = set(int(t) for t in w.pairs[:, 1])
    for i, p in enumerate(w.points):
        p4 = G.to_pts4(p, device=dev)
        cov, nrm = G.estimate_covariances(ctx, p4, k=10)
        perm = G.spatial_order(ctx, p4, 0.5)
        p4, cov, nrm = p4[perm].contiguous(), cov[perm].contiguous(), nrm[perm].contiguous()
        frames.append(G.FrameData(p4, cov, nrm))
        if i in targets:
            maps[i] = G.VoxelMap(ctx, p4, cov, w.resolutions)
    plan = G.Plan(ctx, frames, maps, w.pairs, accum_mode=G.ACC_FP64, block=64, pts_per_thread=64)
    assert plan.opts()["kernel"] == "dense"
    e, H, b, inl = [np.array(x) for x in plan.linearize(w.poses)]
    assert np.isfinite(e).all() and np.isfinite(H).all() and np.isfinite(b).all()
    ids, (e_i, H_i, b_i, inl_i) = plan.correspondence_ids(w.poses)
    assert np.array_equal(e_i, e) and np.array_equal(H_i, H) and np.array_equal(b_i, b)
    L = len(w.resolutions)
    off = np.concatenate([[0], np.cumsum([frames[int(s_)].n * L for s_ in w.pairs[:, 0]])])
    sample = np.sort(synth.Stream(11, "urban-sample").integers(8, 0, len(w.pairs)))
    worst = [0.0, 0.0, 0.0, 0.0]
    for q in sample:
        s, t = int(w.pairs[q, 0]), int(w.pairs[q, 1])
        fs = O.Frame(frames[s].pts4.cpu().numpy(), frames[s].cov6.cpu().numpy(), frames[s].normal3.cpu().numpy())
        ft = O.Frame(frames[t].pts4.cpu().numpy(), frames[t].cov6.cpu().numpy())
        vm = O.VMap(ft.pts4, ft.cov6, w.resolutions)
        ref = O.linearize([fs, ft], [None, vm], np.array([[0, 1]], np.int32), np.stack([w.poses[s], w.poses[t]]),
                          want_comp=True, want_ids=True)
        assert inl[q] == ref["inliers"][0], (q, inl[q], ref["inliers"][0])
        got = ids[int(off[q]):int(off[q + 1])].cpu().numpy()
        assert np.array_equal(got, ref["ids"]), (q, int((got != ref["ids"]).sum()))
        ee, eH, eb = rel_errors(e[q:q + 1], H[q:q + 1], b[q:q + 1], ref)
        ebp = b_rel_plain(b[q:q + 1], ref)
        worst = [max(worst[0], ee[0]), max(worst[1], eH[0]), max(worst[2], eb[0]), max(worst[3], ebp[0])]
    print("urban full size, worst over sampled pairs: e %.2e  H %.2e  b (P7) %.2e  b plain %.2e" % tuple(worst))
    assert max(worst) <= TOL, worst

    # The same step on hashed voxel blocks, in the same launch configuration: the hash kernel
    # resolves every (pair, point, level) to the same record as the dense-grid kernel and runs
    # the same arithmetic, so all 4000 pairs' e, H and b are the same bits.
    hmaps = [None if m is None else G.VoxelMap(ctx, frames[i].pts4, frames[i].cov6, w.resolutions, layout="hash")
             for i, m in enumerate(maps)]
    plan_h = G.Plan(ctx, frames, hmaps, w.pairs, accum_mode=G.ACC_FP64, block=64, pts_per_thread=64)
    assert plan_h.opts()["kernel"] == "hash"
    e_h, H_h, b_h, inl_h = [np.array(x) for x in plan_h.linearize(w.poses)]
    assert np.array_equal(e_h, e) and np.array_equal(H_h, H) and np.array_equal(b_h, b)
    assert np.array_equal(inl_h, inl)
    ids_h, _ = plan_h.correspondence_ids(w.poses)
    assert torch.equal(ids_h, ids)
    # the gradient of the whole step is the same bits on both layouts (the pipelined gradient
    # kernel, one fetch per layout), and the gradient of the sampled pairs alone matches the
    # oracle's analytic gradient at these frame sizes
    g_d = plan.backward(w.poses)
    g_h = plan_h.backward(w.poses)
    for a_, b_ in zip(g_d, g_h):
        assert torch.equal(a_, b_)
    plan_h.close()
    for m in hmaps:
        if m is not None:
            m.free()
    # the same step with surface validation (S3), sampled pairs against the oracle
    plan_v = G.Plan(ctx, frames, maps, w.pairs, accum_mode=G.ACC_FP64, block=64, pts_per_thread=64,
                    validate_surface=True)
    e_v, H_v, b_v, inl_v = [np.array(x) for x in plan_v.linearize(w.poses)]
    ids_v, _ = plan_v.correspondence_ids(w.poses)
    for q in sample[:4]:
        s, t = int(w.pairs[q, 0]), int(w.pairs[q, 1])
        fs = O.Frame(frames[s].pts4.cpu().numpy(), frames[s].cov6.cpu().numpy(), frames[s].normal3.cpu().numpy())
        ft = O.Frame(frames[t].pts4.cpu().numpy(), frames[t].cov6.cpu().numpy())
        vm = O.VMap(ft.pts4, ft.cov6, w.resolutions)
        ref = O.linearize([fs, ft], [None, vm], np.array([[0, 1]], np.int32), np.stack([w.poses[s], w.poses[t]]),
                          validate=True, want_comp=True, want_ids=True)
        assert inl_v[q] == ref["inliers"][0] and inl_v[q] < inl[q]
        assert np.array_equal(ids_v[int(off[q]):int(off[q + 1])].cpu().numpy(), ref["ids"])
        ee, eH, eb = rel_errors(e_v[q:q + 1], H_v[q:q + 1], b_v[q:q + 1], ref)
        assert max(ee[0], eH[0], eb[0]) <= TOL
    plan_v.close()
    used = sorted(set(int(v) for v in w.pairs[sample].ravel()))
    remap = {f: i for i, f in enumerate(used)}
    sub_pairs = np.array([[remap[int(a_)], remap[int(b_)]] for a_, b_ in w.pairs[sample]], np.int32)
    sub_frames = [frames[f] for f in used]
    sub_maps = [maps[f] if f in set(int(t) for t in w.pairs[sample, 1]) else None for f in used]
    sub_poses = np.stack([w.poses[f] for f in used])
    dxi, dmu, dw = G.Plan(ctx, sub_frames, sub_maps, sub_pairs).backward(sub_poses)
    ofr = [O.Frame(f.pts4.cpu().numpy(), f.cov6.cpu().numpy(), f.normal3.cpu().numpy()) for f in sub_frames]
    omp = [None if m is None else O.VMap(ofr[i].pts4, ofr[i].cov6, w.resolutions) for i, m in enumerate(sub_maps)]
    odxi, odmu, odw = O.gradient(ofr, omp, sub_pairs, sub_poses)
    assert np.linalg.norm(dxi.cpu().numpy() - odxi) <= TOL * np.linalg.norm(odxi)
    odmu_all, odw_all = np.concatenate(odmu), np.concatenate(odw)
    assert np.linalg.norm(dmu.cpu().numpy() - odmu_all) <= TOL * np.linalg.norm(odmu_all)
    assert np.linalg.norm(dw.cpu().numpy() - odw_all) <= TOL * np.linalg.norm(odw_all)


def test_odometry_window_gradient_full_size(G, ctx):
    from gpu_helpers import Prepared
    P = Prepared(ctx, synth.corridor(weights=True))
    w = P.w
    assert w.n_pair_points == 300000
    for full in (True, False):
        dxi, dmu, dw = G.backward(ctx, P.gframes, P.gmaps, w.pairs, w.poses, omega_grad_full=full)
        odxi, odmu, odw = O.gradient(P.oframes, P.omaps, w.pairs, w.poses, omega_grad_full=full)
        gxi = dxi.cpu().numpy()
        assert np.linalg.norm(gxi - odxi) <= TOL * np.linalg.norm(odxi)
        n0 = len(w.points[0])
        gmu, gw = dmu.cpu().numpy()[:n0], dw.cpu().numpy()[:n0]
        assert np.linalg.norm(gmu - odmu[0]) <= TOL * np.linalg.norm(odmu[0])
        assert np.linalg.norm(gw - odw[0]) <= TOL * np.linalg.norm(odw[0])
