"""Out-of-memory handling, tested by failing allocations on the host.

glim_debug_fail_allocation makes one chosen allocation of the library report
cudaErrorMemoryAllocation without touching the device. Each public operation runs once per
allocation it makes, with that allocation failing. It must raise GLIM_ENOMEM and leave the
objects it was given as they were. The context must then reproduce, bit for bit, the
results it gave before the sweep. No GPU fault, trap or hang is involved.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_2407_10344_b300 as G
    yield G
    G.debug_fail_allocation(-1)


def sweep(G, op, check=None, limit=400):
    """Run op with the allocation n from its start failing, for n = 0, 1, ... until op
    succeeds; after each failure call check().  Returns the number of allocations op made."""
    for n in range(limit):
        G.debug_fail_allocation(n)
        try:
            op()
        except G.GlimError as e:
            G.debug_fail_allocation(-1)
            assert "ENOMEM" in str(e), str(e)
            if check is not None:
                check()
            continue
        finally:
            G.debug_fail_allocation(-1)
        return n
    raise AssertionError("the operation kept failing")


@pytest.fixture(scope="module")
def batch(G):
    ctx = G.Context(0)
    w = synth.corridor(n_cur=3000, kf_range=(2000, 3000), n_kf=2, weights=True)
    dev = torch.device("cuda", 0)
    frames, maps = [], []
    targets = set(int(t) for t in w.pairs[:, 1])
    for i, p in enumerate(w.points):
        p4 = G.to_pts4(p, w.weights[i], device=dev)
        cov, nrm = G.estimate_covariances(ctx, p4)
        frames.append(G.FrameData(p4, cov, nrm))
        maps.append(G.VoxelMap(ctx, p4, cov, w.resolutions) if i in targets else None)
    ref = [np.asarray(x).copy() for x in G.linearize(ctx, frames, maps, w.pairs, w.poses)]

    def same_as_before():
        got = G.linearize(ctx, frames, maps, w.pairs, w.poses)
        for a, b in zip(got, ref):
            assert np.array_equal(np.asarray(a), b)

    return ctx, w, frames, maps, same_as_before


def test_every_allocation_failure_reports_enomem_and_leaves_the_context_usable(G, batch):
    # the second round runs with every cache warm: device memory it does not give back is a leak
    counts = run_all(G, batch)
    free0 = free_memory()
    assert run_all(G, batch) == counts
    free1 = free_memory()
    assert free1 >= free0 - (8 << 20), (free0, free1, counts)
    print(counts)


def free_memory():
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def run_all(G, batch):
    ctx, w, frames, maps, same_as_before = batch
    counts = {}
    p4, cov = frames[0].pts4, frames[0].cov6
    t = int(w.pairs[0, 1])

    counts["context"] = sweep(G, lambda: G.Context(0).close(), same_as_before)
    counts["covariances"] = sweep(G, lambda: G.estimate_covariances(ctx, p4), same_as_before)
    counts["spatial_order"] = sweep(G, lambda: G.spatial_order(ctx, p4), same_as_before)
    for layout in ("auto", "hash"):
        counts["voxelmap_" + layout] = sweep(
            G, lambda: G.VoxelMap(ctx, p4, cov, w.resolutions, layout=layout).free(), same_as_before)

    # a failed insertion leaves the map as it was
    vm = G.VoxelMap(ctx, frames[t].pts4, frames[t].cov6, w.resolutions)
    keys0 = [vm.export(l)["keys"].cpu().numpy() for l in range(vm.levels)]

    def map_unchanged():
        for l in range(vm.levels):
            assert np.array_equal(vm.export(l)["keys"].cpu().numpy(), keys0[l])

    counts["insert"] = sweep(G, lambda: vm.insert(p4, cov), map_unchanged)
    vm.free()

    def plan_linearize():
        plan = G.Plan(ctx, frames, maps, w.pairs)
        try:
            plan.linearize(w.poses)
        finally:
            plan.close()

    counts["plan"] = sweep(G, plan_linearize, same_as_before)
    counts["one_shot"] = sweep(G, lambda: G.linearize(ctx, frames, maps, w.pairs, w.poses), same_as_before)
    counts["plain"] = sweep(G, lambda: G.linearize(ctx, frames, maps, w.pairs, w.poses, plain=True),
                            same_as_before)
    counts["backward"] = sweep(G, lambda: G.backward(ctx, frames, maps, w.pairs, w.poses), same_as_before)
    counts["overlap"] = sweep(G, lambda: G.overlap(ctx, frames, maps, w.pairs, w.poses), same_as_before)
    counts["correspondences"] = sweep(
        G, lambda: G.correspondences(ctx, frames[0], maps[t], w.poses[0], w.poses[t]), same_as_before)

    # the plan's gradient scratch, and an autotuner whose reconfiguration fails: the plan
    # keeps a configuration it can launch and gives the same results
    plan_b = G.Plan(ctx, frames, maps, w.pairs, block=256, pts_per_thread=1)
    grads0 = G.backward(ctx, frames, maps, w.pairs, w.poses)
    counts["plan_backward"] = sweep(G, lambda: plan_b.backward(w.poses), same_as_before)
    for a, b in zip(plan_b.backward(w.poses), grads0):
        assert torch.equal(a, b)
    plan = G.Plan(ctx, frames, maps, w.pairs)
    ref_plan = [np.asarray(x).copy() for x in plan.linearize(w.poses)]

    def plan_still_launches():
        for a, b in zip(plan.linearize(w.poses), ref_plan):
            assert np.array_equal(np.asarray(a), b)

    counts["autotune"] = sweep(G, lambda: plan.autotune(w.poses, iters=1), plan_still_launches)
    # the tuned configuration groups the FP32 per-lane sums differently: equal up to rounding
    for a, b in zip(plan.linearize(w.poses)[:3], ref_plan[:3]):
        np.testing.assert_allclose(np.asarray(a), b, rtol=1e-5, atol=1e-5 * np.abs(b).max())
    plan.close()
    plan_b.close()

    # the device Gauss-Newton loop's buffers and graph: a failure leaves the plan as it was
    plan_g = G.Plan(ctx, frames, maps, w.pairs)
    ref_g = [np.asarray(x).copy() for x in plan_g.linearize(w.poses)]

    def gn_plan_unchanged():
        for a, b in zip(plan_g.linearize(w.poses), ref_g):
            assert np.array_equal(np.asarray(a), b)

    counts["gauss_newton"] = sweep(G, lambda: plan_g.gauss_newton(w.poses, 0, 2), gn_plan_unchanged)
    plan_g.close()

    e, H, b, _ = G.linearize(ctx, frames, maps, w.pairs, w.poses, out="cuda")
    counts["graph_step"] = sweep(G, lambda: G.graph_step(ctx, w.pairs, len(frames), H, b), same_as_before)
    counts["gn_solve"] = sweep(G, lambda: G.gn_solve(ctx, H, b), same_as_before)

    # every operation that allocates reached its failure paths at least once
    for name in ("context", "covariances", "voxelmap_auto", "voxelmap_hash", "insert", "plan", "one_shot",
                 "backward", "plan_backward", "autotune", "gauss_newton", "graph_step"):
        assert counts[name] >= 1, (name, counts)
    same_as_before()
    return counts
