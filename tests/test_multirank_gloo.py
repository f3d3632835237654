"""Multi-rank host logic on the CPU with the gloo backend (world size 2): sharding the pair
list by source frame and gathering the per-rank (e, H, b) records reproduces the single-rank
result bit for bit (the oracle stands in for the per-rank compute; no GPU), and the bench's
cross-rank aggregation takes the slowest time and the total work."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        from oracle import oracle as O
        from paper_2407_10344_b300.api import frames_needed, shard_pairs
        w = synth.urban(n_submaps=400, keep=8, neighbours=3, point_scale=0.02)
        idx = shard_pairs(w.pairs, rank, world)
        need = frames_needed(w.pairs, idx)
        cov = [np.tile(np.array([1.0, 0, 0, 1.0, 0, 1e-3], np.float32), (len(p), 1)) for p in w.points]
        frames = [O.Frame(O.as_pts4(p), c) for p, c in zip(w.points, cov)]
        vmaps = [O.VMap(frames[f].pts4, frames[f].cov6, w.resolutions) if f in need else None
                 for f in range(len(frames))]
        r = O.linearize(frames, vmaps, w.pairs[idx], w.poses) if len(idx) else dict(e=[], H=[], b=[])
        gathered = [None] * world
        dist.all_gather_object(gathered, (idx.tolist(), np.asarray(r["e"]), np.asarray(r["H"]), np.asarray(r["b"])))
        tmax, total = bench.aggregate_over_ranks(10.0 + rank, 100 * (rank + 1), torch.device("cpu"))
        if rank == 0:
            all_vm = [O.VMap(f.pts4, f.cov6, w.resolutions) for f in frames]
            full = O.linearize(frames, all_vm, w.pairs, w.poses)
            e = np.zeros(len(w.pairs))
            H = np.zeros((len(w.pairs), 12, 12))
            b = np.zeros((len(w.pairs), 12))
            seen = []
            for ids, ee, HH, bb in gathered:
                seen += ids
                if len(ids):
                    e[ids], H[ids], b[ids] = ee, HH, bb
            ok = (sorted(seen) == list(range(len(w.pairs))) and np.array_equal(e, full["e"])
                  and np.array_equal(H, full["H"]) and np.array_equal(b, full["b"])
                  and tmax == 11.0 and total == 300.0 and all(len(g[0]) > 0 for g in gathered))
            out.put(bool(ok))
    finally:
        dist.destroy_process_group()


def test_sharded_pairs_gather_to_the_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=10) is True


def test_shard_pairs_partitions_by_source():
    from paper_2407_10344_b300.api import shard_pairs
    pairs = np.array([[s, t] for s in range(10) for t in range(3) if t != s])
    for world in (1, 2, 3, 4):
        parts = [shard_pairs(pairs, r, world) for r in range(world)]
        cat = np.sort(np.concatenate(parts))
        assert np.array_equal(cat, np.arange(len(pairs)))
        srcs = [set(pairs[p][:, 0].tolist()) for p in parts]
        for i in range(world):
            for j in range(i + 1, world):
                assert not (srcs[i] & srcs[j])
