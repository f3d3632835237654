"""Multi-rank host logic on the CPU with the gloo backend: the global step sharded by source
frame (shard_pairs, frames_needed), each rank's factors packed into records (pack_records)
and exchanged with one all-gather (gather_records) reproduces the single-rank result bit for
bit.  The oracle stands in for each rank's GPU compute (no GPU here); the packing, the
exchange and the placement in pair order are the package's own.  Also: the bench's
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


def _worker(rank, world, port, keep, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        from oracle import oracle as O
        from paper_2407_10344_b300.api import frames_needed, gather_records, pack_records, shard_pairs, unpack_records
        w = synth.urban(n_submaps=400, keep=keep, neighbours=3, point_scale=0.02)
        P = len(w.pairs)
        idx = shard_pairs(w.pairs, rank, world)
        need = frames_needed(w.pairs, idx)
        cov = [np.tile(np.array([1.0, 0, 0, 1.0, 0, 1e-3], np.float32), (len(p), 1)) for p in w.points]
        frames = [O.Frame(O.as_pts4(p), c) for p, c in zip(w.points, cov)]
        vmaps = [O.VMap(frames[f].pts4, frames[f].cov6, w.resolutions) if f in need else None
                 for f in range(len(frames))]
        if len(idx):
            r = O.linearize(frames, vmaps, w.pairs[idx], w.poses)
            rec = pack_records(r["e"], r["H"], r["b"], r["inliers"])
        else:
            rec = np.zeros((0, 92))
        full_rec = gather_records(torch.as_tensor(rec), idx, P)  # every rank gets all records
        tmax, total = bench.aggregate_over_ranks(10.0 + rank, 100 * (rank + 1), torch.device("cpu"))
        if rank == 0:
            all_vm = [O.VMap(f.pts4, f.cov6, w.resolutions) for f in frames]
            full = O.linearize(frames, all_vm, w.pairs, w.poses)
            ref = pack_records(full["e"], full["H"], full["b"], full["inliers"])
            e, H, b, inl = unpack_records(full_rec)
            iu = np.triu_indices(12)
            sizes = [len(shard_pairs(w.pairs, q, world)) for q in range(world)]
            ok = (np.array_equal(full_rec.numpy(), ref) and np.array_equal(e, full["e"])
                  and np.array_equal(H[:, iu[0], iu[1]], full["H"][:, iu[0], iu[1]])
                  and np.array_equal(H, np.transpose(H, (0, 2, 1))) and np.array_equal(b, full["b"])
                  and np.array_equal(inl, full["inliers"]) and sum(sizes) == P
                  and tmax == 10.0 + world - 1 and total == 100.0 * world * (world + 1) / 2)
            out.put((bool(ok), sizes))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,keep", [(2, 8), (3, 2)])
def test_sharded_pairs_gather_to_the_full_result(world, keep):
    """world 2 over 8 source submaps; world 3 over 2 source submaps (one rank holds no pair)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, keep, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    ok, sizes = q.get(timeout=10)
    assert ok, sizes
    if keep == 2:
        assert 0 in sizes


def test_records_round_trip():
    from paper_2407_10344_b300.api import pack_records, unpack_records
    rng = np.random.default_rng(1)
    A = rng.normal(size=(5, 12, 12))
    H = A + np.transpose(A, (0, 2, 1))
    e, b, inl = rng.normal(size=5), rng.normal(size=(5, 12)), np.arange(5) * 1000
    rec = pack_records(e, H, b, inl)
    assert rec.shape == (5, 92)
    e2, H2, b2, inl2 = unpack_records(rec)
    assert np.array_equal(e2, e) and np.array_equal(H2, H) and np.array_equal(b2, b) and np.array_equal(inl2, inl)
    import torch
    rt = pack_records(torch.as_tensor(e), torch.as_tensor(H), torch.as_tensor(b), torch.as_tensor(inl))
    assert np.array_equal(rt.numpy(), rec)


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
