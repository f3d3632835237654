"""kNN covariances at the benchmark's frame sizes (Sec. III-C "Preprocessing", Sec. IV-A: the
per-point covariance from the k = 10 nearest neighbours, plane-regularised), against the
oracle's brute force on sampled query points.

The grid search runs on a whole urban submap (107k-200k points) and on the 20M-point terrain
map; the oracle scans every point of the frame for each sampled query.  The sample is 1,000
uniformly drawn points plus the 200 most isolated points (largest distance to their 10th
neighbour), which the grid search settles only after widening its shells or by the
whole-frame scan.  Neighbour lists must be identical (both sides order by the FP64 squared
distance, then the index); covariances and normals within 1e-4.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-4


def _check_frame(G, ctx, pts, seed):
    p4 = G.to_pts4(pts, device="cuda")
    cov, nrm, knn = G.estimate_covariances_knn(ctx, p4, k=10)
    knn_g = knn.cpu().numpy()
    # the most isolated points by the GPU's own neighbour lists
    P = p4[:, :3].double()
    far = (P[knn[:, -1].long()] - P).norm(dim=1).cpu().numpy()
    iso = np.argsort(-far, kind="stable")[:200]
    rnd = synth.Stream(seed, "cov-scale").integers(1000, 0, len(pts))
    q = np.unique(np.concatenate([rnd, iso]))
    c64, n64, k64, tie = O.covariances_at(pts, q, k=10)
    assert np.array_equal(knn_g[q], k64), int((knn_g[q] != k64).any(axis=1).sum())
    ok = ~tie
    assert tie.sum() <= 0.01 * len(q)
    Cg = cov.cpu().numpy().astype(np.float64)[q][:, [0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(-1, 3, 3)
    Co = c64[:, [0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(-1, 3, 3)
    rel = np.linalg.norm((Cg - Co).reshape(len(q), -1), axis=1) / np.linalg.norm(Co.reshape(len(q), -1), axis=1)
    assert rel[ok].max() <= TOL, rel[ok].max()
    assert np.abs(nrm.cpu().numpy().astype(np.float64)[q][ok] - n64[ok]).max() <= TOL
    return len(q), float(far[iso].min())


def test_knn_covariances_urban_submap_sampled():
    import paper_2407_10344_b300 as G
    ctx = G.Context(0)
    w = synth.urban(n_submaps=400, keep=12)
    sizes = np.array([len(p) for p in w.points])
    f = int(np.argmax(sizes))
    assert 107_000 <= sizes[f] <= 200_000
    nq, far = _check_frame(G, ctx, w.points[f], 31)
    assert nq >= 1000


def test_knn_covariances_terrain_map_sampled():
    import paper_2407_10344_b300 as G
    ctx = G.Context(0)
    w = synth.terrain()
    pts = w.points[1]
    assert len(pts) == 20_000_000
    nq, far = _check_frame(G, ctx, pts, 32)
    assert nq >= 1000
