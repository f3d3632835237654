"""Shared set-up of the GPU parity tests: the same seeded workload is handed to the CUDA
library and to the oracle with bit-identical float32 inputs (points, covariances, normals).

Covariances and normals are computed once (by the library, on the GPU) and then copied to
both sides, so linearization parity never depends on covariance parity; the covariance
kernel is compared with the oracle separately.
"""
from __future__ import annotations

import numpy as np
import torch

import paper_2407_10344_b300 as G
from oracle import oracle as O


class Prepared:
    def __init__(self, ctx, w, k=10, validate_normals=True, cov_source="gpu", layout="auto"):
        self.ctx = ctx
        self.w = w
        dev = torch.device("cuda", ctx.device)
        self.gframes, self.oframes = [], []
        targets = set(int(t) for t in w.pairs[:, 1])
        self.gmaps = [None] * len(w.points)
        self.omaps = [None] * len(w.points)
        weights = w.weights or [None] * len(w.points)
        for i, (p, wt) in enumerate(zip(w.points, weights)):
            p4 = G.to_pts4(p, wt, device=dev)
            if cov_source == "gpu":
                cov, nrm = G.estimate_covariances(ctx, p4, k=k)
            else:
                c64, n64, _, _ = O.estimate_covariances(p, k=k)
                cov = torch.as_tensor(c64.astype(np.float32), device=dev)
                nrm = torch.as_tensor(n64.astype(np.float32), device=dev)
            torch.cuda.synchronize()
            if not validate_normals:
                nrm = None
            self.gframes.append(G.FrameData(p4, cov, nrm))
            self.oframes.append(O.Frame(p4.cpu().numpy(), cov.cpu().numpy(),
                                        None if nrm is None else nrm.cpu().numpy()))
            if i in targets:
                self.gmaps[i] = G.VoxelMap(ctx, p4, cov, w.resolutions, layout=layout)
                self.omaps[i] = O.VMap(self.oframes[i].pts4, self.oframes[i].cov6, w.resolutions)

    def oracle(self, pairs=None, poses=None, validate=False, want_ids=False, nthreads=8):
        pairs = self.w.pairs if pairs is None else pairs
        poses = self.w.poses if poses is None else poses
        return O.linearize(self.oframes, self.omaps, pairs, poses, validate=validate, want_ids=want_ids,
                           want_comp=True, nthreads=nthreads)


def rel_errors(e, H, b, ref):
    """Per-pair errors of (e, H, b) against the oracle result `ref`:
    e: |e - e*| / |e*|;  H: |H - H*|_F / |H*|_F;  b: |b - b*|_2 / max(|b*|_2, sum |J^T Omega d|_2)."""
    e = np.asarray(e, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64).reshape(-1, 12, 12)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 12)
    ee = np.abs(e - ref["e"]) / np.maximum(np.abs(ref["e"]), 1e-300)
    eH = np.linalg.norm((H - ref["H"]).reshape(len(e), -1), axis=1) / np.maximum(
        np.linalg.norm(ref["H"].reshape(len(e), -1), axis=1), 1e-300)
    scale = np.maximum(np.linalg.norm(ref["b"], axis=1), ref["b_scale"])
    eb = np.linalg.norm(b - ref["b"], axis=1) / np.maximum(scale, 1e-300)
    return ee, eH, eb


def numpy_of(x):
    return x.cpu().numpy() if isinstance(x, torch.Tensor) else np.asarray(x)


def b_rel_plain(b, ref):
    """|b - b*|_2 / |b*|_2 per pair: the plain relative error of b, reported beside the P7
    measure (whose denominator also admits the cancellation-free scale)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1, 12)
    return np.linalg.norm(b - ref["b"], axis=1) / np.maximum(np.linalg.norm(ref["b"], axis=1), 1e-300)
