"""Differentiable matching cost: E = sum over factor pairs of e (Eq. (2)), with per-point
weights, as a ``torch.autograd.Function``.

Inputs: per-frame pose increments ``xi`` (nframes x 6, [omega; v], applied on the right,
T_f <- T_f Exp(xi_f)), the source points' coordinates and their weights.  The forward pass
is the library's batched linearization (the cost only is kept); the backward pass is
``glim_backward``, which recomputes the per-point Jacobians instead of storing them.

Conventions: the pose gradient is the gradient with respect to a right perturbation of the
current pose T_f Exp(xi_f); it equals d/dxi exactly at xi = 0 (the usual parameterisation of a
Gauss-Newton or gradient step).  Correspondences are piecewise constant.  Gradients flow to
points in their source role only: the target voxel statistics are data.  Covariances and
normals are constants.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def _hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def se3_exp(xi):
    """Exp of xi = [omega; v] as a 3x4 [R | t] (Rodrigues; left Jacobian on the translation)."""
    w, v = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = float(np.linalg.norm(w))
    K = _hat(w)
    if th < 1e-10:
        R = np.eye(3) + K + 0.5 * K @ K
        V = np.eye(3) + 0.5 * K + K @ K / 6.0
    else:
        R = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * K @ K
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = V @ v
    return T


def retract(T, xi):
    """T Exp(xi) for a 3x4 pose."""
    E = se3_exp(xi)
    out = np.zeros((3, 4))
    out[:, :3] = T[:, :3] @ E[:, :3]
    out[:, 3] = T[:, :3] @ E[:, 3] + T[:, 3]
    return out


class FactorProblem:
    """A fixed batch of factors: frame covariances and normals, target voxelmaps, pairs, the
    base poses, and the split of the concatenated point array into frames."""

    def __init__(self, ctx: api.Context, frames, vmaps, pairs, poses, validate_surface=False,
                 omega_grad_full=True):
        self.ctx = ctx
        self.frames = list(frames)
        self.vmaps = list(vmaps)
        self.pairs = np.asarray(pairs, dtype=np.int32)
        self.poses = np.asarray(poses, dtype=np.float64).reshape(-1, 3, 4)
        self.validate = bool(validate_surface)
        self.full = bool(omega_grad_full)
        self.sizes = [f.n for f in self.frames]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)

    def points(self):
        """Concatenated source coordinates (n, 3) and weights (n,) of the frames."""
        pts = torch.cat([f.pts4[:, :3] for f in self.frames])
        w = torch.cat([f.pts4[:, 3] for f in self.frames])
        return pts, w

    def _frames_with(self, points, weights):
        out = []
        for i, f in enumerate(self.frames):
            a, b = int(self.offsets[i]), int(self.offsets[i + 1])
            p4 = torch.empty((b - a, 4), dtype=torch.float32, device=f.pts4.device)
            p4[:, :3] = points[a:b]
            p4[:, 3] = weights[a:b]
            out.append(api.FrameData(p4, f.cov6, f.normal3))
        return out

    def poses_at(self, xi):
        x = xi.detach().cpu().numpy().astype(np.float64).reshape(-1, 6)
        return np.stack([retract(self.poses[f], x[f]) for f in range(len(self.poses))])

    def energy(self, xi, points, weights):
        """Differentiable E(xi, points, weights) (0-dim float64 CUDA tensor)."""
        return GlimFactorFn.apply(xi, points, weights, self)


class GlimFactorFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, xi, points, weights, problem: FactorProblem):
        frames = problem._frames_with(points.detach().float().contiguous(), weights.detach().float().contiguous())
        poses = problem.poses_at(xi)
        dev = points.device
        e, _, _, _ = api.linearize(problem.ctx, frames, problem.vmaps, problem.pairs, poses, out=dev,
                                   validate_surface=problem.validate)
        fctx.problem = problem
        fctx.frames = frames
        fctx.poses = poses
        fctx.xi_device = xi.device
        fctx.xi_dtype = xi.dtype
        return e.sum()

    @staticmethod
    def backward(fctx, grad_out):
        p: FactorProblem = fctx.problem
        dxi, dmu, dw = api.backward(p.ctx, fctx.frames, p.vmaps, p.pairs, fctx.poses, omega_grad_full=p.full,
                                    validate_surface=p.validate)
        g = grad_out.to(torch.float64)
        gxi = (g * dxi).to(device=fctx.xi_device, dtype=fctx.xi_dtype)
        return gxi, (g * dmu.double()).float(), (g * dw.double()).float(), None
