"""Differentiable matching cost: E = sum over factor pairs of e (Eq. (2)), with per-point
weights, as a ``torch.autograd.Function``.

Inputs: per-frame pose increments ``xi`` (nframes x 6, [omega; v], applied on the right,
T_f <- T_f Exp(xi_f)), the source points' coordinates and their weights.  The forward pass
is the library's batched linearization (the cost only is kept).  The gradient comes from
``glim_plan_backward``, which recomputes the per-point Jacobians instead of storing them.
When an input needs a gradient, the forward pass enqueues that gradient pass right after
the linearization, on the same point buffer and device pose block (no second upload, no
host wait); the backward pass then only scales the three gradients by the incoming one.

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


def retract_many(T, xi):
    """T_f Exp(xi_f) for a stack of 3x4 poses (n, 3, 4) and increments (n, 6), vectorised
    over f with the same Rodrigues / left-Jacobian formulas as se3_exp."""
    T = np.asarray(T, dtype=np.float64).reshape(-1, 3, 4)
    xi = np.asarray(xi, dtype=np.float64).reshape(-1, 6)
    w, v = xi[:, :3], xi[:, 3:]
    th = np.linalg.norm(w, axis=1)
    K = np.zeros((len(xi), 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -w[:, 2], w[:, 1], -w[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = w[:, 2], -w[:, 1], w[:, 0]
    K2 = K @ K
    small = th < 1e-10
    ts = np.where(small, 1.0, th)
    a = np.where(small, 1.0, np.sin(ts) / ts)
    b = np.where(small, 0.5, (1 - np.cos(ts)) / ts ** 2)
    c = np.where(small, 1.0 / 6.0, (ts - np.sin(ts)) / ts ** 3)
    I = np.eye(3)[None]
    R = I + a[:, None, None] * K + b[:, None, None] * K2
    V = I + b[:, None, None] * K + c[:, None, None] * K2
    out = np.empty_like(T)
    out[:, :, :3] = T[:, :, :3] @ R
    out[:, :, 3] = np.einsum("nij,nj->ni", T[:, :, :3], np.einsum("nij,nj->ni", V, v)) + T[:, :, 3]
    return out


class FactorProblem:
    """A fixed batch of factors: frame covariances and normals, target voxelmaps, pairs, the
    base poses, and the split of the concatenated point array into frames.

    The problem owns one packed (n, 4) point buffer (the frames are row ranges of it) and one
    plan over it, so that an evaluation only writes the current points and weights into the
    buffer and launches."""

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
        self._p4 = torch.cat([f.pts4 for f in self.frames]).contiguous()
        self._bufs = [api.FrameData(self._p4[int(self.offsets[i]):int(self.offsets[i + 1])], f.cov6, f.normal3)
                      for i, f in enumerate(self.frames)]
        self._plan = api.Plan(ctx, self._bufs, self.vmaps, self.pairs, validate_surface=self.validate)
        self._out = self._plan.device_outputs_alloc()

    def points(self):
        """Concatenated source coordinates (n, 3) and weights (n,) of the frames."""
        pts = torch.cat([f.pts4[:, :3] for f in self.frames])
        w = torch.cat([f.pts4[:, 3] for f in self.frames])
        return pts, w

    def _load(self, points, weights):
        """Write the points and weights of an evaluation into the plan's buffer (one kernel)."""
        buf = self._p4.untyped_storage().data_ptr()
        if points.untyped_storage().data_ptr() == buf or weights.untyped_storage().data_ptr() == buf:
            self._p4[:, :3].copy_(points)  # views of the buffer itself
            self._p4[:, 3].copy_(weights)
        else:
            torch.cat((points, weights.unsqueeze(1)), dim=1, out=self._p4)

    def poses_at(self, xi):
        x = xi.detach().cpu().numpy().astype(np.float64).reshape(-1, 6)
        return retract_many(self.poses, x)

    def energy(self, xi, points, weights):
        """Differentiable E(xi, points, weights) (0-dim float64 CUDA tensor)."""
        return GlimFactorFn.apply(xi, points, weights, self)


class GlimFactorFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, xi, points, weights, problem: FactorProblem):
        problem._load(points.detach().float(), weights.detach().float())
        poses = problem.poses_at(xi)
        e, _, _, _ = problem._plan.linearize(poses, out=problem._out)
        # The gradient pass reads the buffer as this evaluation wrote it, so later evaluations
        # may reuse the buffer before this one's backward runs.
        fctx.grads = (problem._plan.backward(poses, omega_grad_full=problem.full)
                      if any(fctx.needs_input_grad[:3]) else None)
        fctx.xi_device = xi.device
        fctx.xi_dtype = xi.dtype
        return e.sum()

    @staticmethod
    def backward(fctx, grad_out):
        dxi, dmu, dw = fctx.grads
        fctx.grads = None
        need = fctx.needs_input_grad
        # grad_out is a 0-dim FP64 tensor: the products keep the gradients' own dtypes
        gxi = (dxi * grad_out).to(device=fctx.xi_device, dtype=fctx.xi_dtype) if need[0] else None
        return gxi, dmu * grad_out if need[1] else None, dw * grad_out if need[2] else None, None
