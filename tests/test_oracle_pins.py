"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to the paper or to mathematics: a
hand-computed case, an exact-rational emulation of the FP32 key rule, finite
differences, a gauge symmetry, a closed-form special case (Horn/Kabsch), a
textbook library routine, or brute force on tiny inputs.  A dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import fp32_exact as X
import synth
from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _frames_for(w, k=10, with_normals=True):
    covs, normals = [], []
    for p in w.points:
        c, n, _, _ = O.estimate_covariances(p, k=k, nthreads=os.cpu_count())
        covs.append(c.astype(np.float32))
        normals.append(n.astype(np.float32))
    ws = w.weights or [None] * len(w.points)
    return [O.Frame(O.as_pts4(p, wt), c, n if with_normals else None)
            for p, c, n, wt in zip(w.points, covs, normals, ws)]


@pytest.fixture(scope="module")
def room():
    w = synth.box_room(n_src=800, n_tgt=4000)
    fr = _frames_for(w)
    vm = O.VMap(fr[1].pts4, fr[1].cov6, [0.5, 1.0, 2.0])
    return w, fr, [None, vm]


def _ids_layout(fr, vms, pairs):
    return sum(len(fr[s].pts4) * vms[t].levels for s, t in pairs)


# ---------------------------------------------------------------------------- hand-computed
def test_single_point_hand_computed():
    g = json.load(open(os.path.join(GOLD, "single_point_unit_omega.json")))
    src = O.Frame(O.as_pts4(np.array([g["source_point"]])), np.array([g["cov"]], np.float32))
    tgt = O.Frame(O.as_pts4(np.array([g["target_point"]])), np.array([g["cov"]], np.float32))
    vm = O.VMap(tgt.pts4, tgt.cov6, [g["resolution"]])
    poses = np.stack([np.eye(3, 4), np.eye(3, 4)])
    r = O.linearize([src, tgt], [None, vm], [[0, 1]], poses)
    assert r["inliers"][0] == 1
    assert abs(r["e"][0] - g["e"]) < 1e-12
    np.testing.assert_allclose(r["b"][0], g["b"], atol=1e-12)
    np.testing.assert_allclose(r["H"][0], np.array(g["H"], float), atol=1e-12)


def test_b_scale_of_cancelling_terms():
    """The cancellation-free scale of b (the second denominator of the b parity measure) is
    the sum over terms of |w J^T Omega d|: two terms whose contributions cancel give b = 0
    and a scale of sqrt(29/8), not 0 (the norm of the sum) and not sqrt(29/32) (without w)."""
    g = json.load(open(os.path.join(GOLD, "cancelling_b_terms.json")))
    pts = np.array(g["points"])
    cov = np.array([g["cov"]] * len(pts), np.float32)
    src = O.Frame(O.as_pts4(pts, np.full(len(pts), g["weight"])), cov)
    tgt = O.Frame(O.as_pts4(pts), cov)
    vm = O.VMap(tgt.pts4, tgt.cov6, [g["resolution"]])
    r = O.linearize([src, tgt], [None, vm], [[0, 1]], np.stack([np.eye(3, 4), np.eye(3, 4)]), want_comp=True)
    assert r["inliers"][0] == g["inliers"]
    assert abs(r["e"][0] - g["e"]) < 1e-15
    np.testing.assert_array_equal(r["b"][0], np.array(g["b"]))
    assert abs(r["b_scale"][0] - g["b_scale"]) < 1e-14
    assert abs(g["b_scale"] - np.sqrt(29 / 8)) < 1e-15


def test_voxel_statistics_closed_form():
    g = json.load(open(os.path.join(GOLD, "two_point_voxel.json")))
    vm = O.VMap(O.as_pts4(np.array(g["points"])), np.array(g["covs"], np.float32), [g["resolution"]])
    ex = vm.export(0)
    assert len(ex["keys"]) == len(g["expected"])
    for i, v in enumerate(g["expected"]):
        assert list(ex["keys"][i]) == v["key"]
        assert ex["count"][i] == v["count"]
        np.testing.assert_allclose(ex["mean"][i], v["mean"], atol=1e-15)
        np.testing.assert_allclose(ex["cov"][i], v["cov"], atol=1e-15)


# ---------------------------------------------------------------------------- keys / ids
def _tiny_cloud(seed, n, scale):
    s = synth.Stream(seed, "tiny")
    p = s.uniform(3 * n, -scale, scale).reshape(n, 3)
    # points exactly on voxel faces (multiples of r) and negative zero
    p[: n // 4] = np.round(p[: n // 4] * 2.0) / 2.0
    p[0] = [-0.0, -1.0, 0.5]
    return p.astype(np.float32)


@pytest.mark.parametrize("seed,res", [(11, 0.5), (12, 1.0), (13, 0.3)])
def test_keys_bruteforce_exact(seed, res):
    """Correspondence ids against a brute-force scan, with every FP32 operation of the key
    rule evaluated in exact rational arithmetic and rounded once."""
    src = _tiny_cloud(seed + 100, 60, 2.0)
    Ts = synth.make_pose(synth.rot_axis_angle([0.3, -0.5, 0.8], 0.7), [0.11, -0.23, 0.05])
    Tt = synth.make_pose(synth.rot_axis_angle([-0.2, 0.1, 0.9], -0.4), [-0.3, 0.2, -0.1])
    T = O.compose(O.inverse(Tt), Ts)
    # target: random points plus the source seen through T_rel (so most lookups hit), with
    # a quarter of the points moved onto voxel faces
    near = src.astype(np.float64) @ T[:, :3].T + T[:, 3]
    near[::4] = np.round(near[::4] / res) * res
    tgt = np.concatenate([_tiny_cloud(seed, 140, 2.0), near.astype(np.float32)])
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (200, 1))
    vm = O.VMap(O.as_pts4(tgt), cov, [res])
    inv_r = np.float32(1.0 / res)
    # brute force: keys of all target points, sorted lexicographically
    tkeys = []
    for p in tgt:
        tkeys.append(tuple(X.key(c, inv_r) for c in p))
    occupied = sorted(set(tkeys))
    assert [tuple(k) for k in vm.export(0)["keys"]] == occupied
    rank = {k: i for i, k in enumerate(occupied)}
    poses = np.stack([Ts, Tt])
    Rf = T[:, :3].astype(np.float32)
    tf = T[:, 3].astype(np.float32)
    fr = [O.Frame(O.as_pts4(src), np.tile(cov[:1], (60, 1))), O.Frame(O.as_pts4(tgt), cov)]
    r = O.linearize(fr, [None, vm], [[0, 1]], poses, want_ids=True)
    expect = []
    for mu in src:
        q = [X.transform_axis(Rf[a], tf[a], mu) for a in range(3)]
        k = tuple(X.key(c, inv_r) for c in q)
        expect.append(rank.get(k, -1) if None not in k else -1)
    assert list(r["ids"]) == expect
    assert sum(i >= 0 for i in expect) > 30


def test_key_rule_fma_order_decides_face_points():
    """Points whose transformed coordinate lies within an ulp of a voxel face: the pinned
    FP32 rule (fma nesting t -> x -> y -> z) and a reordered nesting give different keys for
    some of them; the oracle must follow the pinned rule on every one."""
    res = 0.5
    inv_r = np.float32(1.0 / res)
    Ts = synth.make_pose(synth.rot_axis_angle([0.6, -0.2, 0.7], 0.9), [1.3, -0.7, 0.4])
    Tt = np.eye(3, 4)
    T = O.compose(O.inverse(Tt), Ts)
    Rf, tf = T[:, :3].astype(np.float32), T[:, 3].astype(np.float32)
    s = synth.Stream(14, "faces")
    n = 3000
    face = np.stack([np.round(s.uniform(n, -4, 4) / res) * res, s.uniform(n, -4, 4), s.uniform(n, -4, 4)], 1)
    mu = ((face - T[:, 3]) @ T[:, :3]).astype(np.float32)  # R^T (f - t), rounded to FP32

    def alt_axis(Rrow, t, m):
        return X.fma(Rrow[0], m[0], X.fma(Rrow[1], m[1], X.fma(Rrow[2], m[2], t)))

    pinned, other = [], []
    for m in mu:
        pinned.append(tuple(X.key(X.transform_axis(Rf[a], tf[a], m), inv_r) for a in range(3)))
        other.append(tuple(X.key(alt_axis(Rf[a], tf[a], m), inv_r) for a in range(3)))
    diff = [i for i in range(n) if pinned[i] != other[i]]
    assert len(diff) >= 5
    src = mu[diff]
    # target: one point at the centre of each candidate voxel, so every lookup hits
    centres = {tuple((np.array(k) + 0.5) * res) for i in diff for k in (pinned[i], other[i])}
    tgt = np.array(sorted(centres), np.float32)
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (len(tgt), 1))
    vm = O.VMap(O.as_pts4(tgt), cov, [res])
    rank = {tuple(k): i for i, k in enumerate(vm.export(0)["keys"])}
    fr = [O.Frame(O.as_pts4(src), cov[:1].repeat(len(src), 0)), O.Frame(O.as_pts4(tgt), cov)]
    r = O.linearize(fr, [None, vm], [[0, 1]], np.stack([Ts, Tt]), want_ids=True)
    assert list(r["ids"]) == [rank[pinned[i]] for i in diff]


def test_key_range_and_invalid_input():
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (2, 1))
    far = np.array([[0, 0, 0], [2.0 ** 21, 0, 0]], np.float32)
    with pytest.raises(ValueError, match="-5"):
        O.VMap(O.as_pts4(far), cov, [1.0])
    bad = np.array([[0, 0, 0], [np.nan, 0, 0]], np.float32)
    with pytest.raises(ValueError, match="-1"):
        O.VMap(O.as_pts4(bad), cov, [1.0])


def test_empty_source_and_misses():
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (3, 1))
    tgt = O.Frame(O.as_pts4(np.array([[0.1, 0.1, 0.1], [5.1, 0.1, 0.1], [0.2, 0.3, 0.4]])), cov)
    vm = O.VMap(tgt.pts4, tgt.cov6, [1.0])
    empty = O.Frame(np.zeros((0, 4), np.float32), np.zeros((0, 6), np.float32))
    poses = np.stack([np.eye(3, 4), np.eye(3, 4)])
    r = O.linearize([empty, tgt], [None, vm], [[0, 1]], poses)
    assert r["e"][0] == 0 and not r["H"].any() and not r["b"].any() and r["inliers"][0] == 0
    far = O.Frame(O.as_pts4(np.array([[50.0, 50.0, 50.0]])), cov[:1])
    r = O.linearize([far, tgt], [None, vm], [[0, 1]], poses)
    assert r["inliers"][0] == 0 and r["e"][0] == 0


# ---------------------------------------------------------------------------- surface validation
def test_surface_validation_thin_wall():
    """A thin wall seen from one side: a target viewpoint behind the wall discards every
    point, one on the same side keeps every point (Sec. III-C, Fig. 3)."""
    s = synth.Stream(21, "wall")
    n = 300
    p = np.stack([np.full(n, 2.0), s.uniform(n, -1, 1), s.uniform(n, -1, 1)], 1).astype(np.float32)
    normals = np.tile(np.array([[-1.0, 0.0, 0.0]], np.float32), (n, 1))  # facing the origin
    cov = np.tile(np.array([0.01, 0, 0, 1, 0, 1], np.float32), (n, 1))
    src = O.Frame(O.as_pts4(p), cov, normals)
    tgt = O.Frame(O.as_pts4(p), cov)
    vm = O.VMap(tgt.pts4, tgt.cov6, [0.5])
    Ts = np.eye(3, 4)
    for x_t, expect_keep in [(0.5, True), (3.5, False)]:
        Tt = np.eye(3, 4)
        Tt[0, 3] = x_t
        # shift the target cloud so the correspondences exist under this relative pose
        tgt_pts = p.copy()
        tgt_pts[:, 0] -= x_t
        vm = O.VMap(O.as_pts4(tgt_pts), cov, [0.5])
        r = O.linearize([src, O.Frame(O.as_pts4(tgt_pts), cov)], [None, vm], [[0, 1]],
                        np.stack([Ts, Tt]), validate=True)
        r_off = O.linearize([src, O.Frame(O.as_pts4(tgt_pts), cov)], [None, vm], [[0, 1]],
                            np.stack([Ts, Tt]), validate=False)
        assert r_off["inliers"][0] == n
        assert r["inliers"][0] == (n if expect_keep else 0)


def test_surface_validation_exact_rule(room):
    """The discard decision equals the FP32 rule evaluated exactly: d = mu - v in FP32,
    s = n_x d_x, s = fma(n_y, d_y, s), s = fma(n_z, d_z, s), discard if s > 0."""
    w, fr, vms = room
    poses = w.poses.copy()
    # random normals, so that both outcomes of the test occur
    nrm_rand = synth.Stream(22, "normals").unit_vectors(len(fr[0].pts4)).astype(np.float32)
    fr = [O.Frame(fr[0].pts4, fr[0].cov6, nrm_rand)] + fr[1:]
    r_on = O.linearize(fr, vms, w.pairs, poses, validate=True, want_ids=True)
    r_off = O.linearize(fr, vms, w.pairs, poses, validate=False, want_ids=True)
    T = O.compose(O.inverse(poses[1]), poses[0])
    v = (-T[:, :3].T @ T[:, 3]).astype(np.float32)
    L = vms[1].levels
    ids_on = r_on["ids"].reshape(-1, L)
    ids_off = r_off["ids"].reshape(-1, L)
    pts, nrm = fr[0].pts4, fr[0].normal3
    n_drop = 0
    for k in range(len(pts)):
        d = [X.sub(pts[k][a], v[a]) for a in range(3)]
        sacc = X.mul(nrm[k][0], d[0])
        sacc = X.fma(nrm[k][1], d[1], sacc)
        sacc = X.fma(nrm[k][2], d[2], sacc)
        if sacc > 0:
            n_drop += 1
            assert (ids_on[k] == -1).all()
        else:
            assert (ids_on[k] == ids_off[k]).all()
    assert 0.2 * len(pts) < n_drop < 0.8 * len(pts)


# ---------------------------------------------------------------------------- structure of H, b
def test_H_symmetric_psd(room):
    w, fr, vms = room
    r = O.linearize(fr, vms, w.pairs, w.poses)
    H = r["H"][0]
    nrm = np.linalg.norm(H)
    assert np.abs(H - H.T).max() <= 1e-12 * nrm
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() >= -1e-10 * nrm


def _fd_grad(fun, x0, h):
    g = np.zeros_like(x0)
    for i in range(len(x0)):
        xp, xm = x0.copy(), x0.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def test_b_is_half_gradient_of_e(room):
    """Central finite differences of e (Omega and correspondences frozen at the
    linearization point) w.r.t. right perturbations of both poses equal 2 b."""
    w, fr, vms = room
    r = O.linearize(fr, vms, w.pairs, w.poses, want_ids=True)

    def e_of(x):
        P = w.poses.copy()
        P[0] = O.retract(P[0], x[:6])
        P[1] = O.retract(P[1], x[6:])
        return O.energy(fr, vms, w.pairs, P, r["ids"], omega_poses=w.poses)[0]

    g = _fd_grad(e_of, np.zeros(12), 1e-6)
    scale = np.abs(2 * r["b"][0]).max()
    np.testing.assert_allclose(g, 2 * r["b"][0], atol=1e-5 * scale)
    assert abs(e_of(np.zeros(12)) - r["e"][0]) <= 1e-12 * r["e"][0]


def test_H_is_half_hessian_at_zero_residual():
    """With every voxel mean equal to its transformed source point (d = 0), the second
    derivative of e (Omega and correspondences frozen) is exactly 2 H."""
    s = synth.Stream(31, "zres")
    n = 40
    pts = s.uniform(3 * n, -3, 3).reshape(n, 3).astype(np.float32)
    cov = []
    for _ in range(n):
        A = s.normal(9).reshape(3, 3)
        Cm = A @ A.T + 0.2 * np.eye(3)
        cov.append([Cm[0, 0], Cm[0, 1], Cm[0, 2], Cm[1, 1], Cm[1, 2], Cm[2, 2]])
    cov = np.array(cov, np.float32)
    # identical poses => T_rel = I and target = source: each point sits alone in a 0.05 m voxel
    T = synth.make_pose(synth.rot_axis_angle([1, 2, 3], 0.9), [4.0, -2.0, 1.0])
    poses = np.stack([T, T])
    fr = [O.Frame(O.as_pts4(pts), cov), O.Frame(O.as_pts4(pts), cov)]
    vm = O.VMap(fr[1].pts4, fr[1].cov6, [0.05])
    assert vm.size(0) == n
    r = O.linearize(fr, [None, vm], [[0, 1]], poses, want_ids=True)
    assert r["inliers"][0] == n and r["e"][0] < 1e-20

    def e_of(x):
        P = poses.copy()
        P[0] = O.retract(P[0], x[:6])
        P[1] = O.retract(P[1], x[6:])
        return O.energy(fr, [None, vm], [[0, 1]], P, r["ids"], omega_poses=poses)[0]

    h = 1e-4
    Hfd = np.zeros((12, 12))
    for i in range(12):
        for j in range(i, 12):
            def ev(a, b):
                x = np.zeros(12)
                x[i] += a
                x[j] += b
                return e_of(x)
            Hfd[i, j] = Hfd[j, i] = (ev(h, h) - ev(h, -h) - ev(-h, h) + ev(-h, -h)) / (4 * h * h)
    H = r["H"][0]
    np.testing.assert_allclose(0.5 * Hfd, H, atol=2e-5 * np.abs(H).max())


# ---------------------------------------------------------------------------- gauge symmetry
def _adjoint(T):
    R, t = T[:, :3], T[:, 3]
    Ad = np.zeros((6, 6))
    Ad[:3, :3] = R
    Ad[3:, 3:] = R
    Ad[3:, :3] = O.hat(t) @ R
    return Ad


def test_gauge_invariance_and_null_space(room):
    w, fr, vms = room
    r = O.linearize(fr, vms, w.pairs, w.poses, want_ids=True)
    G = synth.make_pose(synth.rot_axis_angle([0.2, 0.9, -0.4], 1.3), [10.0, -7.0, 3.0])
    P2 = np.stack([O.compose(G, w.poses[0]), O.compose(G, w.poses[1])])
    r2 = O.linearize(fr, vms, w.pairs, P2, want_ids=True)
    assert (r["ids"] == r2["ids"]).all()
    assert abs(r2["e"][0] - r["e"][0]) <= 1e-10 * r["e"][0]
    np.testing.assert_allclose(r2["H"][0], r["H"][0], atol=1e-10 * np.abs(r["H"][0]).max())
    np.testing.assert_allclose(r2["b"][0], r["b"][0], atol=1e-10 * np.abs(r["b"][0]).max())
    H, b = r["H"][0], r["b"][0]
    s = synth.Stream(41, "gauge")
    for _ in range(4):
        zeta = s.normal(6)
        v = np.concatenate([_adjoint(O.inverse(w.poses[0])) @ zeta, _adjoint(O.inverse(w.poses[1])) @ zeta])
        assert np.linalg.norm(H @ v) <= 1e-10 * np.linalg.norm(H) * np.linalg.norm(v)
        assert abs(b @ v) <= 1e-10 * np.linalg.norm(b) * np.linalg.norm(v) * 10


# ---------------------------------------------------------------------------- special cases
def _kabsch(P, Q, w):
    """Weighted rigid fit Q ~ R P + t (Horn 1987 / Kabsch 1976, SVD form)."""
    w = w / w.sum()
    cp, cq = w @ P, w @ Q
    Hm = ((P - cp) * w[:, None]).T @ (Q - cq)
    U, _, Vt = np.linalg.svd(Hm)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return R, cq - R @ cp


def test_omega_identity_reduces_to_kabsch(room):
    """With Omega = I and frozen correspondences, Gauss-Newton on the unary factor converges
    to the closed-form rigid fit between the source points and their voxel means."""
    w, fr, vms = room
    r = O.linearize(fr, vms, w.pairs, w.poses, want_ids=True)
    ids = r["ids"]
    L = vms[1].levels
    P, Q, W = [], [], []
    for l in range(L):
        means = vms[1].export(l)["mean"]
        idl = ids.reshape(-1, L)[:, l]
        sel = idl >= 0
        P.append(fr[0].pts4[sel, :3].astype(np.float64))
        Q.append(means[idl[sel]])
        W.append(fr[0].pts4[sel, 3].astype(np.float64))
    R_star, t_star = _kabsch(np.concatenate(P), np.concatenate(Q), np.concatenate(W))
    poses = w.poses.copy()
    for _ in range(30):
        rr = O.linearize(fr, vms, w.pairs, poses, omega_identity=True, ids_in=ids)
        xi = O.gn_solve(rr["H"][0][:6, :6], rr["b"][0][:6])
        poses[0] = O.retract(poses[0], xi)
    T = O.compose(O.inverse(poses[1]), poses[0])
    np.testing.assert_allclose(T[:, :3], R_star, atol=1e-9)
    np.testing.assert_allclose(T[:, 3], t_star, atol=1e-9)


def test_gn_recovers_known_pose_noiseless():
    """Noiseless box room: 10 Gauss-Newton iterations of the unary factor from a 5 degree /
    0.3 m perturbation recover the true pose within 0.05 degree / 5 mm."""
    w = synth.box_room(sigma=0.0)
    fr = _frames_for(w)
    vm = O.VMap(fr[1].pts4, fr[1].cov6, w.resolutions)
    poses = w.poses.copy()
    for _ in range(10):
        r = O.linearize(fr, [None, vm], w.pairs, poses)
        poses[0] = O.retract(poses[0], O.gn_solve(r["H"][0][:6, :6], r["b"][0][:6]))
    D = O.compose(O.inverse(w.poses_true[0]), poses[0])
    ang = math.degrees(math.acos(min(1.0, (np.trace(D[:, :3]) - 1) / 2)))
    assert ang < 0.05 and np.linalg.norm(D[:, 3]) < 0.005


def test_gn_solve_against_library_and_not_pd():
    s = synth.Stream(51, "spd")
    for dim in (6, 12):
        A = s.normal(dim * dim).reshape(dim, dim)
        H = A @ A.T + dim * np.eye(dim)
        b = s.normal(dim)
        np.testing.assert_allclose(O.gn_solve(H, b), -np.linalg.solve(H, b), rtol=1e-12, atol=1e-12)
    H = np.zeros((6, 6))
    with pytest.raises(np.linalg.LinAlgError):
        O.gn_solve(H, np.ones(6))


# ---------------------------------------------------------------------------- covariances
def test_covariance_on_exact_plane():
    """Points exactly on the plane 4z = x + 2y + 2 (exact in FP32): the normal is the plane
    normal, C = I - (1 - eps) n n^T, and the kNN sets equal a full sort of the distances."""
    s = synth.Stream(61, "plane")
    n = 400
    x = np.round(s.uniform(n, -2, 2) * 256) / 256
    y = np.round(s.uniform(n, -2, 2) * 256) / 256
    z = (x + 2 * y + 2) / 4
    pts = np.stack([x, y, z], 1).astype(np.float32)
    assert np.array_equal(pts.astype(np.float64)[:, 2], (pts[:, 0].astype(np.float64) + 2 * pts[:, 1] + 2) / 4)
    eps = 1e-3
    cov, nrm, knn, tie = O.estimate_covariances(pts, k=10, reg_mode=1, eps=eps)
    n_true = np.array([1.0, 2.0, -4.0]) / math.sqrt(21.0)
    p64 = pts.astype(np.float64)
    for i in range(n):
        ni = n_true if n_true @ p64[i] <= 0 else -n_true
        np.testing.assert_allclose(nrm[i], ni, atol=1e-9)
        Cexp = np.eye(3) - (1 - eps) * np.outer(ni, ni)
        np.testing.assert_allclose(cov[i], Cexp[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], atol=1e-9)
        d2 = np.sum((p64 - p64[i]) ** 2, axis=1)
        order = np.lexsort((np.arange(n), d2))[:10]
        assert list(knn[i]) == list(order)


def test_raw_covariance_and_normal_against_library():
    """reg_mode 0 is the 1/k sample covariance of the kNN set (+ eps I); the normal is the
    eigenvector of its smallest eigenvalue (numpy eigh), oriented towards the origin."""
    w = synth.box_room(n_src=300, n_tgt=300, sigma=0.02)
    pts = w.points[0]
    cov, nrm, knn, tie = O.estimate_covariances(pts, k=10, reg_mode=0, eps=1e-6)
    p64 = pts.astype(np.float64)
    for i in range(0, len(pts), 7):
        C = np.cov(p64[knn[i]].T, bias=True) + 1e-6 * np.eye(3)
        np.testing.assert_allclose(cov[i], C[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], atol=1e-12)
        if tie[i]:
            continue
        wv, V = np.linalg.eigh(C)
        n0 = V[:, 0] if V[:, 0] @ p64[i] <= 0 else -V[:, 0]
        np.testing.assert_allclose(nrm[i], n0, atol=1e-8)


# ---------------------------------------------------------------------------- gradients
@pytest.mark.parametrize("full", [False, True])
def test_gradient_against_fd(full):
    """Analytic dE/dxi, dE/dmu, dE/dw against central FD (h = 1e-6) of E with frozen
    correspondences; Omega frozen at the linearization point (full=False) or re-evaluated
    at the perturbed poses (full=True)."""
    w = synth.corridor(n_cur=400, kf_range=(600, 900), n_kf=2, weights=True)
    fr = _frames_for(w)
    vms = [None] + [O.VMap(f.pts4, f.cov6, w.resolutions) for f in fr[1:]]
    r = O.linearize(fr, vms, w.pairs, w.poses, want_ids=True)
    dxi, dmu, dw = O.gradient(fr, vms, w.pairs, w.poses, omega_grad_full=full)
    nf = len(fr)

    def E_of_xi(x):
        P = np.stack([O.retract(w.poses[f], x[6 * f:6 * f + 6]) for f in range(nf)])
        return O.energy(fr, vms, w.pairs, P, r["ids"], omega_poses=None if full else w.poses).sum()

    g = _fd_grad(E_of_xi, np.zeros(6 * nf), 1e-6)
    np.testing.assert_allclose(g.reshape(nf, 6), dxi, atol=2e-6 * np.abs(dxi).max())
    if not full:
        # Omega frozen: dE/dxi_s = 2 b_s summed over the pairs
        np.testing.assert_allclose(dxi[0], 2 * r["b"][:, :6].sum(0), rtol=1e-9, atol=1e-9)
    # point and weight gradients on a few points of the source frame
    base = fr[0].pts4.copy()
    for k in (0, 17, 123, 311):
        for a in range(4):
            def E_pt(hv):
                p = base.copy()
                p[k, a] += hv
                f2 = [O.Frame(p, fr[0].cov6, fr[0].normal3)] + fr[1:]
                return O.energy(f2, vms, w.pairs, w.poses, r["ids"]).sum()
            h = 1e-3 if a < 3 else 1e-2   # FP32 inputs: perturb by representable steps
            fd = (E_pt(h) - E_pt(-h)) / (2 * h)
            an = dmu[0][k, a] if a < 3 else dw[0][k]
            assert abs(fd - an) <= 1e-3 * max(1.0, abs(an)), (k, a, fd, an)


# ---------------------------------------------------------------------------- the oracle's error bar
def test_plain_vs_compensated_sums(room):
    w, fr, vms = room
    r = O.linearize(fr, vms, w.pairs, w.poses, want_comp=True)
    assert abs(r["e"][0] - r["comp_e"][0]) <= 1e-13 * r["e"][0]
    assert np.linalg.norm(r["H"][0] - r["comp_H"][0]) <= 1e-13 * np.linalg.norm(r["H"][0])


def test_threads_do_not_change_results(room):
    w, fr, vms = room
    pairs = np.array([[0, 1]] * 5, np.int32)
    r1 = O.linearize(fr, vms, pairs, w.poses, nthreads=1)
    r4 = O.linearize(fr, vms, pairs, w.poses, nthreads=4)
    assert np.array_equal(r1["H"], r4["H"]) and np.array_equal(r1["e"], r4["e"])


def test_overlap_rate_counts_hits(room):
    """Overlap (Sec. IV-B): the fraction of source points that fall in an occupied voxel."""
    w, fr, vms = room
    r = O.linearize(fr, vms, w.pairs, w.poses, want_ids=True)
    L = vms[1].levels
    ids = r["ids"].reshape(-1, L)
    for l in range(L):
        ov = O.overlap(fr[0], vms[1], w.poses[0], w.poses[1], level=l)
        assert ov == pytest.approx((ids[:, l] >= 0).mean(), abs=0)


# ---------------------------------------------------------------------------- graph step (Sec. V-A)
def _random_graph(seed, n, P):
    s = synth.Stream(seed, "graph-pin")
    pairs = []
    while len(pairs) < P:
        a, b_ = (int(v) for v in s.integers(2, 0, n))
        if a != b_:
            pairs.append((a, b_))
    return s, pairs


def test_graph_step_recovers_a_consistent_linear_model():
    """Each factor p is the Gauss-Newton form of the residual r_p(x) = A_p x_s + B_p x_t + c_p
    (H = J^T J, b = J^T c with J = [A_p, B_p]), where c_p = -(A_p x*_s + B_p x*_t) for fixed
    per-frame offsets x* with x*_0 = 0.  The stacked least-squares problem then has the exact
    solution x*, so the undamped step with frame 0 fixed must return x* (to rounding),
    whatever the pair order and directions."""
    n = 6
    s, pairs = _random_graph(3, n, 16)
    xs = s.normal(6 * n).reshape(n, 6)
    xs[0] = 0.0
    H, b = [], []
    for a, c in pairs:
        A = s.normal(3 * 6 * 3).reshape(9, 6)
        B = s.normal(3 * 6 * 3).reshape(9, 6)
        J = np.hstack([A, B])
        r = -(A @ xs[a] + B @ xs[c])
        H.append(J.T @ J)
        b.append(J.T @ r)
    xi, Hg, bg = O.graph_step(pairs, n, H, b, fixed=0)
    np.testing.assert_allclose(xi, xs, atol=1e-10)
    assert (xi[0] == 0).all()
    # the same graph with the pairs reversed (source and target swapped, blocks swapped)
    perm = np.r_[6:12, 0:6]
    H2 = [h[np.ix_(perm, perm)] for h in H[::-1]]
    b2 = [v[perm] for v in b[::-1]]
    xi2, Hg2, bg2 = O.graph_step([(c, a) for a, c in pairs[::-1]], n, H2, b2, fixed=0)
    np.testing.assert_allclose(xi2, xs, atol=1e-10)
    np.testing.assert_allclose(Hg2, Hg, rtol=1e-14, atol=1e-12)


def test_graph_step_assembly_is_the_sum_of_selected_blocks():
    """H_glob = sum_p E_p^T H_p E_p and b_glob = sum_p E_p^T b_p, with E_p the 12 x 6n matrix
    that selects the source and target variables of pair p; integer-valued factors make both
    sides exact."""
    n = 5
    s, pairs = _random_graph(4, n, 11)
    H = [np.round(s.normal(144).reshape(12, 12) * 8) for _ in pairs]
    b = [np.round(s.normal(12) * 8) for _ in pairs]
    Hn = np.zeros((6 * n, 6 * n))
    bn = np.zeros(6 * n)
    for (a, c), h, v in zip(pairs, H, b):
        E = np.zeros((12, 6 * n))
        E[0:6, 6 * a:6 * a + 6] = np.eye(6)
        E[6:12, 6 * c:6 * c + 6] = np.eye(6)
        Hn += E.T @ h @ E
        bn += E.T @ v
    # make the system positive definite so that the step exists; the assembly is checked as is
    Hpd = [h @ h.T + 12 * np.eye(12) for h in H]
    _, Hg, bg = O.graph_step(pairs, n, Hpd, b, fixed=2)
    Hn_pd = sum(np.block([[np.eye(6 * n)[:, 6 * a:6 * a + 6], np.eye(6 * n)[:, 6 * c:6 * c + 6]]]) @ h @
                np.block([[np.eye(6 * n)[:, 6 * a:6 * a + 6], np.eye(6 * n)[:, 6 * c:6 * c + 6]]]).T
                for (a, c), h in zip(pairs, Hpd))
    assert np.array_equal(Hg, Hn_pd)
    assert np.array_equal(bg, bn)


def test_graph_step_damping_closed_form_and_gauge():
    """One factor between two frames with a diagonal H, frame 0 fixed: the step of frame 1 is
    -b_t / ((1 + lambda) h_t) per variable.  Relative factors alone leave the gauge free: with
    no frame fixed the system is singular and the step is refused."""
    h = np.arange(1.0, 13.0)
    bvec = np.linspace(-3.0, 2.5, 12)
    for lam in (0.0, 0.5, 1e-3):
        xi, _, _ = O.graph_step([(0, 1)], 2, [np.diag(h)], [bvec], fixed=0, lam=lam)
        assert (xi[0] == 0).all()
        np.testing.assert_allclose(xi[1], -bvec[6:] / ((1 + lam) * h[6:]), rtol=1e-15)
    K = np.arange(1.0, 37.0).reshape(6, 6) + 6 * np.eye(6)
    J = np.hstack([K, -K])  # a relative residual: moving both frames together changes nothing
    with pytest.raises(np.linalg.LinAlgError):
        O.graph_step([(0, 1)], 2, [J.T @ J], [np.zeros(12)], fixed=-1)
    xi, _, _ = O.graph_step([(0, 1)], 2, [J.T @ J], [J.T @ np.ones(6)], fixed=0)
    np.testing.assert_allclose(K @ xi[1], np.ones(6), atol=1e-9)  # r = K x_0 - K x_1 + 1 = 0 with x_0 = 0


def test_covariances_at_queries_equal_the_full_brute_force():
    """The query-subset kNN (a k-heap over all points per query) gives, for every listed point,
    the same neighbour list, covariance, normal and near-tie flag as the full brute force (a
    partial sort of all distances), including points with exactly tied distances."""
    s = synth.Stream(21, "cov-at")
    pts = s.uniform(3 * 700, -2, 2).reshape(700, 3)
    pts[:100] = np.round(pts[:100] * 4) / 4  # a lattice patch: many exact distance ties
    for reg in (1, 0):
        c, n, knn, tie = O.estimate_covariances(pts, k=10, reg_mode=reg, eps=1e-3)
        q = np.array([0, 1, 5, 50, 99, 100, 333, 699])
        cq, nq, kq, tq = O.covariances_at(pts, q, k=10, reg_mode=reg, eps=1e-3)
        assert np.array_equal(kq, knn[q]) and np.array_equal(cq, c[q]) and np.array_equal(nq, n[q])
        assert np.array_equal(tq, tie[q])
    assert (kq[:, 0] == q).all()  # the point itself is its own nearest neighbour
