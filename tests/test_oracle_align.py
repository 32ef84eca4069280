"""Pins of the oracle's alignment loss, its derivatives and the Gauss-Newton
polish, against things other than the oracle itself: FP64 central
differences of the loss (in the pose, at a nonzero perturbation, and in the
node values), the closed form on affine fields where trilinear interpolation
is exact, and descent of the polish towards the true pose.
"""
import numpy as np
import pytest

import synth
from synth import Grid

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _orc():
    import oracle
    return oracle


def _room(noise=False):
    scene, fr = synth.room64_frame(0, noise=noise)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=0.0)
    vol = _orc().Volume(synth.ROOM64_GRID, tsdf, weight)
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    return vol, pts, fr


def _interior_points(vol, pts, poses, margin=0.02):
    """Points whose sample under every pose lies in a valid cell, at least
    `margin` voxels from every cell face (so the loss restricted to them is
    a smooth function of the pose over the poses given)."""
    g = vol.grid
    keep = np.ones(len(pts), dtype=bool)
    for T in poses:
        q = pts[:, :3] @ T[:3, :3].T + T[:3, 3]
        gc = (q - np.asarray(g.origin)) / g.voxel_size
        fr = gc - np.floor(gc)
        keep &= np.all((fr > margin) & (fr < 1 - margin), axis=1)
        for j in np.nonzero(keep)[0]:
            if _orc().sample(vol, q[j], band=True) is None:
                keep[j] = False
    return pts[keep]


def test_pose_gradient_matches_central_differences_at_a_nonzero_perturbation():
    o = _orc()
    vol, pts, fr = _room()
    xi0 = np.array([0.012, -0.02, 0.009, 0.011, 0.004, -0.007])
    h = 1e-6
    probes = [o.perturb_pose(fr.init_pose, xi0 + s * h * e) for e in np.eye(6) for s in (-1, 1)]
    sub = _interior_points(vol, pts, probes + [o.perturb_pose(fr.init_pose, xi0)])
    assert len(sub) > 2000
    r = o.align_loss(vol, sub, fr.init_pose, xi=xi0)
    assert r.count == len(sub)
    fd = np.empty(6)
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        fd[i] = (o.align_loss(vol, sub, fr.init_pose, xi=xi0 + e).loss -
                 o.align_loss(vol, sub, fr.init_pose, xi=xi0 - e).loss) / (2 * h)
    np.testing.assert_allclose(r.grad_xi, fd, rtol=2e-6, atol=1e-6 * np.abs(fd).max())


def test_tsdf_gradient_matches_central_differences():
    o = _orc()
    vol, pts, fr = _room()
    r = o.align_loss(vol, pts, fr.init_pose, grad_tsdf=True)
    nz = np.nonzero(np.abs(r.grad_tsdf) > 1e-3)[0]
    assert len(nz) > 100
    rng = np.random.default_rng(3)
    d = 1e-4
    for n in rng.choice(nz, 25, replace=False):
        if abs(vol.tsdf[n]) > 1 - 2 * d:
            continue
        v0 = vol.tsdf[n]
        vol.tsdf[n] = v0 + d
        lp = o.align_loss(vol, pts, fr.init_pose).loss
        vol.tsdf[n] = v0 - d
        lm = o.align_loss(vol, pts, fr.init_pose).loss
        vol.tsdf[n] = v0
        # the loss is quadratic in one node value: central differences are exact
        assert abs((lp - lm) / (2 * d) - r.grad_tsdf[n]) <= 1e-7 * max(1.0, abs(r.grad_tsdf[n]))
    # nodes of no valid sampled cell get nothing
    assert np.all(r.grad_tsdf[vol.weight == 0] == 0)


def test_loss_and_gradient_closed_form_on_an_affine_field():
    o = _orc()
    g = Grid(40, 36, 44, 0.05, 0.15, (-0.9, -0.8, 0.3))
    a = np.array([0.11, -0.07, 0.05])
    b = -0.13
    X = g.node_positions().reshape(-1, 3)
    vol = o.Volume(g, X @ a + b, np.ones(g.n_nodes))
    rng = np.random.default_rng(5)
    pts = rng.uniform([-0.4, -0.3, 0.9], [0.4, 0.3, 1.6], size=(500, 3))
    w = np.array([0.02, -0.03, 0.01])
    P = np.eye(4)
    P[:3, :3] = o.so3_exp(w)
    P[:3, 3] = [0.02, -0.01, 0.05]
    q = pts @ P[:3, :3].T + P[:3, 3]
    t = q @ a + b
    r = o.align_loss(vol, pts, P)
    assert r.count == len(pts)
    np.testing.assert_allclose(r.loss, np.sum(t * t), rtol=1e-12)
    # dL/dv = sum 2 t a ; dL/domega = sum 2 t (q x a)   (at xi = 0)
    np.testing.assert_allclose(r.grad_xi[3:], np.sum(2 * t) * a, rtol=1e-10)
    np.testing.assert_allclose(r.grad_xi[:3], np.sum(2 * t[:, None] * np.cross(q, a), axis=0), rtol=1e-10,
                               atol=1e-12)


def test_perturbation_is_on_the_left():
    o = _orc()
    P = np.eye(4)
    P[:3, :3] = o.so3_exp([0.1, 0.2, -0.3])
    P[:3, 3] = [0.5, -1.0, 2.0]
    xi = np.array([0.0, 0.0, np.pi / 2, 0.1, 0.2, 0.3])
    T = o.perturb_pose(P, xi)
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    np.testing.assert_allclose(T[:3, :3], Rz @ P[:3, :3], atol=1e-15)
    np.testing.assert_allclose(T[:3, 3], Rz @ P[:3, 3] + xi[3:], atol=1e-15)


def test_polish_descends_towards_the_true_pose():
    o = _orc()
    vol, pts, fr = _room()
    e0 = np.linalg.norm(fr.init_pose[:3, 3] - fr.gt_pose[:3, 3])
    P, acc, trace = o.polish(vol, pts, fr.init_pose, steps=10)
    assert acc >= 3
    assert np.all(np.diff(trace) <= 0), trace
    assert trace[-1] < 0.01 * trace[0]
    e1 = np.linalg.norm(P[:3, 3] - fr.gt_pose[:3, 3])
    R = P[:3, :3].T @ fr.gt_pose[:3, :3]
    ang = np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))
    # from 5 cm / 5 deg to within a quarter voxel (noise-free data)
    assert e0 > 0.04 and e1 < 0.25 * synth.ROOM64_GRID.voxel_size and ang < 0.2
    # the true pose is a fixed point: no candidate improves it materially
    P2, _, tr2 = o.polish(vol, pts, fr.gt_pose, steps=3)
    assert np.linalg.norm(P2[:3, 3] - fr.gt_pose[:3, 3]) < 0.1 * synth.ROOM64_GRID.voxel_size


def test_polish_damping_schedule_on_one_point_in_closed_form():
    """The damped Gauss-Newton schedule (lambda_0 = 1e-3, / 10 on an accepted
    step, x 10 on a rejected one, a candidate kept only if it lowers the mean
    squared residual, an invalid candidate never) on one point of an affine
    field f = a . X + b.  There H = J^T J has rank one, and the damped system
    (J^T J + lambda diag(J^2)) d = -r J has the closed-form solution
    d_i = -r / (J_i (lambda + 6)) (Sherman-Morrison; J = (q x a, a), every
    component nonzero), so the whole accept / reject sequence follows by hand
    from the step's closed form and Exp (scipy).  The field's zero level lies
    outside the grid: undamped steps overshoot (larger residual) or leave
    the grid (no valid cell), and the schedule has to raise lambda to 100
    before it moves again."""
    from scipy.spatial.transform import Rotation
    o = _orc()
    g = Grid(40, 40, 40, 0.05, 0.15, (-1.0, -1.0, -1.0))
    a, b = np.array([0.15, -0.1, 0.2]), 0.5           # node values in (0.05, 0.94): all inside the band
    X = g.node_positions().reshape(-1, 3)
    vol = o.Volume(g, X @ a + b, np.ones(g.n_nodes))
    q0 = np.array([0.12, 0.23, -0.09])

    def inside(q):
        gc = (q - np.array(g.origin)) / g.voxel_size
        return bool(np.all((gc >= 0) & (gc < g.nx - 1)))

    q, lam, r = q0.copy(), 1e-3, q0 @ a + b
    obj, decisions, trace = r * r, "", [r * r]
    for _ in range(14):
        J = np.concatenate([np.cross(q, a), a])
        d = -r / (J * (lam + 6.0))
        qc = Rotation.from_rotvec(d[:3]).apply(q) + d[3:]
        objc = (qc @ a + b) ** 2 if inside(qc) else np.inf
        assert not np.isfinite(objc) or abs(objc - obj) > 1e-3 * obj   # clear decisions only
        if objc < obj:
            q, r, obj, lam, decisions = qc, qc @ a + b, objc, lam / 10, decisions + "A"
        else:
            lam, decisions = lam * 10, decisions + "R"
        trace.append(obj)
    # accepts, rejects by overshoot, by leaving the grid, lambda up to 100 and down again
    assert decisions == "AARRRRRRRAARRR"
    P, accepted, tr = o.polish(vol, q0[None, :], np.eye(4), steps=14)
    assert accepted == decisions.count("A")
    np.testing.assert_allclose(tr, trace, rtol=1e-8)
    np.testing.assert_allclose(P[:3, :3] @ q0 + P[:3, 3], q, atol=1e-9)
