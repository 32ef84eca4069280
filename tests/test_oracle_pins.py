"""Pins of the FP64 oracle against closed forms, invariants and library routines.

Each test fixes the oracle to something other than itself: the analytic
scenes' exact geometry, fields on which trilinear interpolation is exact,
symmetries of the grid, textbook rotations (and scipy's), and closed-form
search trajectories on fields where the fitness is linear in the pose.
"""
import json
import os

import numpy as np
import pytest

import synth
from synth import Grid, Intrinsics

pytestmark = pytest.mark.usefixtures("oracle_lib")

HERE = os.path.dirname(os.path.abspath(__file__))


def _orc():
    import oracle
    return oracle


def affine_volume(grid, a, b, observed=None):
    """Volume whose node values are a . X + b (X = node position)."""
    X = grid.node_positions().reshape(-1, 3)
    t = X @ np.asarray(a, dtype=np.float64) + b
    w = np.ones(grid.n_nodes) if observed is None else observed.astype(np.float64)
    return _orc().Volume(grid, t, w)


def pose12(R, t):
    P = np.zeros((3, 4))
    P[:, :3] = R
    P[:, 3] = t
    return P.reshape(12)


# ---------------------------------------------------------------------------
# paper constants
# ---------------------------------------------------------------------------

def test_defaults_are_the_papers_constants():
    gold = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    p = _orc().TrackParams()
    assert p.beta == gold["beta"]["value"]
    assert p.s0_deg == gold["s0_deg"]["value"] and p.s0_cm == gold["s0_cm"]["value"]
    assert list(p.k_sched) == gold["k_sched"]["value"]
    assert list(p.decim_sched) == gold["decim_sched"]["value"]
    assert p.n_iters == gold["max_iters"]["value"]


# ---------------------------------------------------------------------------
# back-projection
# ---------------------------------------------------------------------------

def test_backprojected_points_lie_on_the_analytic_surface():
    scene = synth.room_scene(3)
    intr = Intrinsics(48, 36, 40.0, 44.0, 23.5, 17.0)
    P = synth.room_view(scene, 2)
    depth = synth.render_depth(scene, intr, P)
    pts = _orc().backproject(depth, intr)
    assert pts.shape[0] == np.count_nonzero(depth > 0)
    Xw = pts @ P[:3, :3].T + P[:3, 3]
    # float32 depth rounding is the only error: ~1e-7 relative
    assert np.max(np.abs(scene.sdf(Xw))) < 5e-6


def test_backprojection_tile_order():
    """Points follow 8 x 4-pixel tiles, row-major over tiles and inside each."""
    W, H = 19, 10
    intr = Intrinsics(W, H, 10.0, 10.0, 9.0, 4.5, 0.5, 3.0)
    d = (1.0 + np.arange(W * H, dtype=np.float32) / 1000.0).reshape(H, W)   # depth encodes the pixel
    d[3, 7] = 0.0
    pts = _orc().backproject(d, intr, 1)
    order = []
    for ty in range(0, H, 4):
        for tx in range(0, W, 8):
            for v in range(ty, min(ty + 4, H)):
                for u in range(tx, min(tx + 8, W)):
                    if d[v, u] > 0:
                        order.append((v, u))
    assert pts.shape[0] == len(order) == W * H - 1
    assert np.array_equal(pts[:, 2], np.array([d[v, u] for v, u in order], dtype=np.float64))
    for s in (3, 8):
        assert np.array_equal(_orc().backproject(d, intr, s), pts[::s])


def test_backprojection_validity_order_and_stride():
    intr = Intrinsics(5, 4, 10.0, 10.0, 2.0, 1.5, 0.5, 3.0)
    d = np.full((4, 5), 1.0, dtype=np.float32)
    d[0, 1] = 0.0
    d[1, 2] = np.nan
    d[2, 0] = np.inf
    d[3, 3] = 3.5       # beyond depth_max
    d[3, 4] = 0.49      # below depth_min
    d[2, 2] = 3.0       # exactly depth_max: usable
    d[0, 0] = 0.5       # exactly depth_min: usable
    full = _orc().backproject(d, intr, 1)
    # a 5 x 4 image is a single 8 x 4 tile: tile order is row-major here
    valid = [(v, u) for v in range(4) for u in range(5)
             if np.isfinite(d[v, u]) and 0.5 <= d[v, u] <= 3.0]
    assert full.shape[0] == len(valid) == 15
    # row-major order: the z values follow the image scan
    assert np.array_equal(full[:, 2], np.array([d[v, u] for v, u in valid], dtype=np.float64))
    # pixel (u, v) = (0, 0) at depth 0.5: x = (0 - 2) * 0.5 / 10, y = (0 - 1.5) * 0.5 / 10
    assert np.allclose(full[0], [-0.1, -0.075, 0.5], atol=0, rtol=1e-15)
    for s in (2, 3, 7, 16):
        assert np.array_equal(_orc().backproject(d, intr, s), full[::s])


# ---------------------------------------------------------------------------
# trilinear lookup
# ---------------------------------------------------------------------------

GRID_S = Grid(9, 7, 6, 0.1, 0.3, (-0.35, 0.2, 1.1))
A_FIELD = np.array([0.8, -1.3, 0.45])


def test_trilinear_is_exact_on_affine_fields():
    vol = affine_volume(GRID_S, A_FIELD, 0.25)
    rng = np.random.default_rng(0)
    lo = np.asarray(GRID_S.origin)
    ext = np.array([GRID_S.nx - 1, GRID_S.ny - 1, GRID_S.nz - 1]) * GRID_S.voxel_size
    for q in lo + rng.random((200, 3)) * ext * 0.999:
        v = _orc().sample(vol, q)
        assert v is not None
        assert abs(v - (A_FIELD @ q + 0.25)) < 1e-12


def test_trilinear_reproduces_node_values_and_bilinear_cross_terms():
    # f = x*y*z is trilinear, so interpolation is exact for it too
    g = Grid(4, 4, 4, 1.0, 1.0, (0.0, 0.0, 0.0))
    X = g.node_positions().reshape(-1, 3)
    vol = _orc().Volume(g, X[:, 0] * X[:, 1] * X[:, 2] * 0.01, np.ones(g.n_nodes))
    rng = np.random.default_rng(1)
    for q in rng.random((100, 3)) * 2.999:
        assert abs(_orc().sample(vol, q) - 0.01 * q[0] * q[1] * q[2]) < 1e-14
    assert _orc().sample(vol, np.array([1.0, 2.0, 1.0])) == pytest.approx(0.02, abs=1e-15)


def test_trilinear_bounds_are_half_open():
    vol = affine_volume(GRID_S, A_FIELD, 0.0)
    o = np.asarray(GRID_S.origin)
    vs = GRID_S.voxel_size
    last = np.array([GRID_S.nx - 1, GRID_S.ny - 1, GRID_S.nz - 1]) * vs
    assert _orc().sample(vol, o) is not None                                  # g = 0 is inside
    assert _orc().sample(vol, o + last) is None                              # g = n-1 is outside
    assert _orc().sample(vol, o + last - 1e-9) is not None
    assert _orc().sample(vol, o - np.array([1e-12, 0, 0])) is None


def test_one_unobserved_node_invalidates_exactly_its_eight_cells():
    g = Grid(6, 6, 6, 1.0, 1.0)
    obs = np.ones(g.n_nodes)
    hole = (3, 2, 2)
    obs[hole[0] + 6 * (hole[1] + 6 * hole[2])] = 0
    vol = affine_volume(g, [0.01, 0.02, 0.03], 0.0, obs)
    for k in range(5):
        for j in range(5):
            for i in range(5):
                touches = (i in (hole[0] - 1, hole[0]) and j in (hole[1] - 1, hole[1])
                           and k in (hole[2] - 1, hole[2]))
                v = _orc().sample(vol, np.array([i + 0.5, j + 0.5, k + 0.5]))
                assert (v is None) == touches


# ---------------------------------------------------------------------------
# fitness
# ---------------------------------------------------------------------------

def random_points(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    return lo + rng.random((n, 3)) * (hi - lo)


def test_constant_field_gives_its_magnitude():
    # 3/8 is exact in binary and successive linear interpolation of equal
    # values is exact, so the mean is exactly |c|
    vol = affine_volume(GRID_S, [0, 0, 0], -0.375)
    o = np.asarray(GRID_S.origin)
    pts = random_points(500, o + 0.05, o + 0.45, 2)
    poses = np.stack([pose12(np.eye(3), [0, 0, 0]), pose12(np.eye(3), [0.05, 0.02, 0.01])])
    r = _orc().fitness(vol, pts, poses)
    assert np.all(r.E == 0.375)
    assert np.all(r.C == 500)
    # a node at |tsdf| = 1 is outside the truncation band: its cells drop out
    vol2 = affine_volume(GRID_S, [0, 0, 0], 1.0)
    assert np.all(_orc().fitness(vol2, pts, poses).C == 0)


def test_fitness_equals_brute_force_mean_on_an_affine_field():
    a, b = np.array([2.0, -1.5, 3.1]), -5.0
    vol = affine_volume(GRID_S, a, b)
    o = np.asarray(GRID_S.origin)
    ext = np.array([8, 6, 5]) * 0.1
    pts = random_points(3000, np.array([-0.3, -0.3, -0.3]), np.array([0.3, 0.3, 0.3]), 3)
    rng = np.random.default_rng(4)
    poses = []
    for _ in range(6):
        R = synth.axis_angle_matrix(rng.normal(size=3), rng.uniform(0, 0.5))
        poses.append(pose12(R, o + ext * rng.uniform(0.3, 0.7, 3)))
    poses = np.stack(poses)
    r = _orc().fitness(vol, pts, poses)
    for k in range(len(poses)):
        T = poses[k].reshape(3, 4)
        q = pts @ T[:, :3].T + T[:, 3]
        g = (q - o) / 0.1
        inside = np.all((g >= 0) & (g < np.array([8, 6, 5])), axis=1)
        # a point counts when the field is inside the band at all 8 corners
        i0 = np.floor(g)
        band = np.ones(len(q), dtype=bool)
        for c in range(8):
            corner = o + 0.1 * (i0 + np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]))
            band &= np.abs(corner @ a + b) < 1
        keep = inside & band
        f = q @ a + b
        assert r.C[k] == np.count_nonzero(keep) > 100
        assert r.E[k] == pytest.approx(np.mean(np.abs(f[keep])), rel=1e-12)


def test_fitness_empty_and_stride():
    vol = affine_volume(GRID_S, A_FIELD, 0.0)
    P = pose12(np.eye(3), GRID_S.origin)
    r = _orc().fitness(vol, np.zeros((0, 3)), P[None])
    assert r.C[0] == 0 and np.isinf(r.E[0])
    far = _orc().fitness(vol, np.array([[100.0, 0, 0]]), P[None])
    assert far.C[0] == 0 and np.isinf(far.E[0])
    pts = random_points(101, np.zeros(3), np.array([0.7, 0.5, 0.4]), 5)
    for s in (2, 5, 50):
        a = _orc().fitness(vol, pts, P[None], stride=s)
        b = _orc().fitness(vol, pts[::s], P[None])
        assert a.C[0] == b.C[0] and a.S[0] == b.S[0]


def _room_setup(noise=False, view=0):
    scene, fr = synth.room64_frame(0, view=view, noise=noise)
    g = synth.ROOM64_GRID
    t, w = synth.analytic_tsdf(scene, g)
    vol = _orc().Volume(g, t, w)
    pts = _orc().backproject(fr.depth, synth.ROOM64_INTR)
    return scene, fr, g, vol, pts


def test_fitness_invariant_under_integer_voxel_translation():
    scene, fr, g, vol, pts = _room_setup()
    P = fr.init_pose
    r0 = _orc().fitness(vol, pts, P[:3, :4].reshape(1, 12))
    shift = np.array([3, -2, 5]) * g.voxel_size
    g2 = Grid(g.nx, g.ny, g.nz, g.voxel_size, g.trunc, tuple(np.asarray(g.origin) + shift))
    vol2 = _orc().Volume(g2, vol.tsdf, vol.weight)
    P2 = P.copy()
    P2[:3, 3] += shift
    r1 = _orc().fitness(vol2, pts, P2[:3, :4].reshape(1, 12))
    assert r1.C[0] == r0.C[0]
    assert r1.E[0] == pytest.approx(r0.E[0], rel=1e-12)


def test_fitness_invariant_under_axis_permutation():
    scene, fr, g, vol, pts = _room_setup()
    perm = (2, 0, 1)   # new axis a is old axis perm[a]
    T = vol.tsdf.reshape(g.nz, g.ny, g.nx)  # [k, j, i]
    W = vol.weight.reshape(g.nz, g.ny, g.nx)
    # array axes are (z, y, x); new (z', y', x') = old (perm[2], perm[1], perm[0])
    ax = tuple(2 - perm[2 - a] for a in range(3))
    vol2 = _orc().Volume(g, np.ascontiguousarray(T.transpose(ax)).reshape(-1),
                         np.ascontiguousarray(W.transpose(ax)).reshape(-1))
    Pm = np.eye(4)[list(perm)]          # maps old world coords to new
    P = fr.init_pose
    P2 = Pm @ P
    r0 = _orc().fitness(vol, pts, P[:3, :4].reshape(1, 12))
    r1 = _orc().fitness(vol2, pts, P2[:3, :4].reshape(1, 12))
    assert r1.C[0] == r0.C[0]
    assert r1.E[0] == pytest.approx(r0.E[0], rel=1e-12)


def test_fitness_invariant_under_axis_flip():
    """Mirroring the grid along x (node i -> n-1-i) and the sample positions
    with it (an improper 3x4 map) leaves every E_k unchanged: the trilinear
    weights of a mirrored position are the mirrored weights."""
    scene, fr, g, vol, pts = _room_setup()
    T = vol.tsdf.reshape(g.nz, g.ny, g.nx)[:, :, ::-1]
    W = vol.weight.reshape(g.nz, g.ny, g.nx)[:, :, ::-1]
    vol2 = _orc().Volume(g, np.ascontiguousarray(T).reshape(-1), np.ascontiguousarray(W).reshape(-1))
    c = g.origin[0] + 0.5 * (g.nx - 1) * g.voxel_size      # the mirror plane x = c
    F = np.eye(4)
    F[0, 0] = -1.0
    F[0, 3] = 2.0 * c
    poses = [fr.init_pose, fr.gt_pose, fr.gt_pose @ synth.perturbation(5, 0, 4.0, 4.0)]
    r0 = _orc().fitness(vol, pts, np.stack([P[:3, :4].reshape(12) for P in poses]))
    r1 = _orc().fitness(vol2, pts, np.stack([(F @ P)[:3, :4].reshape(12) for P in poses]))
    assert np.all(r0.C > 1000)
    assert np.array_equal(r1.C, r0.C)
    assert np.allclose(r1.E, r0.E, rtol=1e-12, atol=0)


def test_search_decisions_invariant_under_integer_voxel_translation():
    """The whole random optimization (pivot at the camera centre) on a scene,
    grid and trajectory shifted by whole voxels picks the same best particle
    and advantage set every iteration and ends at the shifted pose; the
    re-orthonormalised rotation is orthonormal to 1e-15."""
    scene, fr, g, vol, pts = _room_setup(noise=True)
    shift = np.array([3, -2, 5]) * g.voxel_size
    g2 = Grid(g.nx, g.ny, g.nz, g.voxel_size, g.trunc, tuple(np.asarray(g.origin) + shift))
    vol2 = _orc().Volume(g2, vol.tsdf, vol.weight)
    P0 = fr.init_pose
    P0s = P0.copy()
    P0s[:3, 3] += shift
    prm = _orc().TrackParams(n_iters=8, k_sched=(512, 512, 512), decim_sched=(2, 2, 2), update_mode=0,
                             compose_mode=1)
    templ = synth.templates(512, 3)
    r0 = _orc().track(vol, fr.depth, synth.ROOM64_INTR, templ, P0, prm)
    r1 = _orc().track(vol2, fr.depth, synth.ROOM64_INTR, templ, P0s, prm)
    assert not r0.lost and not r1.lost
    assert np.array_equal(r0.stats["best"], r1.stats["best"])
    assert np.array_equal(r0.stats["n_adv"], r1.stats["n_adv"])
    assert np.allclose(r1.stats["E0"], r0.stats["E0"], rtol=1e-9, atol=0)
    assert np.allclose(r1.pose[:3, :3], r0.pose[:3, :3], atol=1e-12)
    assert np.allclose(r1.pose[:3, 3], r0.pose[:3, 3] + shift, atol=1e-12)
    for res in (r0, r1):
        R = res.pose[:3, :3]
        assert np.abs(R @ R.T - np.eye(3)).max() <= 1e-15
        assert abs(np.linalg.det(R) - 1.0) <= 1e-15


def test_search_reaches_the_true_pose_on_a_noise_free_room():
    """The 160x120 room frame without noise, 1024 particles, 10 iterations,
    started 5 deg / 5 cm off: the final position is within one voxel (5 cm)
    of the truth, the rotation error below the starting 5 deg (about 1.4 deg
    on this 5 cm grid), and the frame's points sit at most half as far from
    their true positions as at the start."""
    scene, fr, g, vol, pts = _room_setup(noise=False)
    prm = _orc().TrackParams(n_iters=10, k_sched=(1024, 1024, 1024), decim_sched=(1, 1, 1), update_mode=0,
                             compose_mode=1)
    res = _orc().track(vol, fr.depth, synth.ROOM64_INTR, synth.templates(1024, 0), fr.init_pose, prm)
    dt = np.linalg.norm(res.pose[:3, 3] - fr.gt_pose[:3, 3])
    dR = res.pose[:3, :3].T @ fr.gt_pose[:3, :3]
    ang = np.degrees(np.arccos(np.clip((np.trace(dR) - 1) / 2, -1, 1)))
    assert dt < g.voxel_size and ang < 5.0
    X = np.c_[pts, np.ones(len(pts))]
    off = lambda P: np.sqrt(np.mean(np.sum((X @ (P - fr.gt_pose)[:3].T) ** 2, axis=1)))
    assert off(res.pose) < 0.5 * off(fr.init_pose)


def test_fitness_is_minimal_at_the_true_pose():
    scene, fr, g, vol, pts = _room_setup(noise=False)
    gt = fr.gt_pose
    e_gt = _orc().fitness(vol, pts, gt[:3, :4].reshape(1, 12)).E[0]
    poses = []
    for ax in range(3):
        for sgn in (-1, 1):
            d = np.eye(4)
            d[ax, 3] = sgn * g.voxel_size
            poses.append((gt @ d)[:3, :4].reshape(12))
            d = np.eye(4)
            axis = np.eye(3)[ax]
            d[:3, :3] = synth.axis_angle_matrix(axis, sgn * np.deg2rad(0.5))
            poses.append((gt @ d)[:3, :4].reshape(12))
    e = _orc().fitness(vol, pts, np.stack(poses)).E
    assert e_gt < 0.01
    assert np.all(e > e_gt)


# ---------------------------------------------------------------------------
# rotations and particles
# ---------------------------------------------------------------------------

def test_so3_exp_textbook_rotations():
    h = np.pi / 2
    Rx = _orc().so3_exp([h, 0, 0])
    assert np.allclose(Rx, [[1, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-15)
    Ry = _orc().so3_exp([0, h, 0])
    assert np.allclose(Ry, [[0, 0, 1], [0, 1, 0], [-1, 0, 0]], atol=1e-15)
    Rz = _orc().so3_exp([0, 0, h])
    assert np.allclose(Rz, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    assert np.allclose(_orc().so3_exp([np.pi, 0, 0]), np.diag([1, -1, -1]), atol=1e-15)
    assert np.array_equal(_orc().so3_exp([0, 0, 0]), np.eye(3))


def test_so3_exp_matches_scipy():
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(6)
    for w in rng.normal(size=(50, 3)) * np.array([[1.0]] * 25 + [[1e-9]] * 25):
        R = _orc().so3_exp(w)
        assert np.allclose(R, Rotation.from_rotvec(w).as_matrix(), atol=1e-14)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)


def test_particles_compose_on_the_left():
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    templ = synth.templates(16, 11)
    P = synth.look_at([1.0, 2.0, 1.5], [2.5, 1.0, 1.0])
    s_deg, s_cm = 7.0, 4.0
    for mode in (0, 1):
        T = _orc().particles(templ, 16, P, s_deg, s_cm, mode)
        assert np.array_equal(T[0], P[:3, :4].reshape(12))   # template 0 is the identity
        for k in range(1, 16):
            u = templ[k].astype(np.float64)
            dR = Rotation.from_rotvec(np.deg2rad(s_deg) * u[:3]).as_matrix()
            dt = s_cm / 100 * u[3:]
            if mode == 0:
                D = np.eye(4)
                D[:3, :3] = dR
                D[:3, 3] = dt
                ref = (D @ P)[:3, :4]
            else:
                ref = np.concatenate([dR @ P[:3, :3], (P[:3, 3] + dt)[:, None]], axis=1)
            assert np.allclose(T[k].reshape(3, 4), ref, atol=1e-14)


def test_templates_are_reproducible_and_in_range():
    a = synth.templates(4096, 5)
    assert np.array_equal(a, synth.templates(4096, 5))
    assert np.all(a[0] == 0) and np.all(np.abs(a[1:]) <= 1)
    assert abs(a[1:].mean()) < 0.02 and abs(a[1:].var() - 1 / 3) < 0.02
    assert not np.array_equal(a, synth.templates(4096, 6))
    # SplitMix64 published first output for seed 0 after one increment
    assert int(synth.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


# ---------------------------------------------------------------------------
# the search loop
# ---------------------------------------------------------------------------

def _linear_setup(update_mode, compose_mode=0, s0_deg=0.0):
    """Field f = a . X + b with every point inside the band, no rotation:
    E(P + dt) = E(P) + a . dt exactly."""
    g = Grid(40, 40, 40, 0.05, 0.15, (0.0, 0.0, 0.0))
    a = np.array([0.3, -0.2, 0.25])
    b = 0.1
    vol = affine_volume(g, a, b)
    intr = Intrinsics(8, 6, 8.0, 8.0, 3.5, 2.5, 0.1, 8.0)
    depth = np.full((6, 8), 0.8, dtype=np.float32)
    P0 = np.eye(4)
    P0[:3, 3] = [0.9, 1.0, 0.3]
    prm = _orc().TrackParams(n_iters=3, k_sched=(64, 64, 64), decim_sched=(1, 1, 1), s0_deg=s0_deg,
                             s0_cm=5.0, update_mode=update_mode, compose_mode=compose_mode)
    return vol, intr, depth, P0, prm, a, b


def test_search_closed_form_on_a_linear_field_mean_mode():
    vol, intr, depth, P0, prm, a, b = _linear_setup(0)
    templ = synth.templates(64, 21)
    pts = _orc().backproject(depth, intr)
    res = _orc().track(vol, depth, intr, templ, P0, prm)
    t = P0[:3, 3].copy()
    s = prm.s0_cm
    for it in range(3):
        Xw = pts + t
        f = Xw @ a + b
        assert np.all((f > 0) & (f < 1))
        E0 = f.mean()
        dts = s / 100 * templ[:, 3:].astype(np.float64)
        adv = dts[1:] @ a < 0            # E_k < E_0  <=>  a . dt_k < 0
        mu = dts[1:][adv].mean(axis=0)
        assert res.stats["n_adv"][it] == np.count_nonzero(adv)
        assert res.stats["E0"][it] == pytest.approx(E0, rel=1e-12)
        t = t + mu
        E_new = (pts + t) @ a + b
        assert res.stats["E_new"][it] == pytest.approx(E_new.mean(), rel=1e-12)
        assert np.allclose(res.stats["pose"][it].reshape(3, 4)[:, 3], t, atol=1e-14)
        assert res.stats["s"][it][1] == pytest.approx(s, rel=1e-14)
        s = (0.1 + 0.9 * E_new.mean()) * s
    assert np.allclose(res.pose[:3, 3], t, atol=1e-14)
    assert np.allclose(res.pose[:3, :3], np.eye(3), atol=1e-15)


def test_search_closed_form_on_a_linear_field_best_mode():
    vol, intr, depth, P0, prm, a, b = _linear_setup(1)
    templ = synth.templates(64, 22)
    pts = _orc().backproject(depth, intr)
    res = _orc().track(vol, depth, intr, templ, P0, prm)
    t = P0[:3, 3].copy()
    s = prm.s0_cm
    for it in range(3):
        dts = s / 100 * templ[:, 3:].astype(np.float64)
        proj = dts @ a
        kb = int(np.argmin(proj))
        assert res.stats["best"][it] == kb
        t = t + dts[kb]
        e = ((pts + t) @ a + b).mean()
        assert res.stats["E_best"][it] == pytest.approx(e, rel=1e-12)
        s = (0.1 + 0.9 * e) * s
    assert np.allclose(res.pose[:3, 3], t, atol=1e-14)


@pytest.mark.parametrize("compose_mode", [0, 1])
def test_search_closed_form_with_rotations_on_a_linear_field(compose_mode):
    """The rotation half of the advantage-set mean (Sec. III-B: rotations
    averaged in SO(3), read as the arithmetic mean of the rotation vectors
    then Exp): on a field f = a . X + b with every sample in the band, the
    fitness of any pose is E(R, t) = a . (R xbar + t) + b (xbar = the mean
    back-projected point), so the advantage set, its mean rotation vector and
    translation, the composed pose and the search size follow in closed form
    -- computed here with scipy's rotations, from the starting pose on."""
    from scipy.spatial.transform import Rotation
    g = Grid(40, 40, 40, 0.05, 0.15, (0.0, 0.0, 0.0))
    a, b = np.array([0.15, -0.1, 0.12]), 0.3         # node values in (0.1, 0.83): all inside the band
    vol = affine_volume(g, a, b)
    intr = Intrinsics(8, 6, 8.0, 8.0, 3.5, 2.5, 0.1, 8.0)
    depth = np.full((6, 8), 0.8, dtype=np.float32)
    R0 = Rotation.from_rotvec([0.2, -0.3, 0.1]).as_matrix()
    P0 = np.eye(4)
    P0[:3, :3] = R0
    P0[:3, 3] = [0.9, 1.0, 0.5]
    templ = synth.templates(64, 23)
    pts = _orc().backproject(depth, intr)
    xbar = pts.mean(axis=0)
    prm = _orc().TrackParams(n_iters=3, k_sched=(64, 64, 64), decim_sched=(1, 1, 1), s0_deg=8.0, s0_cm=5.0,
                             update_mode=0, compose_mode=compose_mode)
    res = _orc().track(vol, depth, intr, templ, P0, prm)
    R, t, s = R0.copy(), P0[:3, 3].copy(), np.array([8.0, 5.0])
    for it in range(3):
        w = np.deg2rad(s[0]) * templ[:, :3].astype(np.float64)
        dt = s[1] / 100 * templ[:, 3:].astype(np.float64)
        dR = Rotation.from_rotvec(w).as_matrix()
        Rk = dR @ R
        tk = (dR @ t if compose_mode == 0 else np.broadcast_to(t, (64, 3))) + dt
        for k in range(64):   # every sample of every particle lies inside the grid
            gc = (pts @ Rk[k].T + tk[k]) / g.voxel_size
            assert np.all((gc >= 0) & (gc < g.nx - 1))
        E = (Rk @ xbar + tk) @ a + b
        assert np.min(np.abs(E[1:] - E[0])) > 1e-5 * E[0]    # no decision within rounding of its threshold
        adv = E[1:] < E[0]
        assert res.stats["n_adv"][it] == np.count_nonzero(adv)
        assert res.stats["E0"][it] == pytest.approx(E[0], rel=1e-12)
        assert np.allclose(res.stats["s"][it], s, rtol=1e-14)
        mu_w, mu_t = w[1:][adv].mean(axis=0), dt[1:][adv].mean(axis=0)
        dRm = Rotation.from_rotvec(mu_w).as_matrix()
        R_wrong = R @ dRm                                   # the mean applied on the other side
        R, t = dRm @ R, (dRm @ t if compose_mode == 0 else t) + mu_t
        E_new = (R @ xbar + t) @ a + b
        assert res.stats["E_new"][it] == pytest.approx(E_new, rel=1e-12)
        got = res.stats["pose"][it].reshape(3, 4)
        assert np.max(np.abs(got[:, :3] - R)) < 1e-13 and np.max(np.abs(got[:, 3] - t)) < 1e-13
        assert np.max(np.abs(got[:, :3] - R_wrong)) > 1e-3   # the pin tells the sides apart
        s = (0.1 + 0.9 * E_new) * s
    assert np.max(np.abs(res.pose[:3, :3] - R)) < 1e-13 and np.max(np.abs(res.pose[:3, 3] - t)) < 1e-13


def test_search_size_closed_form_on_a_constant_field():
    g = Grid(30, 30, 30, 0.1, 0.3, (-1.5, -1.5, 0.0))
    c = 0.375          # exact in binary, so all particles tie exactly
    vol = affine_volume(g, [0, 0, 0], c)
    intr = Intrinsics(6, 5, 5.0, 5.0, 2.5, 2.0)
    depth = np.full((5, 6), 1.5, dtype=np.float32)
    for mode in (0, 1):
        prm = _orc().TrackParams(n_iters=8, k_sched=(32, 32, 32), decim_sched=(1, 1, 1), update_mode=mode)
        res = _orc().track(vol, depth, intr, synth.templates(32, 1), np.eye(4), prm)
        assert np.all(res.stats["n_adv"] == 0)                     # no particle is strictly better
        assert np.all(res.stats["best"] == 0)                      # ties go to the lowest index
        assert np.array_equal(res.pose, np.eye(4))
        fct = 0.1 + 0.9 * c
        assert np.allclose(res.stats["s"][:, 0], 10.0 * fct ** np.arange(8), rtol=1e-14)


def test_search_improves_the_fit_and_best_mode_is_monotone():
    scene, fr, g, vol, pts = _room_setup(noise=True)
    for mode in (0, 1):
        prm = _orc().TrackParams(n_iters=6, k_sched=(256, 256, 256), decim_sched=(4, 4, 4),
                                 update_mode=mode, compose_mode=1)
        res = _orc().track(vol, fr.depth, synth.ROOM64_INTR, synth.templates(256, 0), fr.init_pose, prm)
        E0 = res.stats["E0"]
        assert E0[-1] < 0.5 * E0[0]
        e_gt = _orc().fitness(vol, pts[::4], fr.gt_pose[:3, :4].reshape(1, 12)).E[0]
        e_init = _orc().fitness(vol, pts[::4], fr.init_pose[:3, :4].reshape(1, 12)).E[0]
        e_fin = _orc().fitness(vol, pts[::4], res.pose[:3, :4].reshape(1, 12)).E[0]
        assert e_gt <= e_fin < e_init
        if mode == 1:
            # the next iteration's particle 0 is the chosen particle (up to the
            # re-orthonormalisation, ~1e-16), so E never increases
            assert np.all(np.diff(E0) <= 1e-12)
            assert np.allclose(E0[1:], res.stats["E_best"][:-1], rtol=1e-12, atol=0)


def test_search_reports_lost_on_an_empty_frame():
    scene, fr, g, vol, pts = _room_setup()
    depth = np.zeros_like(fr.depth)
    res = _orc().track(vol, depth, synth.ROOM64_INTR, synth.templates(64, 0), fr.init_pose,
                       _orc().TrackParams(n_iters=3, k_sched=(64, 64, 64), decim_sched=(1, 1, 1)))
    assert res.lost and np.array_equal(res.pose, fr.init_pose)


# ---------------------------------------------------------------------------
# fusion
# ---------------------------------------------------------------------------

def _plane_case(d_plane=1.03, max_weight=255):
    g = Grid(16, 12, 24, 0.05, 0.12, (-0.4, -0.3, 0.2))
    intr = Intrinsics(64, 48, 60.0, 60.0, 31.5, 23.5)
    depth = np.full((48, 64), d_plane, dtype=np.float32)
    return g, intr, depth, _orc().Volume(g, max_weight=max_weight)


def _expected_plane(g, intr, d_plane):
    X = g.node_positions().reshape(-1, 3)
    z = X[:, 2]
    u = intr.fx * X[:, 0] / z + intr.cx
    v = intr.fy * X[:, 1] / z + intr.cy
    inimg = (np.floor(u + 0.5) >= 0) & (np.floor(u + 0.5) < intr.width) & \
            (np.floor(v + 0.5) >= 0) & (np.floor(v + 0.5) < intr.height) & (z > 0)
    sdf = np.float64(np.float32(d_plane)) - z
    upd = inimg & (sdf >= -g.trunc)
    return upd, np.minimum(1.0, sdf / g.trunc)


def test_fusion_of_a_fronto_parallel_plane_is_the_clamped_distance():
    g, intr, depth, vol = _plane_case()
    _orc().integrate(vol, depth, intr, np.eye(4))
    upd, t = _expected_plane(g, intr, 1.03)
    assert np.count_nonzero(upd) > 1000
    assert np.array_equal(vol.weight > 0, upd)
    assert np.allclose(vol.tsdf[upd], t[upd], atol=1e-15)
    assert np.all(vol.tsdf[~upd] == 1.0)


def test_fusion_running_average_and_weight_cap():
    g, intr, depth, vol = _plane_case(max_weight=3)
    d2 = np.full_like(depth, 1.07)
    _orc().integrate(vol, depth, intr, np.eye(4))
    _orc().integrate(vol, d2, intr, np.eye(4))
    u1, t1 = _expected_plane(g, intr, 1.03)
    u2, t2 = _expected_plane(g, intr, 1.07)
    both = u1 & u2
    assert np.allclose(vol.tsdf[both], 0.5 * (t1[both] + t2[both]), atol=1e-15)
    assert np.all(vol.weight[both] == 2)
    for _ in range(3):
        _orc().integrate(vol, d2, intr, np.eye(4))
    assert np.all(vol.weight[both] == 3)
    # after the cap, each new sample enters with weight 1/(3+1)
    w_before = vol.tsdf[both].copy()
    _orc().integrate(vol, depth, intr, np.eye(4))
    assert np.allclose(vol.tsdf[both], (3 * w_before + t1[both]) / 4, atol=1e-15)


def test_fusion_single_pixel_updates_only_its_cone():
    g, intr, _, vol = _plane_case()
    depth = np.zeros((48, 64), dtype=np.float32)
    pu, pv = 40, 13
    depth[pv, pu] = 1.1
    P = synth.look_at([0.05, -0.02, -0.1], [0.0, 0.0, 1.0], up=(0.0, -1.0, 0.0))
    _orc().integrate(vol, depth, intr, P)
    X = g.node_positions().reshape(-1, 3)
    Xc = (X - P[:3, 3]) @ P[:3, :3]
    u = np.floor(intr.fx * Xc[:, 0] / Xc[:, 2] + intr.cx + 0.5)
    v = np.floor(intr.fy * Xc[:, 1] / Xc[:, 2] + intr.cy + 0.5)
    upd = vol.weight > 0
    assert np.count_nonzero(upd) > 0
    assert np.all((u[upd] == pu) & (v[upd] == pv) & (Xc[upd, 2] > 0))


def test_fused_room_has_the_sign_of_the_true_distance():
    scene = synth.room_scene(1)
    g = Grid(48, 48, 48, 0.0667, 0.2, (0.0, 0.0, 0.0))
    intr = Intrinsics(80, 60, 70.0, 70.0, 39.5, 29.5)
    vol = _orc().Volume(g)
    for view in range(8):
        P = synth.room_view(scene, view)
        _orc().integrate(vol, synth.render_depth(scene, intr, P), intr, P)
    sd = scene.sdf(g.node_positions().reshape(-1, 3))
    obs = vol.weight > 0
    far = np.abs(sd) > 0.75 * g.voxel_size
    assert np.count_nonzero(obs & far) > 10000
    assert np.all(np.sign(vol.tsdf[obs & far]) == np.sign(sd[obs & far]))
    # values near the surface approximate the true distance along view rays
    near = obs & (np.abs(sd) < 0.5 * g.trunc)
    assert np.median(np.abs(vol.tsdf[near] * g.trunc - sd[near])) < 0.25 * g.voxel_size


def _fused_room(scene, g):
    fuse = Intrinsics(160, 120, 140.0, 140.0, 79.5, 59.5)
    vol = _orc().Volume(g)
    for view in range(8):
        P = synth.room_view(synth.room_scene(2), view)
        _orc().integrate(vol, synth.render_depth(scene, fuse, P), fuse, P)
    return vol


@pytest.mark.parametrize("with_spheres", [False, True])
def test_raycast_recovers_the_analytic_depth(with_spheres):
    full = synth.room_scene(2)
    scene = full if with_spheres else synth.Scene("walls", full.prims[:1])
    # the grid extends 20 cm beyond the walls so that the band behind them exists
    g = Grid(72, 72, 72, 0.05, 0.15, (-0.2, -0.2, -0.2))
    intr = Intrinsics(40, 30, 35.0, 35.0, 19.5, 14.5)
    vol = _fused_room(scene, g)
    P = synth.room_view(full, 0)
    truth = synth.render_depth(scene, intr, P)
    depth, normals = _orc().raycast(vol, intr, P)
    hit = depth > 0
    # pixels near the border look through parts of the band whose nodes
    # project outside every fused image; check the interior
    inner = np.zeros_like(hit)
    inner[3:-3, 3:-3] = True
    assert np.count_nonzero(hit & inner) > 0.9 * np.count_nonzero(inner)
    err = np.abs(depth - truth)[hit & inner]
    # silhouette pixels of the spheres may land on either side of the edge
    assert np.mean(err < 0.5 * g.voxel_size) > (0.93 if with_spheres else 0.999)
    assert np.median(err) < 0.1 * g.voxel_size
    # normals point against the viewing ray
    ok = np.isfinite(normals[..., 0]) & hit
    uu, vv = np.meshgrid(np.arange(40), np.arange(30))
    rays = np.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy, np.ones_like(uu, dtype=float)], -1)
    rays_w = rays @ P[:3, :3].T
    assert np.mean(np.sum(normals[ok] * rays_w[ok], axis=-1) < 0) > 0.98
    if not with_spheres:
        # wall normals are the axis directions
        n = normals[ok & inner]
        assert np.mean(np.max(np.abs(n), axis=-1) > 0.97) > 0.9


def test_fusion_of_a_tiny_grid_matches_the_hand_worked_example():
    """4^3 nodes, a 3x3 image, two views (constant depth, then depth that
    differs by image column, so that the nearest-pixel rounding decides
    values): every node's tsdf and weight after each view, worked by hand
    from the fusion rule (fixture tests/golden/fusion_tiny_grid.json, with
    its derivation)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "fusion_tiny_grid.json")) as fh:
        fx = json.load(fh)
    g, c = fx["grid"], fx["camera"]
    grid = synth.Grid(*g["n"], g["voxel"], g["trunc"], tuple(g["origin"]))
    intr = synth.Intrinsics(c["width"], c["height"], c["fx"], c["fy"], c["cx"], c["cy"], c["depth_min"], c["depth_max"])
    vol = _orc().Volume(grid)
    for row, exp in zip(fx["depth_rows"], fx["expected"]):
        depth = np.tile(np.asarray(row, dtype=np.float32), (3, 1))   # the same depth in every image row
        _orc().integrate(vol, depth, intr, np.eye(4))
        tsdf = vol.tsdf.reshape(4, 4, 4)      # [k, j, i]: x fastest
        weight = vol.weight.reshape(4, 4, 4)
        for k in range(4):
            e = exp[f"k{k}"]
            mask = np.zeros((4, 4), dtype=bool)  # [j, i]
            if e["ij"] == "all":
                mask[:] = True
            for i, j in ([] if e["ij"] == "all" else e["ij"]):
                mask[j, i] = True
            want = np.array([num / den for num, den in e["tsdf_by_i"]])[None, :].repeat(4, axis=0)
            assert np.all(weight[k][mask] == e["weight"]), (row, k)
            assert np.allclose(tsdf[k][mask], want[mask], rtol=0, atol=1e-12), (row, k)
            assert np.all(weight[k][~mask] == 0) and np.all(tsdf[k][~mask] == 1.0), (row, k)
