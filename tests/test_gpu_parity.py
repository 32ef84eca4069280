"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the figures the targets fix; only the plain float baseline layout
of the fitness adds an absolute floor of 2e-6, see test_fitness_parity):
  back-projection  point count and order exact; coordinates within 3e-7
                   relative (two float roundings);
  fusion           weights exact, tsdf within 1e-5 (units of the truncation);
  fitness          counts exact, E within 1e-5 relative (the product layouts
                   form sample positions from exact reference products; the
                   largest error measured over every case is 8.6e-7);
  search           same best-particle index and advantage-set size while the
                   oracle's decision margins exceed 1e-5; final pose within
                   1e-4 m and 1e-4 rad.
Elements whose discrete decision lies within the oracle-computed margin of
its threshold (a pixel-rounding boundary, the -tau cut, a cell face across
which validity changes) may take either side; they are counted and bounded.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import Grid, Intrinsics

from gpu_helpers import (abi, compare_fitness, load_pf, perturbed_poses, pose_rot_err, pose_trans_err, to_dev,
                         torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    torch_cuda()
    return load_pf()


# ---------------------------------------------------------------------------
# back-projection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("size", [(160, 120), (173, 97)])
def test_backproject_parity(pf, size):
    W, H = size
    intr = Intrinsics(W, H, 140.0, 137.0, W / 2 - 0.3, H / 2 + 0.7, 0.3, 3.2)
    scene = synth.room_scene(4)
    depth = synth.add_depth_noise(synth.render_depth(scene, intr, synth.room_view(scene, 1)), 5, 0.01)
    rng = np.random.default_rng(9)
    idx = rng.choice(W * H, size=W * H // 10, replace=False)
    flat = depth.reshape(-1)
    flat[idx[0::4]] = 0.0
    flat[idx[1::4]] = np.nan
    flat[idx[2::4]] = np.inf
    flat[idx[3::4]] = 9.0
    flat[0] = 0.3   # exactly depth_min
    flat[1] = 3.2   # exactly depth_max
    pts, n = pf.backproject(to_dev(depth), intr)
    n = int(n.item())
    ref = oracle.backproject(depth, abi(intr))
    assert n == ref.shape[0]
    got = pts[:n].cpu().numpy().astype(np.float64)
    assert np.array_equal(got[:, 2], ref[:, 2])
    np.testing.assert_allclose(got[:, :2], ref[:, :2], rtol=3e-7, atol=1e-9)
    assert np.all(got[:, 3] == 0)


def test_backproject_empty(pf):
    intr = Intrinsics(33, 17, 20.0, 20.0, 16.0, 8.0)
    pts, n = pf.backproject(to_dev(np.zeros((17, 33), np.float32)), intr)
    assert int(n.item()) == 0


# ---------------------------------------------------------------------------
# fusion
# ---------------------------------------------------------------------------

FUSION_CASES = {
    "room64": (synth.ROOM64_GRID, synth.ROOM64_INTR, [0, 1, 2]),
    # ragged grid: partial tiles in every axis, origin off the lattice
    "ragged": (Grid(67, 45, 39, 0.061, 0.17, (0.07, 0.53, -0.21)), Intrinsics(97, 61, 80.0, 82.0, 47.3, 31.1),
               [3, 5, 0]),
}


def _fuse_both(pf, grid, intr, views, seed=0):
    scene = synth.room_scene(seed)
    vol = pf.Volume.from_grid(grid)
    ovol = oracle.Volume(abi(grid))
    amb = np.zeros(grid.n_nodes, dtype=bool)
    for j, view in enumerate(views):
        P = synth.room_view(scene, view)
        depth = synth.add_depth_noise(synth.render_depth(scene, intr, P), 50 + j, 0.002)
        vol.integrate(to_dev(depth), intr, P)
        amb |= oracle.integrate(ovol, depth, abi(intr), P, ambiguity=True, eps_px=3e-4).astype(bool)
    return vol, ovol, amb


@pytest.mark.parametrize("case", sorted(FUSION_CASES))
def test_integrate_parity(pf, case):
    grid, intr, views = FUSION_CASES[case]
    vol, ovol, amb = _fuse_both(pf, grid, intr, views)
    t, w = vol.download()
    ok = ~amb
    updated = ovol.weight > 0
    assert np.count_nonzero(updated) > 1000
    assert np.count_nonzero(amb) < 1e-2 * np.count_nonzero(updated)
    assert np.array_equal(w[ok], ovol.weight[ok].astype(np.float32))
    obs = ok & updated
    assert np.max(np.abs(t[obs].astype(np.float64) - ovol.tsdf[obs])) <= 1e-5
    assert np.all(t[ok & ~updated] == 1.0)


def test_integrate_camera_outside_and_behind(pf):
    grid = Grid(40, 40, 40, 0.05, 0.15, (0.0, 0.0, 0.0))
    intr = Intrinsics(64, 48, 50.0, 50.0, 31.5, 23.5)
    scene = synth.room_scene(0)
    # camera outside the grid looking away from it: nothing may change
    P = synth.look_at([-1.0, 1.0, 1.0], [-3.0, 1.0, 1.0])
    depth = np.full((48, 64), 2.0, dtype=np.float32)
    vol = pf.Volume.from_grid(grid)
    vol.integrate(to_dev(depth), intr, P)
    t, w = vol.download()
    assert np.all(w == 0) and np.all(t == 1.0)
    # camera inside, half the grid behind it
    P = synth.look_at([1.0, 1.0, 1.0], [2.0, 1.3, 0.9])
    depth = synth.render_depth(scene, intr, P)
    ovol = oracle.Volume(abi(grid))
    amb = oracle.integrate(ovol, depth, abi(intr), P, ambiguity=True, eps_px=3e-4).astype(bool)
    vol.integrate(to_dev(depth), intr, P)
    t, w = vol.download()
    ok = ~amb
    assert np.array_equal(w[ok], ovol.weight[ok].astype(np.float32))
    obs = ok & (ovol.weight > 0)
    assert np.max(np.abs(t[obs] - ovol.tsdf[obs])) <= 1e-5


def test_integrate_weight_cap(pf):
    grid = Grid(24, 20, 30, 0.05, 0.12, (-0.6, -0.5, 0.2))
    # non-round intrinsics: a grid seen head-on with round ones puts whole
    # lines of nodes exactly on half-pixel boundaries
    intr = Intrinsics(64, 48, 60.37, 59.81, 31.21, 23.67)
    vol = pf.Volume.from_grid(grid, max_weight=3)
    ovol = oracle.Volume(abi(grid), max_weight=3)
    amb = np.zeros(grid.n_nodes, dtype=bool)
    # plane depths chosen so that d + tau falls between node planes
    for d in (1.0312, 1.0731, 1.0119, 1.0527, 1.0443):
        depth = np.full((48, 64), d, dtype=np.float32)
        vol.integrate(to_dev(depth), intr, np.eye(4))
        amb |= oracle.integrate(ovol, depth, abi(intr), np.eye(4), ambiguity=True, eps_px=3e-4).astype(bool)
    t, w = vol.download()
    assert w.max() == 3
    # nodes projecting onto a half-pixel at the image border may go either way
    assert np.count_nonzero(amb) < 0.01 * grid.n_nodes
    assert np.array_equal(w[~amb], ovol.weight[~amb].astype(np.float32))
    obs = (ovol.weight > 0) & ~amb
    assert np.max(np.abs(t[obs] - ovol.tsdf[obs])) <= 1e-5


# ---------------------------------------------------------------------------
# fitness
# ---------------------------------------------------------------------------

def _room_inputs(seed=0, holes=0.03):
    scene, fr = synth.room64_frame(seed)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=holes, seed=seed)
    return scene, fr, tsdf, weight


@pytest.mark.parametrize("K,N,spread", [(1024, None, 8.0), (1024, None, 0.02), (1000, 12345, 3.0),
                                        (37, 777, 1.0), (1, 19200, 0.0)])
def test_fitness_parity(pf, K, N, spread):
    """Every kernel variant (plain / encoded / cell layout x lane mappings)
    against the oracle; the encoded and cell layouts are bit-identical for
    the same mapping (the plain form rounds its sample positions
    differently and ignores the mapping)."""
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    if N is not None:
        pts = pts[:N]
    poses = perturbed_poses(fr.gt_pose, K, spread, spread, seed=K)
    orc = oracle.fitness(ovol, pts, poses, ambiguity=True, cap=64)
    assert np.all(orc.amb <= 64)
    results = {}
    for mapping in range(3):
        for layout in (1, 2, 3):
            vol.set_fitness_variant(layout + 4 * mapping)
            E, C = vol.fitness(to_dev(pts), to_dev(poses))
            results[layout, mapping] = (E.cpu().numpy(), C.cpu().numpy())
            # the plain float form rounds each sample position once at the
            # scale of the grid coordinate: up to ~ulp(64)/2 = 2e-6 voxel per
            # coordinate, i.e. |dt| <= ~3 x 2e-6 x (vs / tau) = 2e-6 per sample
            compare_fitness(*results[layout, mapping], orc, floor=2e-6 if layout == 1 else 0.0)
        # the same mapping evaluates the same samples in the same order on
        # both layouts (the automatic mapping may differ between layouts)
        if mapping > 0:
            assert np.array_equal(results[3, mapping][0], results[2, mapping][0])
        assert np.array_equal(results[2, mapping][1], results[2, 0][1])
        assert np.array_equal(results[1, mapping][0], results[1, 0][0])


@pytest.mark.parametrize("case", sorted(FUSION_CASES))
def test_cell_view_follows_fusion(pf, case):
    """After fusing several views (tiles reached in different frames), the
    cell view gives bit-identical fitness to the node array it mirrors."""
    grid, intr, views = FUSION_CASES[case]
    vol, ovol, amb = _fuse_both(pf, grid, intr, views + [views[0]])
    scene = synth.room_scene(0)
    P = synth.room_view(scene, views[1])
    pts = synth.render_points(scene, intr, P)
    poses = perturbed_poses(P, 256, 4.0, 4.0, seed=7)
    out = {}
    for layout in (2, 3):
        vol.set_fitness_variant(layout + 4)   # points on lanes: same order on both layouts
        E, C = vol.fitness(to_dev(pts), to_dev(poses))
        out[layout] = (E.cpu().numpy(), C.cpu().numpy())
    assert np.count_nonzero(out[3][1]) > 100
    assert np.array_equal(out[2][0], out[3][0]) and np.array_equal(out[2][1], out[3][1])
    # a volume without the view falls back to the node array
    bare = pf.Volume.from_grid(grid, cell_view=-1)
    with pytest.raises(pf.ProfusionError):
        bare.set_fitness_variant(3)


def test_fitness_edge_cases(pf):
    torch = torch_cuda()
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    poses = perturbed_poses(fr.gt_pose, 5, 3.0, 3.0, seed=1)
    # no points
    E, C = vol.fitness(torch.zeros((0, 4), dtype=torch.float32, device="cuda"), to_dev(poses))
    assert torch.all(torch.isinf(E)) and torch.all(C == 0)
    # every point far outside the grid
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    far = poses.copy()
    far[:, 3] += 100.0
    E, C = vol.fitness(to_dev(pts), to_dev(far))
    assert torch.all(torch.isinf(E)) and torch.all(C == 0)
    # a fully unobserved volume
    vol2 = pf.Volume.from_grid(synth.ROOM64_GRID)
    E, C = vol2.fitness(to_dev(pts), to_dev(poses))
    assert torch.all(C == 0)


def test_fitness_at_the_maximum_pose_count(pf):
    """k = 65536, the largest pose count pf_fitness takes, over every point
    of a room-64 frame, against the oracle; k = 65537 is refused before
    anything runs."""
    torch = torch_cuda()
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    poses = perturbed_poses(fr.gt_pose, 65536, 5.0, 5.0, seed=77)
    E, C = vol.fitness(to_dev(pts), to_dev(poses))
    orc = oracle.fitness(ovol, pts, poses, ambiguity=True, cap=64)
    assert np.all(orc.amb <= 64)
    compare_fitness(E.cpu().numpy(), C.cpu().numpy(), orc)
    too_many = torch.zeros((65537, 12), dtype=torch.float32, device="cuda")
    with pytest.raises(pf.ProfusionError):
        vol.fitness(to_dev(pts), too_many)


def test_fitness_is_deterministic(pf):
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    pts = to_dev(synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose))
    poses = to_dev(perturbed_poses(fr.gt_pose, 3072, 10.0, 10.0, seed=3))
    E1, C1 = vol.fitness(pts, poses)
    E2, C2 = vol.fitness(pts, poses)
    assert np.array_equal(E1.cpu().numpy(), E2.cpu().numpy())
    assert np.array_equal(C1.cpu().numpy(), C2.cpu().numpy())


def test_volume_upload_download_roundtrip(pf):
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    t, w = vol.download()
    assert np.array_equal(w, weight)
    obs = weight > 0
    assert np.array_equal(t[obs], tsdf[obs]) and np.all(t[~obs] == 1.0)


# ---------------------------------------------------------------------------
# the search
# ---------------------------------------------------------------------------

def _track_both(pf, update_mode, compose_mode, K=1024, iters=10, decim=1, seed=0):
    torch = torch_cuda()
    scene, fr, tsdf, weight = _room_inputs(seed, holes=0.0)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    templ = synth.templates(K, seed)
    tdev = torch.from_numpy(templ).cuda()
    params = pf.track_params(tdev, n_iters=iters, k_sched=(K, K, K), decim_sched=(decim,) * 3,
                             update_mode=update_mode, compose_mode=compose_mode)
    status, pose, st = vol.track_frame(to_dev(fr.depth), synth.ROOM64_INTR, params, fr.init_pose)
    oparams = oracle.TrackParams(n_iters=iters, k_sched=(K, K, K), decim_sched=(decim,) * 3,
                                 update_mode=update_mode, compose_mode=compose_mode)
    ores = oracle.track(ovol, fr.depth, abi(synth.ROOM64_INTR), templ, fr.init_pose, oparams)
    return status, pose, st, ores, fr


@pytest.mark.parametrize("update_mode,compose_mode", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_track_parity(pf, update_mode, compose_mode):
    status, pose, st, ores, fr = _track_both(pf, update_mode, compose_mode)
    assert status == pf.PF_OK and not ores.lost
    os_ = ores.stats
    assert st["n_iters"] == os_["n_iters"] == 10
    assert st["n_points"] == os_["n_points"]
    strict = 0
    for i in range(10):
        clear = os_["best_gap"][i] > 3e-5 and (update_mode == 1 or os_["adv_margin"][i] > 3e-5)
        if not clear:
            break
        strict += 1
        assert st["best"][i] == os_["best"][i], i
        if os_["adv_margin"][i] > 3e-5:
            assert st["n_adv"][i] == os_["n_adv"][i], i
        assert abs(st["E0"][i] - os_["E0"][i]) <= 1e-5 * os_["E0"][i]
        np.testing.assert_allclose(st["s"][i], os_["s"][i], rtol=1e-5)
        np.testing.assert_allclose(st["pose"][i], os_["pose"][i], atol=1e-5)
    assert strict >= 2, "the oracle's first iterations should be unambiguous for this seed"
    assert pose_trans_err(pose, ores.pose) <= 1e-4
    assert pose_rot_err(pose, ores.pose) <= 1e-4


def test_track_lost_on_empty_frame(pf):
    torch = torch_cuda()
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    tdev = torch.from_numpy(synth.templates(64, 0)).cuda()
    params = pf.track_params(tdev, n_iters=4, k_sched=(64, 64, 64), decim_sched=(1, 1, 1))
    status, pose, st = vol.track_frame(to_dev(np.zeros_like(fr.depth)), synth.ROOM64_INTR, params, fr.init_pose)
    assert status == pf.PF_ERR_TRACK_LOST
    assert np.array_equal(pose, fr.init_pose)
    assert st["n_points"] == 0 and st["status"] == pf.PF_ERR_TRACK_LOST
    # the same with a decimated schedule: no point is kept at any stride
    params = pf.track_params(tdev, n_iters=3, k_sched=(64, 64, 64), decim_sched=(8, 16, 32))
    status, pose, st = vol.track_frame(to_dev(np.zeros_like(fr.depth)), synth.ROOM64_INTR, params, fr.init_pose)
    assert status == pf.PF_ERR_TRACK_LOST and np.array_equal(pose, fr.init_pose)
    assert st["n_points"] == 0 and st["status"] == pf.PF_ERR_TRACK_LOST


def test_track_decimated_schedule_on_a_ragged_image(pf):
    """Strides 3 / 7 / 13 on a 173 x 97 image (partial tiles on both edges,
    blocks of tiles cut by the image border): the kept points, evaluated in
    their locality order, give the oracle's counts, E0, best index and pose."""
    torch = torch_cuda()
    scene = synth.room_scene(1)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=0.0, seed=1)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    intr = Intrinsics(173, 97, 150.0, 148.0, 86.2, 48.7, 0.1, 8.0)
    gt = synth.room_view(scene, 1)
    depth = synth.render_depth(scene, intr, gt)
    init = gt @ synth.perturbation(41, 0, 3.0, 3.0)
    templ = synth.templates(1024, 3)
    ks, ds = (256, 512, 1024), (3, 7, 13)
    params = pf.track_params(torch.from_numpy(templ).cuda(), n_iters=6, k_sched=ks, decim_sched=ds,
                             update_mode=1, compose_mode=1)
    status, pose, st = vol.track_frame(to_dev(depth), intr, params, init)
    ores = oracle.track(ovol, depth, abi(intr), templ, init,
                        oracle.TrackParams(n_iters=6, k_sched=ks, decim_sched=ds, update_mode=1, compose_mode=1))
    assert status == pf.PF_OK and not ores.lost
    os_ = ores.stats
    assert list(st["n_eval"]) == list(os_["n_eval"])
    strict = 0
    for i in range(6):
        if not os_["best_gap"][i] > 3e-5:
            break
        strict += 1
        assert st["best"][i] == os_["best"][i], i
        assert st["n_valid0"][i] == os_["n_valid0"][i], i
        assert abs(st["E0"][i] - os_["E0"][i]) <= 1e-5 * os_["E0"][i], i
    assert strict >= 2
    assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4


def test_track_decimated_schedule(pf):
    """Alternating particle counts and point strides (the paper's schedule shape)."""
    torch = torch_cuda()
    scene, fr, tsdf, weight = _room_inputs(1, holes=0.0)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    templ = synth.templates(2048, 1)
    ks, ds = (512, 1024, 2048), (2, 3, 5)
    params = pf.track_params(torch.from_numpy(templ).cuda(), n_iters=6, k_sched=ks, decim_sched=ds,
                             update_mode=1, compose_mode=1)
    status, pose, st = vol.track_frame(to_dev(fr.depth), synth.ROOM64_INTR, params, fr.init_pose)
    ores = oracle.track(ovol, fr.depth, abi(synth.ROOM64_INTR), templ, fr.init_pose,
                        oracle.TrackParams(n_iters=6, k_sched=ks, decim_sched=ds, update_mode=1, compose_mode=1))
    assert list(st["k_used"]) == list(ores.stats["k_used"])
    assert list(st["n_eval"]) == list(ores.stats["n_eval"])
    assert st["best"][0] == ores.stats["best"][0]
    assert st["n_valid0"][0] == ores.stats["n_valid0"][0]
    assert abs(st["E0"][0] - ores.stats["E0"][0]) <= 1e-5 * ores.stats["E0"][0]
    assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4


def test_track_paper_schedule_with_10240_particles(pf):
    """The paper's schedule at full scale in particles: 1024 / 3072 / 10240
    particles with strides 8 / 16 / 32 (Sec. IV-A), mean update."""
    torch = torch_cuda()
    scene, fr, tsdf, weight = _room_inputs(2, holes=0.0)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    templ = synth.templates(10240, 2)
    ks, ds = (1024, 3072, 10240), (8, 16, 32)
    params = pf.track_params(torch.from_numpy(templ).cuda(), n_iters=6, k_sched=ks, decim_sched=ds,
                             update_mode=0, compose_mode=1)
    status, pose, st = vol.track_frame(to_dev(fr.depth), synth.ROOM64_INTR, params, fr.init_pose)
    ores = oracle.track(ovol, fr.depth, abi(synth.ROOM64_INTR), templ, fr.init_pose,
                        oracle.TrackParams(n_iters=6, k_sched=ks, decim_sched=ds, update_mode=0, compose_mode=1))
    assert status == pf.PF_OK and not ores.lost
    os_ = ores.stats
    assert list(st["k_used"]) == list(os_["k_used"]) == [1024, 3072, 10240, 1024, 3072, 10240]
    assert list(st["n_eval"]) == list(os_["n_eval"])
    for i in range(6):
        if not (os_["best_gap"][i] > 3e-5 and os_["adv_margin"][i] > 3e-5):
            break
        assert st["best"][i] == os_["best"][i] and st["n_adv"][i] == os_["n_adv"][i], i
        # the kept points are evaluated in a locality order (the same set):
        # the fitness of the entering pose still matches
        assert abs(st["E0"][i] - os_["E0"][i]) <= 1e-5 * os_["E0"][i], i
        assert st["n_valid0"][i] == os_["n_valid0"][i], i
    assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4


def test_track_exact_ties_on_a_constant_field(pf):
    """A constant field c (exact in binary): every particle ties exactly, so
    the best index is 0 (lowest on ties), the advantage set is empty, the
    pose stays, and s follows s0 (beta + (1 - beta) c)^i in both modes."""
    torch = torch_cuda()
    g = Grid(30, 30, 30, 0.1, 0.3, (-1.5, -1.5, 0.0))
    c = 0.375
    vol = pf.Volume.from_grid(g)
    vol.upload(np.full(g.n_nodes, c, dtype=np.float32), np.ones(g.n_nodes, dtype=np.float32))
    intr = Intrinsics(6, 5, 5.0, 5.0, 2.5, 2.0)
    depth = np.full((5, 6), 1.5, dtype=np.float32)
    templ = torch.from_numpy(synth.templates(64, 1)).cuda()
    for mode in (0, 1):
        params = pf.track_params(templ, n_iters=8, k_sched=(64, 64, 64), decim_sched=(1, 1, 1), update_mode=mode)
        status, pose, st = vol.track_frame(to_dev(depth), intr, params, np.eye(4))
        assert status == pf.PF_OK
        assert np.all(st["n_adv"] == 0) and np.all(st["best"] == 0)
        assert np.array_equal(pose, np.eye(4))
        assert np.all(st["E0"] == np.float32(c))
        np.testing.assert_allclose(st["s"][:, 0], 10.0 * (0.1 + 0.9 * c) ** np.arange(8), rtol=1e-12)


# ---------------------------------------------------------------------------
# raycast
# ---------------------------------------------------------------------------

def test_raycast_parity(pf):
    grid = Grid(72, 72, 72, 0.05, 0.15, (-0.2, -0.2, -0.2))
    intr = Intrinsics(160, 120, 140.0, 140.0, 79.5, 59.5)
    vol, ovol, amb = _fuse_both(pf, grid, intr, list(range(8)), seed=2)
    P = synth.room_view(synth.room_scene(2), 0)
    d, n = vol.raycast(intr, P)
    d = d.cpu().numpy()
    od, on = oracle.raycast(ovol, abi(intr), P)
    both = (d > 0) & (od > 0)
    assert np.mean((d > 0) == (od > 0)) > 0.995
    assert np.mean(np.abs(d[both] - od[both]) < 1e-4) > 0.995
    n = n.cpu().numpy()
    good = both & np.isfinite(n[..., 0]) & np.isfinite(on[..., 0])
    assert np.mean(np.sum(n[good] * on[good], axis=-1) > 0.999) > 0.99
