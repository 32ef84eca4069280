"""Parity at the benchmark's full size.

The multiroom workload the bench times -- 640x480 depth, a 512^3 TSDF at
1 cm (tau 3 cm, float tsdf and weights, automatic cell view), 3072 particles
x 20 iterations over all points, mean update about the camera centre --
through the same calls and launch configuration.  The FP64 oracle handles
these sizes in seconds on the host cores, so the checks are complete rather
than sampled:
  * fusion of frames 0-2 at their true poses: every node of the 512^3 grid;
  * the fitness of 3072 particles over all points of frame 3, once at the
    search's initial spread (lanes on points) and once converged to 0.03
    deg / 0.03 cm (lanes on particles);
  * one full search of frame 3 from the bench's initial pose;
  * the ray cast of the fused grid from frame 2's pose.
Fusion is compared with the oracle's own fusion; the fitness, the search
and the ray cast run the oracle on the grid the GPU fused (downloaded), so
that each check isolates its own step (nodes on a pixel-rounding boundary
may legitimately differ between the two fusions).  Tolerances are those of
the small parity tests.
"""
import numpy as np
import pytest

import oracle
import synth

from gpu_helpers import (abi, compare_fitness, load_pf, perturbed_poses, pose_rot_err, pose_trans_err, to_dev,
                         torch_cuda)

pytestmark = pytest.mark.gpu

K, ITERS, FUSED = 3072, 20, 3


@pytest.fixture(scope="module")
def pf():
    torch_cuda()
    return load_pf()


@pytest.fixture(scope="module")
def fused(pf):
    seq = synth.multiroom_sequence(300, 0)
    grid, intr = seq.grid, seq.intr
    vol = pf.Volume.from_grid(grid)
    ovol = oracle.Volume(abi(grid))
    amb = np.zeros(grid.n_nodes, dtype=bool)
    for f in range(FUSED):
        depth = seq.depth(f)
        vol.integrate(to_dev(depth), intr, seq.gt[f])
        amb |= oracle.integrate(ovol, depth, abi(intr), seq.gt[f], ambiguity=True, eps_px=3e-4).astype(bool)
    t, w = vol.download()
    return seq, vol, ovol, amb, (t, w)


@pytest.fixture(scope="module")
def gpu_grid(fused):
    """The oracle's view of the grid the GPU fused."""
    seq, vol, ovol, amb, (t, w) = fused
    return oracle.Volume(abi(seq.grid), t, w)


def _frame_points(seq, f):
    """Frame f's back-projected points (float32, as the library forms them)."""
    pts = oracle.backproject(seq.depth(f), abi(seq.intr)).astype(np.float32)
    return np.ascontiguousarray(np.c_[pts, np.zeros(len(pts), np.float32)])


def test_fullsize_fusion(fused):
    seq, vol, ovol, amb, (t, w) = fused
    assert vol.info()["cell_view"] == 1
    ok = ~amb
    updated = ovol.weight > 0
    assert np.count_nonzero(updated) > 1_000_000
    assert np.count_nonzero(amb) < 1e-2 * np.count_nonzero(updated)
    assert np.array_equal(w[ok], ovol.weight[ok].astype(np.float32))
    obs = ok & updated
    assert np.max(np.abs(t[obs].astype(np.float64) - ovol.tsdf[obs])) <= 1e-5
    assert np.all(t[ok & ~updated] == 1.0)


@pytest.mark.parametrize("phase", ["initial", "converged"])
def test_fullsize_fitness(pf, fused, gpu_grid, phase):
    seq, vol = fused[0], fused[1]
    f = FUSED
    pts = _frame_points(seq, f)
    assert len(pts) > 200_000
    if phase == "initial":
        # the first iteration's particles: templates x (10 deg, 10 cm) about the camera centre
        P0 = seq.gt[f - 1] @ seq.relative_init(f)
        poses = oracle.particles(synth.templates(K, 0), K, P0, 10.0, 10.0, compose_mode=1).astype(np.float32)
    else:
        poses = perturbed_poses(seq.gt[f], K, 0.03, 0.03, seed=11)
    vol.set_fitness_variant(0)
    E, C = vol.fitness(to_dev(pts), to_dev(poses))
    orc = oracle.fitness(gpu_grid, pts[:, :3], poses.astype(np.float64), ambiguity=True, cap=128)
    assert np.all(orc.amb <= 128)
    assert np.count_nonzero(orc.C > 0) > K // 2
    compare_fitness(E.cpu().numpy(), C.cpu().numpy(), orc)


def test_fullsize_track(pf, fused, gpu_grid):
    torch = torch_cuda()
    seq, vol = fused[0], fused[1]
    f = FUSED
    P0 = seq.gt[f - 1] @ seq.relative_init(f)
    templ = synth.templates(K, 0)
    params = pf.track_params(torch.from_numpy(templ).cuda(), n_iters=ITERS, k_sched=(K, K, K), decim_sched=(1, 1, 1),
                             update_mode=0, compose_mode=1, min_valid_frac=0.05)
    vol.set_fitness_variant(0)
    status, pose, st = vol.track_frame(to_dev(seq.depth(f)), seq.intr, params, P0)
    oparams = oracle.TrackParams(n_iters=ITERS, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                                 compose_mode=1, min_valid_frac=0.05)
    ores = oracle.track(gpu_grid, seq.depth(f), abi(seq.intr), templ, P0, oparams)
    assert status == pf.PF_OK and not ores.lost
    os_ = ores.stats
    assert st["n_points"] == os_["n_points"] > 200_000
    strict = 0
    for i in range(ITERS):
        if not (os_["best_gap"][i] > 3e-5 and os_["adv_margin"][i] > 3e-5):
            break
        strict += 1
        assert st["best"][i] == os_["best"][i] and st["n_adv"][i] == os_["n_adv"][i], i
        assert abs(st["E0"][i] - os_["E0"][i]) <= 1e-5 * os_["E0"][i]
        np.testing.assert_allclose(st["s"][i], os_["s"][i], rtol=1e-5)
        np.testing.assert_allclose(st["pose"][i], os_["pose"][i], atol=1e-5)
    assert strict >= 1
    print(f"\nfullsize track: {strict} of {ITERS} iterations with clear margins; "
          f"|t - t_oracle| = {pose_trans_err(pose, ores.pose):.2e} m, rot {pose_rot_err(pose, ores.pose):.2e} rad")
    assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4


def test_fullsize_raycast(pf, fused, gpu_grid):
    seq, vol = fused[0], fused[1]
    P = seq.gt[FUSED - 1]
    d, n = vol.raycast(seq.intr, P)
    d, n = d.cpu().numpy(), n.cpu().numpy()
    od, on = oracle.raycast(gpu_grid, abi(seq.intr), P)
    both = (d > 0) & (od > 0)
    assert np.count_nonzero(both) > 0.5 * d.size
    assert np.mean((d > 0) == (od > 0)) > 0.995
    assert np.mean(np.abs(d[both] - od[both]) < 1e-4) > 0.995
    good = both & np.isfinite(n[..., 0]) & np.isfinite(on[..., 0])
    assert np.mean(np.sum(n[good] * on[good], axis=-1) > 0.999) > 0.99
