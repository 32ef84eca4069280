"""A narrow search view of a float grid (pf_volume_desc.search_dtype): fusion
averages in the float master grid, and each refresh of the cell view rounds
the current node values once into half, bfloat16 or scaled e4m3 records.
The search and pf_fitness (default layout) read that rounded grid; the node
layout still reads the float master.

So the fitness and the search must match the FP64 oracle run on the master
grid rounded to the view's format (the host model of the rounding is written
from the formats' definitions in test_gpu_precision), with the float
tolerances of the parity tests, and the node layout must match the oracle on
the unrounded master -- after an upload and after fusion alike."""
import numpy as np
import pytest

import oracle
import synth

from gpu_helpers import (abi, compare_fitness, load_pf, perturbed_poses, pose_rot_err, pose_trans_err, to_dev,
                         torch_cuda)
from test_gpu_precision import _room_inputs, dtype_code, expected_download

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    torch_cuda()
    return load_pf()


def _search_view_volume(pf, name, view=0):
    vol = pf.Volume.from_grid(synth.ROOM64_GRID, cell_view=view, search_dtype=dtype_code(pf, name))
    assert vol.info()["cell_view"] == (1 if view == 0 else view)
    return vol


def _check_fitness(pf, vol, name, pts, poses, cap=64):
    ts, ws = vol.download()                      # the float master
    rounded = oracle.Volume(abi(synth.ROOM64_GRID), expected_download(ts, ws, name), ws)
    master = oracle.Volume(abi(synth.ROOM64_GRID), ts, ws)
    orc_r = oracle.fitness(rounded, pts, poses, ambiguity=True, cap=cap)
    orc_m = oracle.fitness(master, pts, poses, ambiguity=True, cap=cap)
    assert np.all(orc_r.amb <= cap) and np.all(orc_m.amb <= cap)
    for mapping in range(3):
        for layout, orc in ((3, orc_r), (2, orc_m)):
            vol.set_fitness_variant(layout + 4 * mapping)
            E, C = vol.fitness(to_dev(pts), to_dev(poses))
            compare_fitness(E.cpu().numpy(), C.cpu().numpy(), orc)
    vol.set_fitness_variant(0)
    E, C = vol.fitness(to_dev(pts), to_dev(poses))          # the default reads the search view
    compare_fitness(E.cpu().numpy(), C.cpu().numpy(), orc_r)
    return orc_r, orc_m


@pytest.mark.parametrize("name", ["f16", "bf16", "fp8"])
@pytest.mark.parametrize("view", [0, 2])
def test_search_view_fitness_on_the_rounded_grid(pf, name, view):
    scene, fr, tsdf, weight = _room_inputs()
    vol = _search_view_volume(pf, name, view)
    vol.upload(tsdf, weight)
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    for K, spread in ((1024, 8.0), (1000, 0.05)):
        orc_r, orc_m = _check_fitness(pf, vol, name, pts, perturbed_poses(fr.gt_pose, K, spread, spread, seed=K))
        # the two grids do differ
        assert not np.array_equal(orc_r.E, orc_m.E)
    vol.close()


@pytest.mark.parametrize("name", ["f16", "bf16", "fp8"])
def test_search_view_follows_fusion(pf, name):
    """Fusion of several noisy views into the float master; every refresh
    rounds the fused values into the view."""
    torch = torch_cuda()
    scene = synth.room_scene(2)
    vol = _search_view_volume(pf, name)
    for view in range(4):
        P = synth.room_view(scene, view)
        d = synth.add_depth_noise(synth.render_depth(scene, synth.ROOM64_INTR, P), 50 + view, sigma_const=0.002)
        vol.integrate(to_dev(d), synth.ROOM64_INTR, P)
    torch.cuda.synchronize()
    fr_pose = synth.room_view(scene, 1)
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr_pose)
    # (at the fused view's own pose, pose 0, a few hundred surface points lie
    # on the faces of cells whose validity changes there: the axis-aligned
    # walls sit on grid planes; the oracle reports them all)
    _check_fitness(pf, vol, name, pts, perturbed_poses(fr_pose, 512, 2.0, 2.0, seed=7), cap=1024)
    vol.close()


@pytest.mark.parametrize("name", ["f16", "bf16"])
def test_search_view_track_parity(pf, name):
    torch = torch_cuda()
    K, iters = 1024, 10
    scene, fr, tsdf, weight = _room_inputs(0, holes=0.0)
    vol = _search_view_volume(pf, name)
    vol.upload(tsdf, weight)
    ts, ws = vol.download()
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), expected_download(ts, ws, name), ws)
    templ = synth.templates(K, 0)
    params = pf.track_params(torch.from_numpy(templ).cuda(), n_iters=iters, k_sched=(K, K, K),
                             decim_sched=(1, 1, 1), update_mode=0, compose_mode=1)
    status, pose, st = vol.track_frame(to_dev(fr.depth), synth.ROOM64_INTR, params, fr.init_pose)
    oparams = oracle.TrackParams(n_iters=iters, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                                 compose_mode=1)
    ores = oracle.track(ovol, fr.depth, abi(synth.ROOM64_INTR), templ, fr.init_pose, oparams)
    assert status == pf.PF_OK and not ores.lost
    os_ = ores.stats
    strict = 0
    for i in range(iters):
        if not (os_["best_gap"][i] > 3e-5 and os_["adv_margin"][i] > 3e-5):
            break
        strict += 1
        assert st["best"][i] == os_["best"][i] and st["n_adv"][i] == os_["n_adv"][i], i
        np.testing.assert_allclose(st["pose"][i], os_["pose"][i], atol=1e-5)
    assert strict >= 2
    assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4
    vol.close()
