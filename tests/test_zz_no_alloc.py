"""pf_fitness_noalloc: the fitness entry point for callers that must not
allocate device memory once running.  Its results must agree with
pf_fitness (same kernel, scratch in a fixed array inside the library) on
consecutive calls, which share that array; and it must not allocate.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

from gpu_helpers import load_pf, perturbed_poses, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_fitness_matches_pf_fitness_on_consecutive_calls():
    torch = torch_cuda()
    pf = load_pf()
    lib = pf.load()
    scene, fr = synth.room64_frame(0)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=0.03)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    pts = to_dev(synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose))
    n = pts.shape[0]
    pose_sets = [to_dev(perturbed_poses(fr.gt_pose, 1024, 8.0, 8.0, seed=11)),
                 to_dev(perturbed_poses(fr.gt_pose, 777, 0.5, 0.5, seed=12))]
    outs = [(torch.empty(p.shape[0], dtype=torch.float32, device="cuda"),
             torch.empty(p.shape[0], dtype=torch.int32, device="cuda")) for p in pose_sets]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(poses, E, Cn):
        return lib.pf_fitness_noalloc(vol.handle, C.c_void_p(pts.data_ptr()), n, C.c_void_p(poses.data_ptr()),
                                      poses.shape[0], C.c_void_p(E.data_ptr()), C.c_void_p(Cn.data_ptr()), stream)

    # first call on this device: looks up the scratch array (set-up)
    assert call(pose_sets[0], *outs[0]) == pf.PF_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for poses, (E, Cn) in zip(pose_sets, outs):
        assert call(poses, E, Cn) == pf.PF_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before, "pf_fitness_noalloc allocated device memory"

    for poses, (E, Cn) in zip(pose_sets, outs):
        E_ref, C_ref = vol.fitness(pts, poses)
        E, Cn, E_ref, C_ref = (t.cpu().numpy() for t in (E, Cn, E_ref, C_ref))
        assert np.array_equal(Cn, C_ref)
        fin = C_ref > 0
        assert np.all(np.isinf(E[~fin]))
        assert np.all(np.abs(E[fin] - E_ref[fin]) <= 1e-5 * E_ref[fin] + 1e-7)


def test_noalloc_fitness_rejects_oversized_calls():
    torch = torch_cuda()
    pf = load_pf()
    lib = pf.load()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(16, dtype=torch.int32, device="cuda")
    k = pf.PF_NOALLOC_MAX_SLOTS + 1
    st = lib.pf_fitness_noalloc(vol.handle, C.c_void_p(buf.data_ptr()), 4, C.c_void_p(buf.data_ptr()), k,
                                C.c_void_p(buf.data_ptr()), C.c_void_p(cnt.data_ptr()), None)
    assert st == pf.PF_ERR_INVALID_ARG
