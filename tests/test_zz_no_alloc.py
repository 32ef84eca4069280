"""pf_fitness_noalloc: the fitness entry point for callers that must not
allocate device memory once running (a process whose device memory belongs
to another allocator, a real-time loop that cannot take the device-wide
synchronisation of cudaMalloc).  Its results must agree with pf_fitness
(same kernels, scratch in a fixed array inside the library) on consecutive
calls, which share that array, for every storage type and lane mapping; and
after its first call on a device (the set-up) it must not allocate: neither
through the library (pf_alloc_count) nor at all (free device memory).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

from gpu_helpers import load_pf, perturbed_poses, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# (storage, variant): variant = layout + 4 * mapping; mapping 0 automatic,
# 1 points on lanes, 2 particles on lanes
CASES = [("f32", 0), ("f32", 4), ("f32", 8), ("f16", 0), ("f16", 8), ("fp8", 0), ("fp8", 4)]


def _volumes(pf, scene):
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=0.03)
    dtypes = {"f32": pf.PF_F32, "f16": pf.PF_F16, "fp8": pf.PF_FP8E4M3}
    vols = {}
    for name, dt in dtypes.items():
        v = pf.Volume.from_grid(synth.ROOM64_GRID, tsdf_dtype=dt, weight_u8=int(dt != pf.PF_F32))
        v.upload(tsdf, weight)
        vols[name] = v
    return vols


def test_noalloc_fitness_matches_pf_fitness_and_allocates_nothing():
    torch = torch_cuda()
    pf = load_pf()
    lib = pf.load()
    scene, fr = synth.room64_frame(0)
    vols = _volumes(pf, scene)
    pts = to_dev(synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose))
    n = pts.shape[0]
    # 1024 poses spread over 8 deg / 8 cm, 777 within 0.5 deg / 0.5 cm, and
    # 16384 poses: PF_NOALLOC_MAX_SLOTS / 16384 = 4 point tiles, fewer than
    # pf_fitness takes for them (a different float summation order)
    pose_sets = [to_dev(perturbed_poses(fr.gt_pose, 1024, 8.0, 8.0, seed=11)),
                 to_dev(perturbed_poses(fr.gt_pose, 777, 0.5, 0.5, seed=12)),
                 to_dev(perturbed_poses(fr.gt_pose, 16384, 3.0, 3.0, seed=13))]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(vol, poses, E, Cn):
        return lib.pf_fitness_noalloc(vol.handle, C.c_void_p(pts.data_ptr()), n, C.c_void_p(poses.data_ptr()),
                                      poses.shape[0], C.c_void_p(E.data_ptr()), C.c_void_p(Cn.data_ptr()), stream)

    # expected values from pf_fitness (itself checked against the oracle),
    # and every output buffer, before anything is counted
    refs, outs = {}, {}
    for storage, variant in CASES:
        vol = vols[storage]
        vol.set_fitness_variant(variant)
        for i, poses in enumerate(pose_sets):
            refs[storage, variant, i] = tuple(t.cpu().numpy() for t in vol.fitness(pts, poses))
            outs[storage, variant, i] = [(torch.empty(poses.shape[0], dtype=torch.float32, device="cuda"),
                                          torch.empty(poses.shape[0], dtype=torch.int32, device="cuda"))
                                         for _ in range(2)]
    # first call on this device: the set-up (looks up the scratch array and
    # loads every fitness kernel the call can launch)
    vols["f32"].set_fitness_variant(0)
    E0, C0 = outs["f32", 0, 0][0]
    assert call(vols["f32"], pose_sets[0], E0, C0) == pf.PF_OK
    torch.cuda.synchronize()

    allocs_before = pf.pf_alloc_count()
    free_before = torch.cuda.mem_get_info()[0]
    for storage, variant in CASES:
        vol = vols[storage]
        vol.set_fitness_variant(variant)
        for i, poses in enumerate(pose_sets):
            for E, Cn in outs[storage, variant, i]:          # two calls in a row on the shared array
                assert call(vol, poses, E, Cn) == pf.PF_OK
    torch.cuda.synchronize()
    assert pf.pf_alloc_count() == allocs_before, "pf_fitness_noalloc allocated through the library"
    assert torch.cuda.mem_get_info()[0] == free_before, "pf_fitness_noalloc allocated device memory"

    for (storage, variant, i), (E_ref, C_ref) in refs.items():
        fin = C_ref > 0
        for E, Cn in outs[storage, variant, i]:
            E, Cn = E.cpu().numpy(), Cn.cpu().numpy()
            assert np.array_equal(Cn, C_ref), (storage, variant, i)
            assert np.all(np.isinf(E[~fin]))
            # same samples, possibly another order of the float sums of
            # non-negative terms: within 1e-5 relative
            assert np.all(np.abs(E[fin] - E_ref[fin]) <= 1e-5 * E_ref[fin]), (storage, variant, i)
    for v in vols.values():
        v.close()


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
    vol.close()
