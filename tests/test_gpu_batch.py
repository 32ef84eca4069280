"""Batches of sequences (pf_batch_*): several volumes of different sizes and
cameras stepped together, the search iterations of all sequences sharing
launches, the step captured in a CUDA graph.

Each sequence's search is checked against the FP64 oracle exactly as a
single-sequence search is (same best particle and advantage-set size while
the oracle's margins are clear, final pose within 1e-4 m / 1e-4 rad);
graph replay must be bit-identical to direct launches; the autotuner must
pick one of its candidates and leave the batch usable.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import Grid, Intrinsics

from gpu_helpers import abi, load_pf, pose_rot_err, pose_trans_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

# (grid, camera, view): three sequences of unequal size over the room scene
SEQS = [
    (synth.ROOM64_GRID, synth.ROOM64_INTR, 0),
    (Grid(48, 40, 44, 0.07, 0.21, (0.0, 0.0, 0.0)), Intrinsics(200, 150, 175.0, 176.0, 99.3, 74.8, 0.1, 8.0), 1),
    (Grid(80, 80, 80, 0.04, 0.12, (0.0, 0.0, 0.0)), Intrinsics(320, 240, 280.0, 280.0, 159.5, 119.5, 0.1, 8.0), 2),
]
K, ITERS = 1024, 10


@pytest.fixture(scope="module")
def pf():
    torch_cuda()
    return load_pf()


def _setup(pf, seed=0, dtype=None, views=(0, 0, 0)):
    """Volumes fused from three noise-free views each, the frame to track
    (noisy) and its initial pose per sequence."""
    torch = torch_cuda()
    scene = synth.room_scene(seed)
    vols, frames = [], []
    for (g, intr, view), cv in zip(SEQS, views):
        v = pf.Volume.from_grid(g, tsdf_dtype=pf.PF_F32 if dtype is None else dtype, cell_view=cv,
                                weight_u8=int(dtype is not None))
        for j in range(3):
            P = synth.room_view(scene, (view + 1 + j) % 8)
            v.integrate(to_dev(synth.render_depth(scene, intr, P)), intr, P)
        gt = synth.room_view(scene, view)
        depth = synth.add_depth_noise(synth.render_depth(scene, intr, gt), 60 + view, 0.001)
        init = gt @ synth.perturbation(70 + view, 0, 3.0, 3.0)
        vols.append(v)
        frames.append((depth, gt, init))
    torch.cuda.synchronize()
    templ = torch.from_numpy(synth.templates(K, seed)).cuda()
    params = [pf.track_params(templ, n_iters=ITERS, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                              compose_mode=1) for _ in SEQS]
    return vols, frames, templ, params


def _load_inputs(batch, frames):
    for i, (depth, gt, init) in enumerate(frames):
        batch.depth[i].copy_(to_dev(depth))
        batch.pose[i].copy_(to_dev(init))
        batch.rel[i].copy_(to_dev(np.eye(4)))


STORAGE = {"f32": ("PF_F32", (0, 0, 0)), "bf16": ("PF_BF16", (0, 0, 0)), "fp8": ("PF_FP8E4M3", (0, 0, 0)),
           "f16-narrow": ("PF_F16", (2, 2, 2)), "fp8-mixed-views": ("PF_FP8E4M3", (1, 2, 1))}


@pytest.mark.parametrize("storage", sorted(STORAGE))
def test_batch_step_matches_the_oracle_per_sequence(pf, storage):
    """Per storage type (uint8 weights for the narrow ones) and cell view
    (full, narrow, or mixed within the batch): the oracle runs on each
    volume's downloaded grid, i.e. the stored values.  Decisions are compared
    while the oracle's margins stay clear (at least one iteration per
    sequence, four over the batch); the final pose always."""
    torch = torch_cuda()
    code, views = STORAGE[storage]
    dtype = None if storage == "f32" else getattr(pf, code)
    vols, frames, templ, params = _setup(pf, dtype=dtype, views=views)
    for v, cv in zip(vols, views):
        assert v.info()["cell_view"] == (cv or 1)
    grids = [v.download() for v in vols]  # the state each search runs against
    batch = pf.Batch(vols, [s[1] for s in SEQS], params, use_graph=True)
    _load_inputs(batch, frames)
    batch.step()
    torch.cuda.synchronize()
    oparams = oracle.TrackParams(n_iters=ITERS, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                                 compose_mode=1)
    total_strict = 0
    for i, ((g, intr, view), (depth, gt, init)) in enumerate(zip(SEQS, frames)):
        st = batch.stats_dict(i)
        pose = batch.pose[i].cpu().numpy()
        ovol = oracle.Volume(abi(g), *grids[i])
        ores = oracle.track(ovol, depth, abi(intr), templ.cpu().numpy(), init, oparams)
        assert st["status"] == pf.PF_OK and not ores.lost
        os_ = ores.stats
        assert st["n_points"] == os_["n_points"]
        strict = 0
        for it in range(ITERS):
            if not (os_["best_gap"][it] > 3e-5 and os_["adv_margin"][it] > 3e-5):
                break
            strict += 1
            assert st["best"][it] == os_["best"][it] and st["n_adv"][it] == os_["n_adv"][it], (i, it)
        assert strict >= 1, i
        total_strict += strict
        assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4, i
    assert total_strict >= 4
    batch.close()


def test_many_small_sequences_match_the_oracle(pf):
    """64 sequences of different grids (20^3 .. 27^3 nodes over the room),
    cameras (40x30 .. 71x53) and particle counts (64 .. 256): every CTA finds
    its problem among 64 in the batched launches; each sequence's search
    matches the oracle on its own fused grid."""
    torch = torch_cuda()
    scene = synth.room_scene(3)
    n = 64
    vols, gdefs, cams, frames, params, kk = [], [], [], [], [], []
    templ_np = synth.templates(256, 3)
    templ = torch.from_numpy(templ_np).cuda()
    for i in range(n):
        m = 20 + i % 8
        g = Grid(m, m, m, 3.6 / (m - 1), 3.0 * 3.6 / (m - 1), (-0.2, -0.2, -0.2))
        w, h = 40 + (i * 7) % 32, 30 + (i * 5) % 24
        cam = Intrinsics(w, h, 0.9 * w, 0.9 * w, (w - 1) / 2, (h - 1) / 2, 0.1, 8.0)
        v = pf.Volume.from_grid(g)
        for j in range(2):
            P = synth.room_view(scene, (i + 1 + j) % 8)
            v.integrate(to_dev(synth.render_depth(scene, cam, P)), cam, P)
        gt = synth.room_view(scene, i % 8)
        depth = synth.add_depth_noise(synth.render_depth(scene, cam, gt), 500 + i, 0.001)
        init = gt @ synth.perturbation(600 + i, 0, 3.0, 3.0)
        K_i = (64, 128, 192, 256)[i % 4]
        vols.append(v)
        gdefs.append(g)
        cams.append(cam)
        frames.append((depth, gt, init))
        kk.append(K_i)
        params.append(pf.track_params(templ, n_iters=4, k_sched=(K_i,) * 3, decim_sched=(1, 1, 1), update_mode=0,
                                      compose_mode=1))
    torch.cuda.synchronize()
    grids = [v.download() for v in vols]
    batch = pf.Batch(vols, cams, params, use_graph=False)
    _load_inputs(batch, frames)
    batch.step()
    torch.cuda.synchronize()
    total_strict = 0
    for i in range(n):
        depth, gt, init = frames[i]
        st = batch.stats_dict(i)
        pose = batch.pose[i].cpu().numpy()
        ovol = oracle.Volume(abi(gdefs[i]), *grids[i])
        ores = oracle.track(ovol, depth, abi(cams[i]), templ_np, init,
                            oracle.TrackParams(n_iters=4, k_sched=(kk[i],) * 3, decim_sched=(1, 1, 1), update_mode=0,
                                               compose_mode=1))
        assert st["status"] == (pf.PF_ERR_TRACK_LOST if ores.lost else pf.PF_OK), i
        if ores.lost:
            continue
        os_ = ores.stats
        assert st["n_points"] == os_["n_points"], i
        for it in range(4):
            if not (os_["best_gap"][it] > 3e-5 and os_["adv_margin"][it] > 3e-5):
                break
            total_strict += 1
            assert st["best"][it] == os_["best"][it] and st["n_adv"][it] == os_["n_adv"][it], (i, it)
        assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4, i
    assert total_strict >= n
    batch.close()


def test_graph_replay_equals_direct_launches(pf):
    torch = torch_cuda()
    results = []
    for use_graph in (False, True):
        vols, frames, templ, params = _setup(pf)
        batch = pf.Batch(vols, [s[1] for s in SEQS], params, use_graph=use_graph)
        _load_inputs(batch, frames)
        out = []
        for step in range(3):
            # the same frame again, from a pose nudged away from the last result
            for i in range(batch.n):
                batch.rel[i].copy_(to_dev(synth.perturbation(80 + step, i, 1.0, 1.0)))
            batch.step()
            torch.cuda.synchronize()
            out.append([(batch.pose[i].cpu().numpy().copy(), batch.stats[i].cpu().numpy().copy())
                        for i in range(batch.n)])
        tsdf = [v.download()[0] for v in vols]
        results.append((out, tsdf))
        batch.close()
    (o1, t1), (o2, t2) = results
    for s1, s2 in zip(o1, o2):
        for (p1, st1), (p2, st2) in zip(s1, s2):
            assert np.array_equal(p1, p2) and np.array_equal(st1, st2)
    for a, b in zip(t1, t2):
        assert np.array_equal(a, b, equal_nan=True)


def test_autotune_and_validation(pf):
    torch = torch_cuda()
    vols, frames, templ, params = _setup(pf)
    batch = pf.Batch(vols, [s[1] for s in SEQS], params, use_graph=True)
    _load_inputs(batch, frames)
    batch.step()  # captures
    p = batch.autotune()
    assert p in (1024, 2048, 4096, 8192, 16384, 32768, 65536, 131072)
    tuned = batch.tuning()
    assert tuned["points_per_block"] == p and tuned["mapping_threshold"] in (0.0, 2.0, 3.0, 8.0, 12.0, 20.0)
    batch.step()  # recaptures with the chosen tiling
    torch.cuda.synchronize()
    # a forced threshold changes only which lanes carry which samples: the
    # step still runs and reports the value back
    batch.set_mapping_threshold(1e6)
    assert batch.tuning()["mapping_threshold"] == 1e6
    batch.set_mapping_threshold(0.0)
    assert batch.tuning()["mapping_threshold"] == 0.0
    torch.cuda.synchronize()
    for i in range(batch.n):
        assert batch.stats_dict(i)["status"] == pf.PF_OK
    with pytest.raises(pf.ProfusionError):
        batch.set_points_per_block(100)
    with pytest.raises(pf.ProfusionError):
        batch.set_mapping_threshold(float("nan"))
    batch.close()
    # a volume may appear once; storage types may not mix
    with pytest.raises(pf.ProfusionError):
        pf.Batch([vols[0], vols[0]], [SEQS[0][1]] * 2, params[:2])
    v16 = pf.Volume.from_grid(SEQS[0][0], tsdf_dtype=pf.PF_F16)
    with pytest.raises(pf.ProfusionError):
        pf.Batch([vols[0], v16], [SEQS[0][1]] * 2, params[:2])


# Closed loop over the multiroom trajectory, with camera / volume / particle
# mixes from the small end of the batch workload: (camera, nodes per axis over
# the 5.12 m scene, seed, particles).
TRAJ = [((160, 120), 128, 0, 1024), ((320, 240), 128, 1, 2048), ((160, 120), 256, 2, 1024)]
TRAJ_FRAMES = 4
_TRAJ_ORACLE = {}


def _traj_sequence(res, n, seed):
    w, h = res
    f = 525.0 * w / 640.0
    intr = Intrinsics(w, h, f, f, (w - 1) / 2.0, (h - 1) / 2.0, 0.1, 8.0)
    vs = 5.12 / n
    return synth.multiroom_sequence(300, seed, grid=Grid(n, n, n, vs, 3.0 * vs, (0.0, 0.0, 0.0)), intr=intr)


def _traj_params(K):
    return dict(n_iters=20, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0, compose_mode=1,
                min_valid_frac=0.05)


def _oracle_trajectory(i):
    """The FP64 oracle's closed loop for sequence i: frame 0 fused at its true
    pose, then per frame P0 = P_prev @ perturbed relative pose, search, and
    fusion at the pose found."""
    if i not in _TRAJ_ORACLE:
        res, n, seed, K = TRAJ[i]
        seq = _traj_sequence(res, n, seed)
        ovol = oracle.Volume(abi(seq.grid))
        intr = abi(seq.intr)
        oracle.integrate(ovol, seq.depth(0), intr, seq.gt[0])
        poses = [seq.gt[0]]
        prm = oracle.TrackParams(**_traj_params(K))
        for f in range(1, TRAJ_FRAMES + 1):
            r = oracle.track(ovol, seq.depth(f), intr, synth.templates(2048, 0), poses[-1] @ seq.relative_init(f), prm)
            poses.append(r.pose)
            oracle.integrate(ovol, seq.depth(f), intr, r.pose)
        _TRAJ_ORACLE[i] = np.array(poses)
    return _TRAJ_ORACLE[i]


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_batched_trajectory_stays_with_the_oracle(pf, storage):
    """Three sequences stepped as one batch under a CUDA graph for four
    frames, each frame tracked from the previous frame's result and fused at
    the pose found, against the oracle's FP64 closed loop on its own FP64
    grid.  Float storage: every frame within 1e-4 m and 1e-4 rad of the
    oracle.  half or bfloat16 storage with uint8 weights: the first frame
    within 1 mm (from then on the two grids differ by the storage's
    rounding, which can tip later decisions of the search)."""
    torch = torch_cuda()
    seqs = [_traj_sequence(res, n, seed) for res, n, seed, _ in TRAJ]
    dtype, u8 = {"f32": (pf.PF_F32, 0), "f16": (pf.PF_F16, 1), "bf16": (pf.PF_BF16, 1)}[storage]
    vols = [pf.Volume.from_grid(s.grid, tsdf_dtype=dtype, weight_u8=u8) for s in seqs]
    templ = torch.from_numpy(synth.templates(2048, 0)).cuda()
    params = [pf.track_params(templ, **_traj_params(K)) for *_, K in TRAJ]
    batch = pf.Batch(vols, [s.intr for s in seqs], params, use_graph=True)
    for i, s in enumerate(seqs):
        batch.pose[i].copy_(to_dev(s.gt[0]))
        batch.depth[i].copy_(to_dev(s.depth(0)))
    batch.fuse()
    n_frames = TRAJ_FRAMES if storage == "f32" else 1
    gpu = np.zeros((len(seqs), n_frames + 1, 4, 4))
    for f in range(1, n_frames + 1):
        for i, s in enumerate(seqs):
            batch.depth[i].copy_(to_dev(s.depth(f)))
            batch.rel[i].copy_(to_dev(s.relative_init(f)))
        batch.step()
        torch.cuda.synchronize()
        for i in range(len(seqs)):
            gpu[i, f] = batch.pose[i].cpu().numpy()
    batch.close()
    for i in range(len(seqs)):
        ref = _oracle_trajectory(i)
        for f in range(1, n_frames + 1):
            if storage == "f32":
                assert pose_trans_err(gpu[i, f], ref[f]) <= 1e-4, (i, f)
                assert pose_rot_err(gpu[i, f], ref[f]) <= 1e-4, (i, f)
            else:
                assert pose_trans_err(gpu[i, f], ref[f]) <= 1e-3, (i, f)
