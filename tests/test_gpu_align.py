"""Alignment loss, its derivatives (pose and node values), the autograd
wrapper and the Gauss-Newton polish: CUDA path against the FP64 oracle.

Tolerances (from the arithmetic): per-sample work is float with the point's
grid coordinate formed from error-free products, so a residual carries a
few float roundings (~2e-7) and the per-thread float sums ~1e-6 relative;
sums across threads are FP64.  Loss within 1e-5 relative, pose gradient
within 1e-5 of its norm, node-value gradient within 1e-5 relative plus 1e-6
absolute (the fixed-point unit is 2^-40).  Valid counts are exact.  The
polish matches the oracle's first objective to 1e-5 and its final pose to
1e-4 m / 1e-4 rad (the search's pose tolerance); near convergence the
accept / reject decisions compare objectives that differ by rounding only,
so the step sequences may differ after that point.
"""
import numpy as np
import pytest

import oracle
import synth

from gpu_helpers import abi, load_pf, pose_rot_err, pose_trans_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    torch_cuda()
    return load_pf()


def _frames(n_frames=3, holes=0.03, seed=0):
    """Room-64 volume plus n_frames point sets (ragged) and perturbed poses."""
    scene = synth.room_scene(seed)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=holes, seed=seed)
    pts, poses = [], []
    for f in range(n_frames):
        gt = synth.room_view(scene, f)
        p = synth.render_points(scene, synth.ROOM64_INTR, gt)
        pts.append(p[: len(p) - 997 * f])  # ragged counts
        D = synth.perturbation(40 + f, 0, 2.0 + f, 2.0 + f)
        poses.append(gt @ D)
    n_max = max(len(p) for p in pts)
    P = np.full((n_frames, n_max, 4), np.nan, dtype=np.float32)
    for f, p in enumerate(pts):
        P[f, : len(p)] = p
    counts = np.array([len(p) for p in pts], dtype=np.int32)
    return tsdf, weight, P, counts, np.stack(poses)


def _check_against_oracle(ovol, P, counts, poses, xi, res, gV_gpu=None, dloss=None):
    loss, cnt, gx = res
    F = len(counts)
    gV = np.zeros(ovol.grid.n_nodes)
    for f in range(F):
        o = oracle.align_loss(ovol, P[f, : counts[f]], poses[f], xi=None if xi is None else xi[f],
                              grad_tsdf=gV_gpu is not None)
        w = 1.0 if dloss is None else dloss[f]
        assert cnt[f] == o.count, (f, cnt[f], o.count)
        assert abs(loss[f] - o.loss) <= 1e-5 * o.loss + 1e-9
        if gx is not None:
            assert np.all(np.abs(gx[f] - w * o.grad_xi) <= 1e-5 * np.linalg.norm(w * o.grad_xi) + 1e-9), \
                (f, gx[f], w * o.grad_xi)
        if gV_gpu is not None:
            gV += w * o.grad_tsdf
    if gV_gpu is not None:
        err = np.abs(gV_gpu.astype(np.float64) - gV)
        assert np.all(err <= 1e-5 * np.abs(gV) + 1e-6), float(np.max(err - 1e-5 * np.abs(gV)))
        assert np.count_nonzero(gV) > 1000


def test_align_loss_and_gradients_match_the_oracle(pf):
    torch = torch_cuda()
    tsdf, weight, P, counts, poses = _frames()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), tsdf, weight)
    xi = np.array([[0.0] * 6, [0.01, -0.02, 0.005, 0.02, -0.01, 0.015], [-0.03, 0.01, 0.02, -0.01, 0.0, 0.02]])
    dloss = np.array([1.0, 0.5, -2.0])
    loss, cnt, gx, gV = vol.align_loss(to_dev(P), to_dev(poses), counts=to_dev(counts), xi=to_dev(xi),
                                       dloss=to_dev(dloss), grad_xi=True, grad_tsdf=True)
    torch.cuda.synchronize()
    _check_against_oracle(ovol, P, counts, poses, xi, (loss.cpu().numpy(), cnt.cpu().numpy(), gx.cpu().numpy()),
                          gV.cpu().numpy(), dloss)
    # without optional outputs and inputs: same loss (xi = 0 for frame 0 only)
    l2, c2, _, _ = vol.align_loss(to_dev(P[:1]), to_dev(poses[:1]), counts=to_dev(counts[:1]))
    assert float(l2[0]) == float(loss[0]) and int(c2[0]) == int(cnt[0])


def test_node_gradient_is_reproducible(pf):
    tsdf, weight, P, counts, poses = _frames(2)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    outs = [vol.align_loss(to_dev(P), to_dev(poses), counts=to_dev(counts), grad_xi=True, grad_tsdf=True)
            for _ in range(2)]
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


@pytest.mark.parametrize("name,view", [("f16", 0), ("bf16", 0), ("fp8", 0), ("bf16", 2), ("fp8", 2)])
def test_align_loss_on_narrow_storage(pf, name, view):
    """16-bit and scaled e4m3 grids, full or narrow cell view: loss and
    gradients against the oracle on the stored (downloaded) grid; the node
    gradient is with respect to the decoded float values."""
    tsdf, weight, P, counts, poses = _frames(2)
    code = {"f16": pf.PF_F16, "bf16": pf.PF_BF16, "fp8": pf.PF_FP8E4M3}[name]
    vol = pf.Volume.from_grid(synth.ROOM64_GRID, tsdf_dtype=code, cell_view=view)
    vol.upload(tsdf, weight)
    ts, ws = vol.download()
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), ts, ws)
    loss, cnt, gx, gV = vol.align_loss(to_dev(P), to_dev(poses), counts=to_dev(counts), grad_xi=True,
                                       grad_tsdf=True)
    _check_against_oracle(ovol, P, counts, poses, None, (loss.cpu().numpy(), cnt.cpu().numpy(), gx.cpu().numpy()),
                          gV.cpu().numpy())


def test_align_loss_edge_cases(pf):
    torch = torch_cuda()
    tsdf, weight, P, counts, poses = _frames(2)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    # an empty frame and a frame of non-finite points
    P2 = P.copy()
    P2[1] = np.nan
    counts2 = np.array([0, counts[1]], dtype=np.int32)
    loss, cnt, gx, gV = vol.align_loss(to_dev(P2), to_dev(poses), counts=to_dev(counts2), grad_xi=True,
                                       grad_tsdf=True)
    assert loss.cpu().numpy().tolist() == [0.0, 0.0] and cnt.cpu().numpy().tolist() == [0, 0]
    assert np.all(gx.cpu().numpy() == 0) and np.all(gV.cpu().numpy() == 0)
    # a pose far outside the grid sees nothing
    far = poses.copy()
    far[:, :3, 3] += 1e7
    loss, cnt, _, _ = vol.align_loss(to_dev(P), to_dev(far), counts=to_dev(counts))
    assert cnt.cpu().numpy().tolist() == [0, 0]
    torch.cuda.synchronize()


def test_autograd_function(pf):
    torch = torch_cuda()
    tsdf, weight, P, counts, poses = _frames(2)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    vol.upload(tsdf, weight)
    Pd, posed, cd = to_dev(P), to_dev(poses), to_dev(counts)
    xi = torch.tensor([[0.01, 0.0, -0.01, 0.0, 0.01, 0.0], [0.0] * 6], dtype=torch.float64, device="cuda",
                      requires_grad=True)
    sink = torch.zeros(vol.n_nodes, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = pf.align_loss(vol, Pd, posed, xi, counts=cd, tsdf_sink=sink)
    w = torch.tensor([0.3, -1.7], dtype=torch.float64, device="cuda")
    (loss * w).sum().backward()
    _, _, gx, gV = vol.align_loss(Pd, posed, counts=cd, xi=xi.detach(), dloss=w, grad_xi=True, grad_tsdf=True)
    assert torch.equal(xi.grad, gx)
    assert torch.equal(sink.grad, gV)


@pytest.mark.parametrize("name", ["f32", "bf16", "fp8"])
def test_polish_matches_the_oracle(pf, name):
    """Gauss-Newton polish on float, bfloat16 and scaled e4m3 grids against
    the oracle's polish of the same stored values."""
    torch = torch_cuda()
    scene, fr = synth.room64_frame(0, noise=False)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=0.0)
    code = {"f32": pf.PF_F32, "bf16": pf.PF_BF16, "fp8": pf.PF_FP8E4M3}[name]
    vol = pf.Volume.from_grid(synth.ROOM64_GRID, tsdf_dtype=code)
    vol.upload(tsdf, weight)
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), *vol.download())
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    pose = torch.from_numpy(fr.init_pose.reshape(16).copy()).cuda()
    trace, acc = vol.polish(to_dev(pts), pose, steps=10)
    P = pose.cpu().numpy().reshape(4, 4)
    tr = trace.cpu().numpy()
    Po, acc_o, tr_o = oracle.polish(ovol, pts, fr.init_pose, steps=10)
    assert abs(tr[0] - tr_o[0]) <= 1e-5 * tr_o[0]
    assert np.all(np.diff(tr) <= 0)
    assert int(acc.item()) >= 3
    assert pose_trans_err(P, Po) <= 1e-4 and pose_rot_err(P, Po) <= 1e-4
    assert tr[-1] <= 1.01 * tr_o[-1] + 1e-9
    # closer to the truth than the start (on the float grid by a factor 10)
    e0, e1 = pose_trans_err(fr.init_pose, fr.gt_pose), pose_trans_err(P, fr.gt_pose)
    print(f"\npolish {name}: |t - t_gt| {100 * e0:.3f} cm -> {100 * e1:.3f} cm")
    assert e1 < (0.1 if name == "f32" else 1.0) * e0
    # zero steps: the pose is untouched and the trace holds its objective
    pose0 = torch.from_numpy(fr.init_pose.reshape(16).copy()).cuda()
    t0, a0 = vol.polish(to_dev(pts), pose0, steps=0)
    assert np.array_equal(pose0.cpu().numpy(), fr.init_pose.reshape(16)) and int(a0.item()) == 0
    assert abs(float(t0[0]) - tr_o[0]) <= 1e-5 * tr_o[0]
