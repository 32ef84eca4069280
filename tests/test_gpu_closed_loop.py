"""The benchmark's closed loop against the FP64 oracle at full size.

The bench's device-resident frame loop -- P_t^(0) = P_(t-1) P_(t,t-1)
(pf_pose_compose, Sec. III-A), the randomized search from it
(pf_track_frame_async: 3072 particles x 20 iterations over all points,
advantage-set mean update, Sec. III-B) and fusion at the result
(pf_integrate_async, Sec. III) -- runs on the 640x480 / 512^3 multiroom
workload for frames 1-5, and the oracle runs the same loop on the host in
FP64 (its own fusion, its own poses).  Each frame's pose must stay within
1 mm and 1e-3 rad of the oracle's, so the trajectory error the bench reports
(ate_cm) is the method's, not the kernels': the two ATEs against ground
truth agree to 1 mm.  The same holds for the reduced-precision form (a
half-precision search view of the float grid) against the oracle running
that form.
"""
import numpy as np
import pytest

import oracle
import synth

from gpu_helpers import abi, load_pf, pose_rot_err, pose_trans_err, torch_cuda

pytestmark = pytest.mark.gpu

N_TRACKED = 5
K = 3072


def _gpu_loop(pf, torch, seq, depths, rels, templ, search_dtype):
    """The bench's device-resident loop on the GPU; poses of frames 0..N."""
    intr, grid = seq.intr, seq.grid
    dev = torch.device("cuda", 0)
    vol = pf.Volume.from_grid(grid, search_dtype=search_dtype)
    params = pf.track_params(torch.from_numpy(templ).to(dev), n_iters=20, k_sched=(K,) * 3, decim_sched=(1,) * 3,
                             update_mode=0, compose_mode=1, min_valid_frac=0.05)
    vol.reserve(intr.width * intr.height, K)
    depth_dev = [torch.from_numpy(d).to(dev) for d in depths]
    rel_dev = torch.from_numpy(np.stack([r.reshape(16) for r in rels])).to(dev)
    pose_dev = torch.zeros((N_TRACKED + 1, 16), dtype=torch.float64, device=dev)
    init_dev = torch.zeros((N_TRACKED + 1, 16), dtype=torch.float64, device=dev)
    pose_dev[0] = torch.from_numpy(seq.gt[0].reshape(16)).to(dev)
    vol.integrate_async(depth_dev[0], intr, pose_dev[0])
    for f in range(1, N_TRACKED + 1):
        pf.pf_pose_compose(pose_dev[f - 1], rel_dev[f], init_dev[f])
        vol.track_frame_async(depth_dev[f], intr, params, init_dev[f], pose_dev[f])
        vol.integrate_async(depth_dev[f], intr, pose_dev[f])
    torch.cuda.synchronize()
    out = pose_dev.cpu().numpy().reshape(-1, 4, 4)
    vol.close()
    return out


def _oracle_loop(seq, depths, rels, templ, round_name=None):
    """The same loop in FP64 on the host; with round_name, every search runs
    on a copy of the fused grid rounded to that storage format (the grid's
    float value rounded once, as the GPU's search view rounds its float
    master), while fusion stays FP64."""
    intr, grid = seq.intr, seq.grid
    ovol = oracle.Volume(abi(grid))
    oparams = oracle.TrackParams(n_iters=20, k_sched=(K,) * 3, decim_sched=(1,) * 3, s0_deg=10.0, s0_cm=10.0,
                                 beta=0.1, update_mode=0, compose_mode=1, min_valid_frac=0.05)
    oracle.integrate(ovol, depths[0], abi(intr), seq.gt[0])
    P = seq.gt[0]
    out = [P]
    for f in range(1, N_TRACKED + 1):
        search = ovol
        if round_name is not None:
            from test_gpu_precision import expected_download
            search = oracle.Volume(abi(grid), expected_download(ovol.tsdf.astype(np.float32), ovol.weight,
                                                                round_name), ovol.weight)
        res = oracle.track(search, depths[f], abi(intr), templ, P @ rels[f], oparams)
        assert not res.lost
        P = res.pose
        out.append(P)
        oracle.integrate(ovol, depths[f], abi(intr), P)
    return out


def _check(seq, name, gpu, orc):
    ate = lambda poses: float(np.sqrt(np.mean([np.sum((poses[f][:3, 3] - seq.gt[f][:3, 3]) ** 2)
                                               for f in range(1, N_TRACKED + 1)])))
    dt = [pose_trans_err(gpu[f], orc[f]) for f in range(1, N_TRACKED + 1)]
    dr = [pose_rot_err(gpu[f], orc[f]) for f in range(1, N_TRACKED + 1)]
    print(f"closed loop ({name}), frames 1-{N_TRACKED}: GPU vs oracle position difference max "
          f"{1e3 * max(dt):.4f} mm, rotation max {max(dr):.2e} rad; ATE GPU {100 * ate(gpu):.3f} cm, "
          f"oracle {100 * ate(orc):.3f} cm")
    assert max(dt) <= 1e-3, (name, dt)
    assert max(dr) <= 1e-3, (name, dr)
    assert abs(ate(gpu) - ate(orc)) <= 1e-3, (name, ate(gpu), ate(orc))


def test_closed_loop_follows_the_oracle_at_full_size():
    """The float form against the FP64 oracle's loop; the reduced-precision
    form with a half-precision search view of the float grid against the
    oracle running the same method (FP64 fusion, searches on the fused grid
    rounded to half).  How far the rounding itself moves the loop from the
    unrounded oracle is printed, not bounded: on this trajectory the
    search's decisions are sensitive to rounding-level changes of E."""
    torch = torch_cuda()
    pf = load_pf()
    seq = synth.multiroom_sequence(300, 0)
    depths = [seq.depth(f) for f in range(N_TRACKED + 1)]
    rels = [np.eye(4)] + [seq.relative_init(f) for f in range(1, N_TRACKED + 1)]
    templ = synth.templates(K, 0)
    gpu32 = _gpu_loop(pf, torch, seq, depths, rels, templ, pf.PF_F32)
    gpu16 = _gpu_loop(pf, torch, seq, depths, rels, templ, pf.PF_F16)
    orc64 = _oracle_loop(seq, depths, rels, templ)
    _check(seq, "f32", gpu32, orc64)
    orc16 = _oracle_loop(seq, depths, rels, templ, "f16")
    _check(seq, "f32 + f16 search view", gpu16, orc16)
    cost = [1e3 * pose_trans_err(orc16[f], orc64[f]) for f in range(1, N_TRACKED + 1)]
    print("rounding the search grid to half moves the oracle's own loop by (mm): "
          + ", ".join(f"{c:.3f}" for c in cost))
