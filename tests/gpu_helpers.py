"""Shared set-up of the GPU parity tests (inputs from synth, expectations from
the oracle; nothing here computes any step of the method)."""
import numpy as np

import synth


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def load_pf():
    from paper_2509_24236_gb300 import build
    build.build()
    import paper_2509_24236_gb300 as pf
    pf.load()
    return pf


def to_dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def pose_rot_err(Pa, Pb):
    R = Pa[:3, :3].T @ Pb[:3, :3]
    return float(np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))


def pose_trans_err(Pa, Pb):
    return float(np.linalg.norm(Pa[:3, 3] - Pb[:3, 3]))


def perturbed_poses(P, K, max_deg, max_cm, seed):
    """K float32 3x4 poses: P itself first, then seeded perturbations."""
    out = np.empty((K, 12), dtype=np.float32)
    out[0] = P[:3, :4].reshape(12)
    u = synth.uniform01(seed, 2 * K)
    for k in range(1, K):
        D = synth.perturbation(seed + 1, k, max_deg * u[2 * k], max_cm * u[2 * k + 1])
        out[k] = (P @ D)[:3, :4].reshape(12)
    return out


def compare_fitness(E_gpu, C_gpu, orc, rel=1e-5):
    """Element-wise check of GPU fitness against the oracle, allowing the
    points the oracle flags as lying on a validity boundary to flip.
    Returns the number of particles with any flagged point."""
    E_o, C_o, amb = orc.E, orc.C, orc.amb
    K = len(E_o)
    assert E_gpu.shape == (K,) and C_gpu.shape == (K,)
    for k in range(K):
        a = int(amb[k]) if amb is not None else 0
        if a == 0:
            assert C_gpu[k] == C_o[k], (k, C_gpu[k], C_o[k])
            if C_o[k] == 0:
                assert np.isinf(E_gpu[k])
            else:
                assert abs(E_gpu[k] - E_o[k]) <= rel * E_o[k] + 1e-12, (k, E_gpu[k], E_o[k])
        else:
            assert abs(int(C_gpu[k]) - int(C_o[k])) <= a
            if C_o[k] > 0 and C_gpu[k] > 0:
                assert abs(E_gpu[k] - E_o[k]) <= rel * E_o[k] + 2.0 * a / min(C_o[k], C_gpu[k])
    return int(np.count_nonzero(amb)) if amb is not None else 0
