"""Shared set-up of the GPU parity tests (inputs from synth, expectations from
the oracle; nothing here computes any step of the method)."""
import numpy as np

import synth


def abi(x):
    """The same intrinsics or grid with every real parameter rounded to
    float32: the C ABI takes them as float, so the oracle must see the same
    numbers."""
    from dataclasses import fields, replace
    f32 = lambda v: float(np.float32(v))
    kw = {}
    for fd in fields(x):
        v = getattr(x, fd.name)
        if isinstance(v, float):
            kw[fd.name] = f32(v)
        elif isinstance(v, tuple):
            kw[fd.name] = tuple(f32(e) for e in v)
    return replace(x, **kw)


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


def compare_fitness(E_gpu, C_gpu, orc, rel=1e-5, floor=0.0):
    """Element-wise check of GPU fitness against the oracle.

    The oracle leaves out the points lying on a cell face across which
    validity changes (FP32 and FP64 may put them on either side) and reports
    the value each would add.  The GPU count must be the oracle's plus some
    m of those points, and the GPU fitness must match, within `rel`, the
    oracle's sum plus the values of some m of them, within `rel` (1e-5, the
    target's relative bound) plus an absolute `floor` -- zero for the
    product layouts, whose sample positions are formed from exact reference
    products (measured: at most 8.6e-7 relative over every parity case,
    converged E ~ 0.004 included); only the plain float baseline, which
    rounds each sample position at the scale of the grid coordinate, passes
    a floor.  Returns the number of poses that had ambiguous points."""
    from itertools import combinations
    from math import comb
    K = len(orc.E)
    assert E_gpu.shape == (K,) and C_gpu.shape == (K,)
    for k in range(K):
        a = int(orc.amb[k]) if orc.amb is not None else 0
        m = int(C_gpu[k]) - int(orc.C[k])
        assert 0 <= m <= a, (k, C_gpu[k], orc.C[k], a)
        if C_gpu[k] == 0:
            assert np.isinf(E_gpu[k])
            continue
        assert a <= orc.vals.shape[1] if orc.vals is not None else a == 0
        vals = np.sort(orc.vals[k, :a]) if a else np.zeros(0)
        ref = (orc.S[k] + vals[:m].sum()) / C_gpu[k]
        if comb(a, m) <= 5000:
            best = min(abs(E_gpu[k] - (orc.S[k] + sum(sub)) / C_gpu[k]) for sub in combinations(vals, m))
        else:
            # too many subsets to try: the sum must lie between the m smallest
            # and the m largest values
            lo = (orc.S[k] + vals[:m].sum()) / C_gpu[k]
            hi = (orc.S[k] + vals[a - m:].sum()) / C_gpu[k]
            best = max(0.0, lo - E_gpu[k], E_gpu[k] - hi)
        assert best <= rel * ref + floor, (k, E_gpu[k], ref, best / ref)
    return int(np.count_nonzero(orc.amb)) if orc.amb is not None else 0
