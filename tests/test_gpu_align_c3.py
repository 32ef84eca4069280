"""The alignment loss and its derivatives at the size the bench times them:
320x240 frames of the multiroom trajectory against a 256^3 volume at 2 cm
(truncation 6 cm), fused on the GPU from eight views.  Four frames, at their
true poses perturbed by up to 1 deg / 1 cm (one of them also at a nonzero
left perturbation xi and with upstream gradients), are compared with the
FP64 oracle run on the downloaded grid: counts exact, loss within 1e-5
relative, dL/dxi within 1e-5 of its norm, dL/dV within 1e-5 relative plus
1e-6 (the tolerances of test_gpu_align)."""
import numpy as np
import pytest

import oracle
import synth

from gpu_helpers import abi, load_pf, to_dev, torch_cuda
from test_gpu_align import _check_against_oracle

pytestmark = pytest.mark.gpu


def test_align_loss_and_gradients_at_the_benchmark_shape():
    torch = torch_cuda()
    pf = load_pf()
    intr = synth.Intrinsics(320, 240, 262.5, 262.5, 159.5, 119.5, 0.1, 8.0)
    grid = synth.Grid(256, 256, 256, 0.02, 0.06, (0.0, 0.0, 0.0))
    seq = synth.multiroom_sequence(300, 0, grid=grid, intr=intr)
    vol = pf.Volume.from_grid(grid)
    fused = [4 * i for i in range(8)]
    depth = {f: to_dev(seq.depth(f)) for f in fused}
    for f in fused:
        vol.integrate(depth[f], intr, seq.gt[f])
    ts, ws = vol.download()
    ovol = oracle.Volume(abi(grid), ts, ws)

    frames = [0, 8, 16, 28]
    n_max = intr.width * intr.height
    P = np.full((len(frames), n_max, 4), np.nan, dtype=np.float32)
    counts = np.zeros(len(frames), dtype=np.int32)
    for i, f in enumerate(frames):
        p, n = pf.backproject(depth[f], intr)
        n = int(n.item())
        P[i, :n] = p[:n].cpu().numpy()
        counts[i] = n
    u = synth.uniform01(91, 2 * len(frames))
    poses = np.stack([seq.gt[f] @ synth.perturbation(92, i, 1.0 * u[2 * i], 1.0 * u[2 * i + 1])
                      for i, f in enumerate(frames)])
    xi = np.zeros((len(frames), 6))
    xi[2] = [0.004, -0.003, 0.002, 0.003, 0.001, -0.002]
    dloss = np.array([1.0, 0.25, -1.5, 2.0])
    loss, cnt, gx, gV = vol.align_loss(to_dev(P), to_dev(poses), counts=to_dev(counts), xi=to_dev(xi),
                                       dloss=to_dev(dloss), grad_xi=True, grad_tsdf=True)
    torch.cuda.synchronize()
    assert np.all(counts > 0.5 * n_max)
    _check_against_oracle(ovol, P, counts, poses, xi,
                          (loss.cpu().numpy(), cnt.cpu().numpy(), gx.cpu().numpy()), gV.cpu().numpy(), dloss)
    vol.close()
