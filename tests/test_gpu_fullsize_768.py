"""Parity at the largest workload: 640x480 depth into a 768^3 TSDF at 8 mm
(tau 2.4 cm) of the multiroom scene, stored in half precision with uint8
weights and the full cell view -- the reduced-precision configuration the
precision benchmark runs.  The grid holds 453 M nodes (22 GB on the device
with its cell view); the first frames observe about 5 M of them.

  * fusion of frames 0 and 1 at their true poses against the FP64 oracle's
    own fusion, every node: weights exact, tsdf within the storage's rounding
    bound (one half-ulp of half precision per update, plus the float
    tolerance);
  * the fitness of 3072 poses over every 4th point of frame 2, spread
    within 3 deg / 3 cm (lanes on points) and within 0.03 deg / 0.03 cm
    (lanes on particles), against the oracle run on the downloaded grid.
"""
import numpy as np
import pytest

import oracle
import synth

from gpu_helpers import abi, compare_fitness, load_pf, perturbed_poses, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

GRID = synth.Grid(768, 768, 768, 0.008, 0.024, (-0.5, -0.5, -0.5))
HALF_ULP_F16 = 2.0 ** -12   # half of half precision's spacing just below 1
K, FUSED = 3072, 2


@pytest.fixture(scope="module")
def fused768():
    torch_cuda()
    pf = load_pf()
    seq = synth.multiroom_sequence(300, 0, grid=GRID)
    intr = seq.intr
    vol = pf.Volume.from_grid(GRID, tsdf_dtype=pf.PF_F16, weight_u8=1, cell_view=1)
    ovol = oracle.Volume(abi(GRID))
    amb = np.zeros(GRID.n_nodes, dtype=bool)
    for f in range(FUSED):
        depth = seq.depth(f)
        vol.integrate(to_dev(depth), intr, seq.gt[f])
        amb |= oracle.integrate(ovol, depth, abi(intr), seq.gt[f], ambiguity=True, eps_px=3e-4).astype(bool)
    t, w = vol.download()
    yield pf, seq, vol, ovol, amb, (t, w)
    vol.close()


def test_768_fusion_into_half_storage(fused768):
    pf, seq, vol, ovol, amb, (t, w) = fused768
    assert vol.info()["cell_view"] == 1
    ok = ~amb
    updated = ovol.weight > 0
    assert np.count_nonzero(updated) > 3_000_000
    assert np.count_nonzero(amb) < 2e-2 * np.count_nonzero(updated)
    assert np.array_equal(w[ok], ovol.weight[ok].astype(np.float32))
    obs = ok & updated
    err = np.abs(t[obs].astype(np.float64) - ovol.tsdf[obs])
    bound = ovol.weight[obs] * HALF_ULP_F16 + 1e-5
    assert np.all(err <= bound), float(np.max(err - bound))
    assert np.all(t[ok & ~updated] == 1.0)


@pytest.mark.parametrize("spread", [3.0, 0.03])
def test_768_fitness_on_the_stored_grid(fused768, spread):
    pf, seq, vol, ovol, amb, (t, w) = fused768
    f = FUSED
    pts = oracle.backproject(seq.depth(f), abi(seq.intr), stride=4).astype(np.float32)
    pts = np.ascontiguousarray(np.c_[pts, np.zeros(len(pts), np.float32)])
    assert len(pts) > 50_000
    poses = perturbed_poses(seq.gt[f], K, spread, spread, seed=21)
    vol.set_fitness_variant(0)
    E, C = vol.fitness(to_dev(pts), to_dev(poses))
    grid_view = oracle.Volume(abi(GRID), t, w)
    orc = oracle.fitness(grid_view, pts[:, :3], poses.astype(np.float64), ambiguity=True, cap=128)
    assert np.all(orc.amb <= 128)
    assert np.count_nonzero(orc.C > 0) > K // 2
    compare_fitness(E.cpu().numpy(), C.cpu().numpy(), orc)
