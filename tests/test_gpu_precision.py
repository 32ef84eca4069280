"""Reduced-precision storage: half / bfloat16 / scaled e4m3 TSDF (and cell
view), uint8 fusion weights.  Every operation stays float; only stored
values narrow.

Two questions, two kinds of test.
  1. Is the arithmetic unchanged?  A 16-bit volume holds a rounded grid.  The
     fitness and the search run on it must match the FP64 oracle run on that
     same rounded grid (downloaded and decoded) with the float-storage
     tolerances of the parity tests.
  2. How far does the rounding move fusion?  Each update of the running
     average (Sec. III, fusion as in KinectFusion) re-rounds the stored
     value, and the average only damps earlier errors (factor w / (w + 1)),
     so after n updates a node is off the FP64 result by at most n
     half-units-in-the-last-place of the format just below 1 (2^-12 for
     half, 2^-9 for bfloat16, 2^-5 for e4m3 holding 256 x the value) plus
     the float tolerance.  Weights are integers below 256 and stay exact in
     uint8.
The measured deviations are printed (run with -s to see them).
"""
import numpy as np
import pytest

import oracle
import synth
from synth import Grid, Intrinsics

from gpu_helpers import (abi, compare_fitness, load_pf, perturbed_poses, pose_rot_err, pose_trans_err, to_dev,
                         torch_cuda)

pytestmark = pytest.mark.gpu

# half-ulp just below 1.0 of each storage format (e4m3 holds 256 x the
# value: in [128, 256) its step is 16, i.e. 1/16 of the value's unit)
HALF_ULP = {"f16": 2.0 ** -12, "bf16": 2.0 ** -9, "fp8": 2.0 ** -5}


def _e4m3_values():
    """All non-negative finite e4m3 values by code (bias 7, 3 mantissa bits,
    subnormals at exponent 0, the all-ones code is NaN)."""
    out = []
    for code in range(0x7f):
        e, m = code >> 3, code & 7
        out.append(m / 8.0 * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(out)


@pytest.fixture(scope="module")
def pf():
    torch_cuda()
    return load_pf()


def dtype_code(pf, name):
    return {"f32": pf.PF_F32, "f16": pf.PF_F16, "bf16": pf.PF_BF16, "fp8": pf.PF_FP8E4M3}[name]


def round_storage(x, name):
    """Round float32 values to the storage format (to nearest, ties to even)
    and back to float32."""
    x = np.asarray(x, dtype=np.float32)
    if name == "f16":
        return x.astype(np.float16).astype(np.float32)
    if name == "bf16":
        b = x.view(np.uint32).astype(np.uint64)
        r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return r.astype(np.uint32).view(np.float32)
    if name == "fp8":
        # 256 x the value to the nearest e4m3 value (ties to the even code)
        vals = _e4m3_values()
        a = np.abs(x.astype(np.float64)) * 256.0
        hi = np.clip(np.searchsorted(vals, a), 1, len(vals) - 1)
        lo = hi - 1
        dlo, dhi = a - vals[lo], vals[hi] - a
        pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
        pick = np.where(a >= vals[-1], len(vals) - 1, pick)
        return (np.sign(x) * vals[pick] / 256.0).astype(np.float32)
    return x


def expected_download(tsdf, weight, name):
    """What a volume of storage `name` returns after upload(tsdf, weight):
    observed values rounded, a value that rounds to +-1 reads back as +-1
    (the outside-the-band code), unobserved nodes read 1."""
    r = round_storage(tsdf, name)
    r = np.where(r >= 1.0, 1.0, np.where(r <= -1.0, -1.0, r)).astype(np.float32)
    return np.where(weight > 0, r, np.float32(1.0))


def _room_inputs(seed=0, holes=0.03):
    scene, fr = synth.room64_frame(seed)
    tsdf, weight = synth.analytic_tsdf(scene, synth.ROOM64_GRID, hole_bricks=holes, seed=seed)
    return scene, fr, tsdf, weight


# ---------------------------------------------------------------------------
# storage round trip
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,u8", [("f16", 0), ("bf16", 0), ("f16", 1), ("f32", 1), ("fp8", 1)])
def test_upload_download_rounds_to_storage(pf, name, u8):
    scene, fr, tsdf, weight = _room_inputs()
    weight = np.minimum(weight, 200).astype(np.float32)
    # values near the band edge, where rounding reaches +-1
    tsdf = tsdf.copy()
    tsdf[:64] = np.linspace(0.99, 1.0, 64, dtype=np.float32)
    tsdf[64:128] = -np.linspace(0.99, 1.0, 64, dtype=np.float32)
    weight[:128] = 1.0
    vol = pf.Volume.from_grid(synth.ROOM64_GRID, tsdf_dtype=dtype_code(pf, name), weight_u8=u8)
    vol.upload(tsdf, weight)
    t, w = vol.download()
    assert np.array_equal(w, weight)
    assert np.array_equal(t, expected_download(tsdf, weight, name))
    if u8:
        with pytest.raises(pf.ProfusionError):
            vol.upload(tsdf, np.where(weight > 0, weight + 0.5, 0).astype(np.float32))


# ---------------------------------------------------------------------------
# arithmetic parity on the stored grid
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["f16", "bf16", "fp8"])
@pytest.mark.parametrize("K,N,spread,view", [(1024, None, 8.0, 1), (1000, 12345, 0.05, 1), (37, 777, 1.0, 1),
                                             (1024, None, 8.0, 2), (1000, 12345, 0.05, 2)])
def test_fitness_parity_on_stored_grid(pf, name, K, N, spread, view):
    """view 1: the full cell view (lanes on particles read float records);
    2: the narrow view (they convert the 16-/8-bit records on load)."""
    scene, fr, tsdf, weight = _room_inputs()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID, tsdf_dtype=dtype_code(pf, name), cell_view=view)
    assert vol.info()["cell_view"] == view
    vol.upload(tsdf, weight)
    ts, ws = vol.download()
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), ts, ws)
    pts = synth.render_points(scene, synth.ROOM64_INTR, fr.gt_pose)
    if N is not None:
        pts = pts[:N]
    poses = perturbed_poses(fr.gt_pose, K, spread, spread, seed=K + 5)
    orc = oracle.fitness(ovol, pts, poses, ambiguity=True, cap=64)
    assert np.all(orc.amb <= 64)
    results = {}
    for mapping in range(3):
        for layout in (2, 3):
            vol.set_fitness_variant(layout + 4 * mapping)
            E, C = vol.fitness(to_dev(pts), to_dev(poses))
            results[layout, mapping] = (E.cpu().numpy(), C.cpu().numpy())
            compare_fitness(*results[layout, mapping], orc)
        # (e4m3 cell records are read in a scaled form, so their roundings
        # differ from the node layout's; 16-bit records are bit-identical)
        if mapping > 0 and name != "fp8":
            assert np.array_equal(results[2, mapping][0], results[3, mapping][0])
    # the plain layout reads float arrays and is refused for 16-bit storage
    with pytest.raises(pf.ProfusionError):
        vol.set_fitness_variant(1)


@pytest.mark.parametrize("name", ["f16", "bf16"])
@pytest.mark.parametrize("view,mapping", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_cell_view_follows_fusion_16bit(pf, name, view, mapping):
    """After fusion into a 16-bit grid the cell view (raw corners, and float
    records in the full view) gives the same fitness as the node layout, bit
    for bit, with lanes on points (mapping 1) and on particles (2)."""
    grid, intr = synth.ROOM64_GRID, synth.ROOM64_INTR
    scene = synth.room_scene(0)
    vol = pf.Volume.from_grid(grid, tsdf_dtype=dtype_code(pf, name), weight_u8=1, cell_view=view)
    for j in (0, 1, 2):
        P = synth.room_view(scene, j)
        vol.integrate(to_dev(synth.add_depth_noise(synth.render_depth(scene, intr, P), 50 + j, 0.002)), intr, P)
    P = synth.room_view(scene, 1)
    pts = to_dev(synth.render_points(scene, intr, P))
    poses = to_dev(perturbed_poses(P, 512, 4.0, 4.0, seed=3))
    out = []
    for layout in (2, 3):
        vol.set_fitness_variant(layout + 4 * mapping)
        E, C = vol.fitness(pts, poses)
        out.append((E.cpu().numpy(), C.cpu().numpy()))
    assert np.count_nonzero(out[0][1]) > 100
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_volume_info_reports_storage_and_view(pf):
    grid = synth.ROOM64_GRID
    n = grid.n_nodes
    info = {}
    for name, ts in (("f32", 4), ("f16", 2), ("bf16", 2), ("fp8", 1)):
        for view in (-1, 0, 1, 2):
            vol = pf.Volume.from_grid(grid, tsdf_dtype=dtype_code(pf, name), weight_u8=1, cell_view=view)
            info[name, view] = vol.info()
            vol.close()
        assert info[name, -1] == {"storage_bytes": n * (ts + 1), "cell_view": -1}
        # a small grid takes the full view on its own
        assert info[name, 0] == info[name, 1] and info[name, 1]["cell_view"] == 1
        full, narrow = info[name, 1]["storage_bytes"], info[name, 2]["storage_bytes"]
        if name == "f32":
            assert info[name, 2] == info[name, 1]
        else:
            assert info[name, 2]["cell_view"] == 2 and full - narrow == 32 * n
        # records of 8 values, plus a few bytes of fusion stamps
        assert 0 <= narrow - n * (ts + 1) - 8 * ts * n < 65536
    print("\nprecision: storage bytes per node (u8 weights; none / narrow / full view): " + ", ".join(
        f"{nm} {info[nm, -1]['storage_bytes'] / n:.0f}/{info[nm, 2]['storage_bytes'] / n:.0f}/"
        f"{info[nm, 1]['storage_bytes'] / n:.0f}" for nm in ("f32", "f16", "bf16", "fp8")))


@pytest.mark.parametrize("name", ["f16", "bf16", "fp8"])
def test_track_parity_on_stored_grid(pf, name):
    torch = torch_cuda()
    K, iters = 1024, 10
    scene, fr, tsdf, weight = _room_inputs(0, holes=0.0)
    vol = pf.Volume.from_grid(synth.ROOM64_GRID, tsdf_dtype=dtype_code(pf, name), weight_u8=1)
    vol.upload(tsdf, weight)
    ts, ws = vol.download()
    ovol = oracle.Volume(abi(synth.ROOM64_GRID), ts, ws)
    templ = synth.templates(K, 0)
    params = pf.track_params(torch.from_numpy(templ).cuda(), n_iters=iters, k_sched=(K, K, K),
                             decim_sched=(1, 1, 1), update_mode=0, compose_mode=1)
    status, pose, st = vol.track_frame(to_dev(fr.depth), synth.ROOM64_INTR, params, fr.init_pose)
    oparams = oracle.TrackParams(n_iters=iters, k_sched=(K, K, K), decim_sched=(1, 1, 1), update_mode=0,
                                 compose_mode=1)
    ores = oracle.track(ovol, fr.depth, abi(synth.ROOM64_INTR), templ, fr.init_pose, oparams)
    assert status == pf.PF_OK and not ores.lost
    os_ = ores.stats
    assert st["n_points"] == os_["n_points"]
    strict = 0
    for i in range(iters):
        if not (os_["best_gap"][i] > 3e-5 and os_["adv_margin"][i] > 3e-5):
            break
        strict += 1
        assert st["best"][i] == os_["best"][i] and st["n_adv"][i] == os_["n_adv"][i], i
        np.testing.assert_allclose(st["pose"][i], os_["pose"][i], atol=1e-5)
    assert strict >= 2
    assert pose_trans_err(pose, ores.pose) <= 1e-4 and pose_rot_err(pose, ores.pose) <= 1e-4
    print(f"\nprecision: track {name}: |t - t_gt| = {100 * pose_trans_err(pose, fr.gt_pose):.3f} cm, "
          f"rot {np.degrees(pose_rot_err(pose, fr.gt_pose)):.4f} deg")


@pytest.mark.parametrize("name", ["f16", "bf16", "fp8"])
def test_raycast_parity_on_stored_grid(pf, name):
    """Ray casting a narrow grid fused on the GPU against the oracle's ray
    cast of the same stored values (downloaded and decoded)."""
    grid = Grid(72, 72, 72, 0.05, 0.15, (-0.2, -0.2, -0.2))
    intr = Intrinsics(160, 120, 140.0, 140.0, 79.5, 59.5)
    scene = synth.room_scene(2)
    vol = pf.Volume.from_grid(grid, tsdf_dtype=dtype_code(pf, name), weight_u8=1)
    for j in range(8):
        P = synth.room_view(scene, j)
        vol.integrate(to_dev(synth.add_depth_noise(synth.render_depth(scene, intr, P), 50 + j, 0.002)), intr, P)
    ts, ws = vol.download()
    ovol = oracle.Volume(abi(grid), ts, ws)
    P = synth.room_view(scene, 0)
    d, n = vol.raycast(intr, P)
    d, n = d.cpu().numpy(), n.cpu().numpy()
    od, on = oracle.raycast(ovol, abi(intr), P)
    both = (d > 0) & (od > 0)
    assert np.count_nonzero(both) > 0.3 * d.size
    assert np.mean((d > 0) == (od > 0)) > 0.995
    assert np.mean(np.abs(d[both] - od[both]) < 1e-4) > 0.995
    good = both & np.isfinite(n[..., 0]) & np.isfinite(on[..., 0])
    assert np.mean(np.sum(n[good] * on[good], axis=-1) > 0.999) > 0.99


# ---------------------------------------------------------------------------
# fusion: deviation from the FP64 oracle bounded by the storage rounding
# ---------------------------------------------------------------------------

FUSION = {
    "room64": (synth.ROOM64_GRID, synth.ROOM64_INTR),
    "ragged": (Grid(67, 45, 39, 0.061, 0.17, (0.07, 0.53, -0.21)), Intrinsics(97, 61, 80.0, 82.0, 47.3, 31.1)),
}


@pytest.mark.parametrize("case", sorted(FUSION))
@pytest.mark.parametrize("name,u8", [("f16", 0), ("bf16", 0), ("f16", 1), ("bf16", 1), ("f32", 1), ("fp8", 1)])
def test_fusion_error_bound(pf, case, name, u8):
    grid, intr = FUSION[case]
    scene = synth.room_scene(0)
    n_views = 8
    vol = pf.Volume.from_grid(grid, tsdf_dtype=dtype_code(pf, name), weight_u8=u8)
    ovol = oracle.Volume(abi(grid))
    amb = np.zeros(grid.n_nodes, dtype=bool)
    for j in range(n_views):
        P = synth.room_view(scene, j)
        depth = synth.add_depth_noise(synth.render_depth(scene, intr, P), 70 + j, 0.003)
        vol.integrate(to_dev(depth), intr, P)
        amb |= oracle.integrate(ovol, depth, abi(intr), P, ambiguity=True, eps_px=3e-4).astype(bool)
    t, w = vol.download()
    ok = ~amb
    obs = ok & (ovol.weight > 0)
    assert np.count_nonzero(obs) > 1000
    assert np.array_equal(w[ok], ovol.weight[ok].astype(np.float32))
    err = np.abs(t[obs].astype(np.float64) - ovol.tsdf[obs])
    n_upd = ovol.weight[obs]
    bound = n_upd * HALF_ULP.get(name, 0.0) + 1e-5
    assert np.all(err <= bound), float(np.max(err - bound))
    assert np.all(t[ok & (ovol.weight == 0)] == 1.0)
    print(f"\nprecision: fusion {case} {name}{'+u8' if u8 else ''}: {n_views} views, "
          f"tsdf rms {np.sqrt(np.mean(err ** 2)):.3e}, max {err.max():.3e} (bound at max weight "
          f"{int(n_upd.max()) * HALF_ULP.get(name, 0.0) + 1e-5:.3e})")
