"""Ray casting of a fused TSDF against the analytic surface (the closed-form
ray intersection and face normals of the room's walls), on the GPU.

Noise-free views of the room are fused; the depth cast from a further view
must lie within half a voxel of the analytic depth on pixels that see a wall
away from edges (the fused zero crossing of a plane lies within vs/2 of it).
The normal is the gradient of the fused field, and a projective TSDF (the
distance along the camera axis, Sec. III) is not the Euclidean distance: for
a wall seen at an angle its gradient leans towards the viewing directions of
the fused views, so the normal is only checked to face the camera and to lie
within 30 degrees of the wall's normal on 95% of the wall pixels.
"""
import numpy as np
import pytest

import synth

from gpu_helpers import load_pf, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_raycast_depth_and_normals_match_the_analytic_room():
    torch = torch_cuda()
    pf = load_pf()
    scene = synth.room_scene(0)
    grid, intr = synth.ROOM64_GRID, synth.ROOM64_INTR
    vol = pf.Volume.from_grid(grid)
    for j in range(8):
        P = synth.room_view(scene, j)
        vol.integrate(to_dev(synth.render_depth(scene, intr, P)), intr, P)
    P = synth.room_view(scene, 3)
    depth, normals = vol.raycast(intr, P)
    torch.cuda.synchronize()
    d = depth.cpu().numpy()
    n = normals.cpu().numpy()
    ref = synth.render_depth(scene, intr, P)
    # pixels on walls (not spheres), with the analytic depth smooth around them
    walls_only = synth.render_depth(synth.Scene(scene.name, [p for p in scene.prims if p.kind == "room"]), intr, P)
    on_wall = (np.abs(walls_only - ref) < 1e-9) & (ref > 0)
    smooth = np.zeros_like(on_wall)
    smooth[2:-2, 2:-2] = True
    for dy in (-2, 0, 2):
        for dx in (-2, 0, 2):
            smooth &= np.roll(np.roll(on_wall, dy, 0), dx, 1)
    sel = smooth & (d > 0)
    assert np.count_nonzero(sel) > 0.3 * d.size
    err = np.abs(d[sel] - ref[sel])
    assert np.max(err) <= 0.5 * grid.voxel_size, float(np.max(err))
    # wall normals are axis-aligned in the world; the cast normal is in world coordinates
    nn = n[sel]
    ok = np.all(np.isfinite(nn), axis=1)
    assert np.count_nonzero(ok) > 0.95 * len(nn)
    cos = np.max(np.abs(nn[ok]), axis=1)  # |component along the wall's axis|
    ang = np.degrees(np.arccos(np.clip(cos, -1, 1)))
    assert np.percentile(ang, 95) < 30.0, np.percentile(ang, 95)
    # facing the camera: negative along the viewing ray
    v, u = np.nonzero(sel)
    rays = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, np.ones_like(u, dtype=np.float64)], 1)
    rays_w = rays @ P[:3, :3].T
    assert np.mean(np.sum(nn[ok] * rays_w[ok], axis=1) < 0) > 0.99
