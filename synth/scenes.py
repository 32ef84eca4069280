"""Analytic scenes: closed-form signed distances and exact ray casting.

Every primitive gives (a) its signed distance f(X) (positive in free space,
negative inside matter) and (b) the first ray hit lambda > 0 of X = o + lambda d.
A scene is a list of primitives; its distance is the minimum over them and its
rendered depth is the nearest hit.  World frame: metres, z up.

Primitive kinds
  "room"     interior of an axis-aligned box; matter is outside it (walls).
  "box"      solid axis-aligned box.
  "sphere"   solid sphere.
  "cylinder" solid capped cylinder with a vertical (world z) axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import uniform01


@dataclass(frozen=True)
class Primitive:
    kind: str
    a: tuple  # room/box: lo corner; sphere: centre; cylinder: (cx, cy, z0)
    b: tuple  # room/box: hi corner; sphere: (radius,); cylinder: (radius, z1)


@dataclass
class Scene:
    name: str
    prims: list = field(default_factory=list)

    # ---- signed distance -------------------------------------------------
    def sdf(self, X: np.ndarray) -> np.ndarray:
        """Signed distance (metres) at points X[..., 3]; > 0 in free space."""
        X = np.asarray(X, dtype=np.float64)
        out = np.full(X.shape[:-1], np.inf)
        for p in self.prims:
            out = np.minimum(out, _prim_sdf(p, X))
        return out

    # ---- ray casting -----------------------------------------------------
    def intersect(self, o: np.ndarray, d: np.ndarray) -> np.ndarray:
        """First hit parameter lambda > 0 along o + lambda d (inf if none)."""
        o = np.asarray(o, dtype=np.float64)
        d = np.asarray(d, dtype=np.float64)
        out = np.full(d.shape[:-1], np.inf)
        for p in self.prims:
            out = np.minimum(out, _prim_hit(p, o, d))
        return out


def _box_sdf(lo, hi, X):
    c = 0.5 * (np.asarray(lo) + np.asarray(hi))
    h = 0.5 * (np.asarray(hi) - np.asarray(lo))
    q = np.abs(X - c) - h
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return outside + inside


def _prim_sdf(p: Primitive, X):
    if p.kind == "room":
        return -_box_sdf(p.a, p.b, X)
    if p.kind == "box":
        return _box_sdf(p.a, p.b, X)
    if p.kind == "sphere":
        return np.linalg.norm(X - np.asarray(p.a), axis=-1) - p.b[0]
    if p.kind == "cylinder":
        cx, cy, z0 = p.a
        r, z1 = p.b
        radial = np.hypot(X[..., 0] - cx, X[..., 1] - cy) - r
        zc, hz = 0.5 * (z0 + z1), 0.5 * (z1 - z0)
        axial = np.abs(X[..., 2] - zc) - hz
        outside = np.hypot(np.maximum(radial, 0.0), np.maximum(axial, 0.0))
        inside = np.minimum(np.maximum(radial, axial), 0.0)
        return outside + inside
    raise ValueError(p.kind)


def _slabs(lo, hi, o, d):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (np.asarray(lo) - o) * inv
        t2 = (np.asarray(hi) - o) * inv
    # a zero direction component: the slab is either always or never crossed
    par = d == 0.0
    inside_slab = (o >= np.asarray(lo)) & (o <= np.asarray(hi))
    tmin_ax = np.where(par, np.where(inside_slab, -np.inf, np.inf), np.minimum(t1, t2))
    tmax_ax = np.where(par, np.where(inside_slab, np.inf, -np.inf), np.maximum(t1, t2))
    return np.max(tmin_ax, axis=-1), np.min(tmax_ax, axis=-1)


def _prim_hit(p: Primitive, o, d):
    o = np.broadcast_to(o, d.shape)
    if p.kind == "room":
        tmin, tmax = _slabs(p.a, p.b, o, d)
        ok = (tmax > 0.0) & (tmin <= 0.0)  # camera inside the room
        return np.where(ok, tmax, np.inf)
    if p.kind == "box":
        tmin, tmax = _slabs(p.a, p.b, o, d)
        ok = (tmax >= tmin) & (tmin > 0.0)
        return np.where(ok, tmin, np.inf)
    if p.kind == "sphere":
        c = np.asarray(p.a)
        r = p.b[0]
        oc = o - c
        A = np.sum(d * d, axis=-1)
        B = np.sum(oc * d, axis=-1)
        C = np.sum(oc * oc, axis=-1) - r * r
        disc = B * B - A * C
        with np.errstate(invalid="ignore"):
            sq = np.sqrt(np.maximum(disc, 0.0))
            t0 = (-B - sq) / A
            t1 = (-B + sq) / A
        t = np.where(t0 > 0.0, t0, np.where(t1 > 0.0, t1, np.inf))
        return np.where(disc >= 0.0, t, np.inf)
    if p.kind == "cylinder":
        cx, cy, z0 = p.a
        r, z1 = p.b
        ox, oy, oz = o[..., 0] - cx, o[..., 1] - cy, o[..., 2]
        dx, dy, dz = d[..., 0], d[..., 1], d[..., 2]
        A = dx * dx + dy * dy
        B = ox * dx + oy * dy
        C = ox * ox + oy * oy - r * r
        disc = B * B - A * C
        with np.errstate(invalid="ignore", divide="ignore"):
            sq = np.sqrt(np.maximum(disc, 0.0))
            ts = (-B - sq) / A
            zs = oz + ts * dz
            side = np.where((disc >= 0.0) & (A > 0.0) & (ts > 0.0) & (zs >= z0) & (zs <= z1), ts, np.inf)
            best = side
            for zc in (z0, z1):
                tc = (zc - oz) / dz
                px, py = ox + tc * dx, oy + tc * dy
                cap = np.where((dz != 0.0) & (tc > 0.0) & (px * px + py * py <= r * r), tc, np.inf)
                best = np.minimum(best, cap)
        return best
    raise ValueError(p.kind)


# ---------------------------------------------------------------------------
# The scenes of the workloads
# ---------------------------------------------------------------------------

def room_scene(seed: int = 0) -> Scene:
    """Single room: a 3.2 m axis-aligned box with 10 cm walls (3.0 m interior,
    x, y, z in [0.1, 3.1]) and 3 solid spheres of radius 0.2-0.5 m at seeded
    positions well inside the room."""
    u = uniform01(1000 + seed, 12)
    prims = [Primitive("room", (0.1, 0.1, 0.1), (3.1, 3.1, 3.1))]
    for s in range(3):
        r = 0.2 + 0.3 * u[4 * s + 3]
        lo, hi = 0.1 + r + 0.25, 3.1 - r - 0.25
        c = tuple(float(lo + (hi - lo) * u[4 * s + a]) for a in range(3))
        prims.append(Primitive("sphere", c, (float(r),)))
    return Scene("room3", prims)


def multiroom_scene() -> Scene:
    """Two rooms joined by a doorway, with boxes, cylinders and spheres, inside
    a 5.12 m cube (x, y in [0.25, 4.85], z in [0.25, 3.05])."""
    P = Primitive
    prims = [
        P("room", (0.25, 0.25, 0.25), (4.85, 4.85, 3.05)),
        # dividing wall at x = 3.0 with a 1 m doorway (y 1.9-2.9) under a lintel
        P("box", (2.95, 0.25, 0.25), (3.05, 1.90, 3.05)),
        P("box", (2.95, 2.90, 0.25), (3.05, 4.85, 3.05)),
        P("box", (2.95, 1.90, 2.25), (3.05, 2.90, 3.05)),
        # partial wall in the right room
        P("box", (3.05, 3.45, 0.25), (4.00, 3.55, 2.40)),
        # furniture
        P("box", (0.70, 3.60, 0.25), (1.60, 4.50, 0.95)),    # table
        P("box", (0.35, 0.40, 0.25), (0.95, 1.40, 2.00)),    # cabinet
        P("box", (3.60, 0.60, 0.25), (4.30, 1.10, 0.60)),    # low box
        P("box", (1.90, 0.35, 0.25), (2.60, 0.75, 1.10)),    # dresser
        P("cylinder", (2.55, 4.35, 0.25), (0.18, 3.05)),     # pillar
        P("cylinder", (4.10, 2.30, 0.25), (0.30, 1.20)),     # drum
        P("cylinder", (0.70, 2.20, 0.25), (0.22, 0.80)),     # stool
        P("sphere", (1.15, 4.05, 1.20), (0.25,)),
        P("sphere", (3.70, 4.20, 0.70), (0.35,)),
        P("sphere", (4.30, 2.30, 1.55), (0.25,)),
        P("sphere", (2.40, 1.20, 2.40), (0.20,)),
    ]
    return Scene("multiroom", prims)
