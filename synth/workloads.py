"""The workloads, as seeded synthetic inputs.

room64     single frame: 3.2 m room with 3 spheres, 64^3 grid at 5 cm
           (truncation 15 cm), one 160x120 depth image (f = 140, c = (80, 60))
           with 1 mm Gaussian noise, initial pose = ground truth perturbed by
           5 deg and 5 cm, 1024 particles x 10 iterations.
multiroom  300-frame 30 Hz trajectory of 640x480 depth (f = 525,
           c = (319.5, 239.5), noise sigma = 0.0012 z^2) through a two-room
           scene held in a 512^3 grid at 1 cm (truncation 3 cm); initial poses
           are ground-truth relative poses perturbed by 3 deg and 3 cm;
           3072 particles x 20 iterations per frame, then fusion.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

from .camera import (Intrinsics, add_depth_noise, multiroom_trajectory, perturbation,
                     relative, render_depth, room_view)
from .rng import templates
from .scenes import multiroom_scene, room_scene
from .volume import Grid

ROOM64_INTR = Intrinsics(160, 120, 140.0, 140.0, 80.0, 60.0, 0.1, 8.0)
ROOM64_GRID = Grid(64, 64, 64, 0.05, 0.15, (0.0, 0.0, 0.0))
MULTIROOM_INTR = Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5, 0.1, 8.0)
MULTIROOM_GRID = Grid(512, 512, 512, 0.01, 0.03, (0.0, 0.0, 0.0))


@dataclass
class Frame:
    depth: np.ndarray          # float32 H x W
    gt_pose: np.ndarray        # 4x4 float64 camera-to-world
    init_pose: np.ndarray      # 4x4 float64 initial estimate


def room64_frame(seed: int = 0, view: int = 0, noise: bool = True,
                 deg: float = 5.0, cm: float = 5.0) -> tuple:
    """(scene, Frame) of the single-frame room workload."""
    scene = room_scene(seed)
    gt = room_view(scene, view)
    depth = render_depth(scene, ROOM64_INTR, gt)
    if noise:
        depth = add_depth_noise(depth, 100 + seed, sigma_const=0.001)
    init = gt @ perturbation(200 + seed, view, deg, cm)
    return scene, Frame(depth, gt, init)


@dataclass
class Sequence:
    """A lazily rendered depth sequence with per-frame perturbations."""
    scene: object
    intr: Intrinsics
    grid: Grid
    gt: list
    seed: int = 0
    deg: float = 3.0
    cm: float = 3.0
    noise_quad: float = 0.0012
    _cache: dict = field(default_factory=dict)

    def __len__(self):
        return len(self.gt)

    def depth(self, f: int) -> np.ndarray:
        if f not in self._cache:
            d = render_depth(self.scene, self.intr, self.gt[f])
            if self.noise_quad > 0.0:
                d = add_depth_noise(d, 10_000 * (self.seed + 1) + f, sigma_quad=self.noise_quad)
            self._cache[f] = d
        return self._cache[f]

    def relative_init(self, f: int, step: int = 1) -> np.ndarray:
        """Perturbed relative pose from frame f - step to frame f (the frames
        in between dropped): P0_f = P_{f-step} @ relative_init(f, step)."""
        return relative(self.gt[f - step], self.gt[f]) @ perturbation(300 + self.seed, f, self.deg, self.cm)


@lru_cache(maxsize=4)
def _multiroom_gt(n_frames: int):
    return tuple(multiroom_trajectory(n_frames))


def multiroom_sequence(n_frames: int = 300, seed: int = 0, grid: Grid = MULTIROOM_GRID,
                       intr: Intrinsics = MULTIROOM_INTR) -> Sequence:
    return Sequence(multiroom_scene(), intr, grid, list(_multiroom_gt(n_frames)), seed)


def default_templates(k_max: int = 10240, seed: int = 0) -> np.ndarray:
    return templates(k_max, seed)
