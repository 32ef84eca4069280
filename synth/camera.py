"""Pinhole intrinsics, depth rendering, trajectories and pose perturbations.

Conventions (shared by every input built here)
  * Camera frame: x right, y down, z forward.  Pixel (u, v) are integer indices
    at pixel centres; a depth value is the z coordinate (metres) of the hit.
  * A pose is a 4x4 float64 camera-to-world matrix [R | t]: X_w = R X_c + t.
  * Depth value 0.0 means "no measurement".
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import uniform01


@dataclass(frozen=True)
class Intrinsics:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    depth_min: float = 0.1
    depth_max: float = 8.0


def axis_angle_matrix(axis, angle: float) -> np.ndarray:
    """Rotation by `angle` radians about the unit vector `axis` (input builder)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def pose_matrix(R: np.ndarray, t) -> np.ndarray:
    P = np.eye(4)
    P[:3, :3] = R
    P[:3, 3] = t
    return P


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world pose at `eye` whose optical axis points at `target`."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return pose_matrix(np.stack([r, d, f], axis=1), eye)


def yaw_pitch_roll_pose(eye, yaw: float, pitch: float, roll: float) -> np.ndarray:
    """Camera looking along heading `yaw` (about world z), tilted up by `pitch`
    and rolled by `roll` about its optical axis (radians)."""
    f = np.array([np.cos(pitch) * np.cos(yaw), np.cos(pitch) * np.sin(yaw), np.sin(pitch)])
    r = np.array([np.sin(yaw), -np.cos(yaw), 0.0])
    d = np.cross(f, r)
    c, s = np.cos(roll), np.sin(roll)
    r2 = c * r + s * d
    d2 = -s * r + c * d
    return pose_matrix(np.stack([r2, d2, f], axis=1), eye)


def render_depth(scene, intr: Intrinsics, pose: np.ndarray) -> np.ndarray:
    """Noise-free depth image (float32, H x W) of an analytic scene."""
    u = np.arange(intr.width, dtype=np.float64)
    v = np.arange(intr.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy, np.ones_like(uu)], axis=-1)
    dw = dc @ pose[:3, :3].T
    lam = scene.intersect(pose[:3, 3], dw)
    depth = np.where(np.isfinite(lam), lam, 0.0)
    return depth.astype(np.float32)


def render_points(scene, intr: Intrinsics, pose: np.ndarray, stride: int = 1) -> np.ndarray:
    """Camera-frame hit points (float32, N x 4, last column 0) of the rays
    of every `stride`-th pixel that hits the scene, in row-major order."""
    u = np.arange(intr.width, dtype=np.float64)
    v = np.arange(intr.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy, np.ones_like(uu)], axis=-1)
    lam = scene.intersect(pose[:3, 3], dc @ pose[:3, :3].T)
    hit = np.isfinite(lam).reshape(-1)
    pts = (dc * lam[..., None]).reshape(-1, 3)[hit][::stride]
    out = np.zeros((pts.shape[0], 4), dtype=np.float32)
    out[:, :3] = pts
    return out


def add_depth_noise(depth: np.ndarray, seed: int, sigma_const: float = 0.0,
                    sigma_quad: float = 0.0) -> np.ndarray:
    """Additive Gaussian noise with sigma = sigma_const + sigma_quad * z^2 on
    measured pixels (value 0 stays 0)."""
    rng = np.random.default_rng(seed)
    z = depth.astype(np.float64)
    n = rng.standard_normal(z.shape)
    out = np.where(z > 0.0, z + (sigma_const + sigma_quad * z * z) * n, 0.0)
    return out.astype(np.float32)


def random_unit(u1: float, u2: float) -> np.ndarray:
    z = 2.0 * u1 - 1.0
    phi = 2.0 * np.pi * u2
    rr = np.sqrt(max(0.0, 1.0 - z * z))
    return np.array([rr * np.cos(phi), rr * np.sin(phi), z])


def perturbation(seed: int, index: int, deg: float, cm: float) -> np.ndarray:
    """Rigid perturbation: exactly `deg` degrees about a seeded uniform axis and
    exactly `cm` centimetres along a seeded uniform direction (4x4)."""
    u = uniform01(seed, 4, offset=4 * index)
    R = axis_angle_matrix(random_unit(u[0], u[1]), np.deg2rad(deg))
    return pose_matrix(R, 0.01 * cm * random_unit(u[2], u[3]))


def relative(Pa: np.ndarray, Pb: np.ndarray) -> np.ndarray:
    """Relative pose P_(b,a) with Pb = Pa @ P_(b,a)."""
    return np.linalg.inv(Pa) @ Pb


# ---------------------------------------------------------------------------
# Trajectories
# ---------------------------------------------------------------------------

def multiroom_trajectory(n_frames: int = 300, fps: float = 30.0,
                         max_deg_s: float = 90.0, max_m_s: float = 1.0) -> list:
    """Camera loop in the left room of the multi-room scene.

    The eye runs along an ellipse (centre (1.65, 2.55), radii 0.55 x 1.1 m,
    height 1.45 +- 0.12 m) with a speed profile peaking at `max_m_s`, while the
    heading turns at 10-90 deg/s and the camera pitches and rolls gently; the
    angular speed is scaled so its maximum over the sequence is `max_deg_s`.
    """
    sub = 64
    T = n_frames / fps
    ts = np.linspace(0.0, T, n_frames * sub + 1)
    dt = ts[1] - ts[0]
    a, b, c = 0.55, 1.10, np.array([1.65, 2.55])
    speed = (0.55 + 0.45 * np.sin(2.0 * np.pi * ts / 3.3 + 1.0)) * max_m_s
    phi = np.zeros_like(ts)
    for i in range(1, len(ts)):
        dpdphi = np.hypot(a * np.sin(phi[i - 1]), b * np.cos(phi[i - 1]))
        phi[i] = phi[i - 1] + speed[i - 1] / dpdphi * dt
    yaw_rate = np.deg2rad(50.0 + 40.0 * np.sin(2.0 * np.pi * ts / 4.0))
    yaw = np.deg2rad(200.0) + np.concatenate([[0.0], np.cumsum(yaw_rate[:-1] * dt)])
    pitch = np.deg2rad(-12.0 + 10.0 * np.sin(2.0 * np.pi * ts / 3.7))
    roll = np.deg2rad(4.0 * np.sin(2.0 * np.pi * ts / 5.3))
    # scale the rotation speed so that its peak is max_deg_s
    rate = np.sqrt(np.gradient(yaw, dt) ** 2 + np.gradient(pitch, dt) ** 2 + np.gradient(roll, dt) ** 2)
    scale = np.deg2rad(max_deg_s) / rate.max()
    yaw = yaw[0] + (yaw - yaw[0]) * scale
    pitch = np.deg2rad(-12.0) + (pitch - np.deg2rad(-12.0)) * scale
    roll = roll * scale
    poses = []
    for f in range(n_frames):
        i = f * sub
        eye = np.array([c[0] + a * np.cos(phi[i]), c[1] + b * np.sin(phi[i]),
                        1.45 + 0.12 * np.sin(2.0 * np.pi * ts[i] / 4.7)])
        poses.append(yaw_pitch_roll_pose(eye, yaw[i], pitch[i], roll[i]))
    return poses


def room_view(scene, view: int = 0) -> np.ndarray:
    """A view from inside the single-room scene towards the spheres."""
    centres = np.array([p.a for p in scene.prims if p.kind == "sphere"])
    target = centres.mean(axis=0)
    eyes = [(0.55, 0.60, 2.00), (2.60, 0.50, 1.80), (2.55, 2.60, 2.40), (0.50, 2.55, 0.90),
            (1.60, 0.45, 0.60), (0.45, 1.60, 2.60), (2.65, 1.50, 0.50), (1.50, 2.70, 1.60)]
    return look_at(eyes[view % len(eyes)], target)
