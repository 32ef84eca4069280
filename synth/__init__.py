"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Analytic scenes with closed-form signed distances, exact depth rendering,
trajectories, depth noise, pose perturbations and the SplitMix64 particle
templates.  Nothing here computes any step of the pose search or of fusion:
random numbers the method consumes (the templates) are produced here and passed
to both implementations as inputs.
"""
from .camera import (Intrinsics, add_depth_noise, axis_angle_matrix, look_at, multiroom_trajectory,
                     perturbation, pose_matrix, relative, render_depth, render_points, room_view,
                     yaw_pitch_roll_pose)
from .rng import splitmix64, templates, uniform01
from .scenes import Primitive, Scene, multiroom_scene, room_scene
from .volume import Grid, analytic_tsdf
from .workloads import (MULTIROOM_GRID, MULTIROOM_INTR, ROOM64_GRID, ROOM64_INTR, Frame, Sequence,
                        default_templates, multiroom_sequence, room64_frame)
