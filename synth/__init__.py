"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This package holds no arithmetic of the method itself (no voxelization, no
covariance, no residual): only random numbers, scene geometry and poses.
"""
from .rng import Stream
from .scenes import (Workload, box_room, corridor, urban, terrain, make_pose, rot_axis_angle,
                     to_local, perturb_pose)

__all__ = ["Stream", "Workload", "box_room", "corridor", "urban", "terrain", "make_pose",
           "rot_axis_angle", "to_local", "perturb_pose"]
