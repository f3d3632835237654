"""B300-native linearization of GLIM matching-cost factors (voxelized GICP, Sec. III-C).

The compute path is the CUDA library ``libglimlin.so`` (C ABI in ``include/glim_lin.h``);
this package only marshals arguments to it.  See ``api`` for the calls and ``autograd`` for
the differentiable cost.
"""
from .api import (ACC_FP32, ACC_FP64, ACC_KAHAN, Context, FrameData, GlimError, Plan, VoxelMap, backward,
                  correspondences, debug_fail_allocation, estimate_covariances, estimate_covariances_knn, frames_needed, gather_records,
                  gn_solve, graph_step, linearize, overlap, pack_records, shard_pairs, spatial_order, to_pts4,
                  unpack_records)

__all__ = ["ACC_FP32", "ACC_FP64", "ACC_KAHAN", "Context", "FrameData", "GlimError", "Plan", "VoxelMap",
           "backward", "correspondences", "debug_fail_allocation", "estimate_covariances", "estimate_covariances_knn", "frames_needed",
           "gather_records", "gn_solve", "graph_step", "linearize", "overlap", "pack_records", "shard_pairs",
           "spatial_order", "to_pts4", "unpack_records"]
