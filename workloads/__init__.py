"""Seeded synthetic inputs shaped like the paper's 2D/3D scenarios.

This module holds no arithmetic of the multigrid method: only media generators
(velocity fields and their conversion to Lame parameters), frequency selection
and source placement. Both the FP64 oracle tests and the GPU path draw their
inputs from here, so the two share nothing else.
"""
from .media import (Workload, config_c1_homogeneous, config_c2_random2d, config_c3_layered3d, config_c4_batch,
                    config_c5_adjoint, small_heterogeneous, lame_from_velocity, gaussian_random_velocity,
                    point_source, random_field)

__all__ = ["Workload", "config_c1_homogeneous", "config_c2_random2d", "config_c3_layered3d", "config_c4_batch",
           "config_c5_adjoint", "small_heterogeneous", "lame_from_velocity", "gaussian_random_velocity",
           "point_source", "random_field"]
