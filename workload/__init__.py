"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package generates *inputs only*: meshes (node coordinates, triangles,
Dirichlet flags, the refinement mask P), the random-field basis evaluated at
element centroids, the random draws xi, nodal initial data and the weights of
the box-average quantity of interest; ``workload.channel`` the narrow channel
of random width (reference mesh, vertex displacement mode, width draws,
line-mean weights).  It contains none of the method's
arithmetic (no mass or stiffness assembly, no time stepping, no MLMC
estimator); those live independently in ``oracle/`` and in the CUDA library.
"""
from .mesh import Mesh, lshape_graded_mesh, square_mesh, refined_mask_from_elements
from .fields import (point_source, psi_sine, xi_uniform, gaussian_bump, box_qoi_weights,
                     coarse_dt, SquareConfig, CONFIG_PLAIN, CONFIG_BATCHED,
                     CONFIG_BANDWIDTH, CONFIG_ADJOINT, level_problem, LShapeConfig,
                     CONFIG_LSHAPE, lshape_level, lshape_steps, xi_gaussian)

__all__ = ["Mesh", "square_mesh", "point_source", "refined_mask_from_elements", "psi_sine",
           "xi_uniform", "gaussian_bump", "box_qoi_weights", "coarse_dt",
           "SquareConfig", "CONFIG_PLAIN", "CONFIG_BATCHED",
           "CONFIG_BANDWIDTH", "CONFIG_ADJOINT", "level_problem", "LShapeConfig",
           "CONFIG_LSHAPE", "lshape_level", "lshape_steps", "xi_gaussian"]
