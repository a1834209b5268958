"""Seeded synthetic inputs: box meshes and the hierarchical-P2 systems of Sec. 2.

This package produces the problem data (the block systems of Sec. 2.4 with node
tags and right-hand sides) that both the CUDA path and the CPU oracle consume.
It contains no step of the multigrid method of Sec. 3.
"""
from .mesh import BoxMesh, box_mesh, boundary_faces  # noqa: F401
from .problems import (KIND_CODES, TAG_DIRICHLET, TAG_EDGE, TAG_VERTEX, Problem,  # noqa: F401
                       elasticity_problem, elasticity_quadratic_problem, lame,
                       mixed_elasticity_problem, rigid_body_modes, stokes_lid_problem,
                       paper_setting_problem, unconstrained_elasticity,
                       vector_laplace_problem)
from .configs import CONFIGS, make_config  # noqa: F401
