"""Seeded synthetic inputs for repeated-pattern FETI (Gosselet, Rixen & Rey, arXiv 1208.6387).

Meshes, occurrence layouts, rotations, signed Boolean links and loads; nothing of the FETI arithmetic.
Both the CUDA library's tests/bench and the CPU oracle read the same Problem objects made here.
"""
from .mesh import Pattern, heat_pattern, elastic_pattern, q1_laplace, q1_elastic3d, elastic_D, lame
from .layout import Problem, Occurrence, build_grid_problem, cube_rotations, square_rotations, dense_B, set_nodal_load
from .configs import (heat_grid, elastic_grid, config, library_patterns, fill_structure, request_stream, LIBRARY,
                      merge_structures, batched_uneven)
from .ring import (ring_heat, ring_elastic, ring_structure, ring_permutation, sector_pattern, q1_laplace_quad,
                   q1_plane_strain_quad)
