"""The five synthetic workloads (2D heat and 3D elasticity, shaped like the paper's thermal and elastic tests)
plus small variants for tests.  Every draw is seeded: numpy.random.default_rng([seed, purpose])."""
from __future__ import annotations

import numpy as np

from .layout import build_grid_problem, cube_rotations, square_rotations
from .mesh import elastic_pattern, heat_pattern


def heat_grid(m: int, grid=(2, 2), kappas=(1.0,), seed: int = 0, k=None, checker: bool = False,
              rotate: bool = False, dirichlet="x0", dirichlet_fn=None, load="uniform", name=None):
    """2D heat: square Q1 patterns of m x m elements on a grid; u = 0 on x = 0; f ~ U(0,1) per node."""
    pats = [heat_pattern(m, kappa=kap, name=f"heat{m}_k{kap:g}") for kap in kappas]
    n = grid[0] * grid[1]
    if checker:
        colour = int(np.random.default_rng([seed, 2]).integers(2))
        cp = np.array([((i % grid[0]) + (i // grid[0]) + colour) % 2 for i in range(n)])
    else:
        cp = np.zeros(n, dtype=np.int64)
    rot_index, rots = None, None
    if rotate:
        rots = square_rotations()
        rot_index = np.random.default_rng([seed, 3]).integers(len(rots), size=n)
    return build_grid_problem(name or f"heat_m{m}_{grid[0]}x{grid[1]}", pats, cp, grid, rot_index, rots,
                              load=load, seed=seed, dirichlet=dirichlet, dirichlet_fn=dirichlet_fn, k=k)


def elastic_grid(m: int, grid=(2, 2, 2), n_patterns: int = 1, seed: int = 0, k=None, rotate: bool = True,
                 dirichlet="x0", dirichlet_fn=None, load="normal", E=1.0, nu=0.3, name=None):
    """3D elasticity: cube Q1 patterns of m^3 elements; clamped x = 0; body force N(0,1) per dof;
    each occurrence takes a seeded proper rotation of the cube; cells get patterns by a seeded permutation."""
    pats = [elastic_pattern(m, E=E, nu=nu, name=f"elastic{m}_{i}") for i in range(n_patterns)]
    n = int(np.prod(grid))
    base = np.arange(n) % n_patterns
    cp = np.random.default_rng([seed, 4]).permutation(base)
    rot_index, rots = None, None
    if rotate:
        rots = cube_rotations()
        rot_index = np.random.default_rng([seed, 5]).integers(len(rots), size=n)
    return build_grid_problem(name or f"elastic_m{m}_{'x'.join(map(str, grid))}", pats, cp, grid, rot_index, rots,
                              load=load, seed=seed, dirichlet=dirichlet, dirichlet_fn=dirichlet_fn, k=k)


def config(name: str, seed: int = 0, k=None):
    """Named workloads: c1 (2D heat 8x8 pattern, 2x2 occurrences, k = 4), c2 (2D heat, 32x32 patterns with
    conductivity 1 / 1000 checkerboard over 8x8), c3 (3D elasticity, three 16^3 patterns, 4x6x8
    occurrences with rotations), c3r (reduced c3: 4^3 patterns on 2x2x2)."""
    if name == "c1":
        return heat_grid(8, (2, 2), seed=seed, k=4 if k is None else k, name="c1_heat8_2x2")
    if name == "c2":
        return heat_grid(32, (8, 8), kappas=(1.0, 1000.0), checker=True, seed=seed,
                         k=32 if k is None else k, name="c2_heat32_8x8_checker")
    if name == "c3":
        return elastic_grid(16, (4, 6, 8), n_patterns=3, seed=seed, k=32 if k is None else k,
                            name="c3_elastic16_4x6x8")
    if name == "c3r":
        return elastic_grid(4, (2, 2, 2), n_patterns=3, seed=seed, k=8 if k is None else k,
                            name="c3r_elastic4_2x2x2")
    raise ValueError(name)
