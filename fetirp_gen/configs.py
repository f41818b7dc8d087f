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
    occurrences with rotations), c4 (batched uneven 3D elasticity: 8^3/12^3/16^3/24^3 patterns, 256 occurrences
    in four clamped blocks solved together), c3r (reduced c3: 4^3 patterns on 2x2x2)."""
    if name == "c1":
        return heat_grid(8, (2, 2), seed=seed, k=4 if k is None else k, name="c1_heat8_2x2")
    if name == "c2":
        return heat_grid(32, (8, 8), kappas=(1.0, 1000.0), checker=True, seed=seed,
                         k=32 if k is None else k, name="c2_heat32_8x8_checker")
    if name == "c3":
        return elastic_grid(16, (4, 6, 8), n_patterns=3, seed=seed, k=32 if k is None else k,
                            name="c3_elastic16_4x6x8")
    if name == "c4":
        return batched_uneven(seed=seed, k_each=16 if k is None else max(1, k // 4))   # <= 64 columns in all
    if name == "c3r":
        return elastic_grid(4, (2, 2, 2), n_patterns=3, seed=seed, k=8 if k is None else k,
                            name="c3r_elastic4_2x2x2")
    raise ValueError(name)


# ------------------------------------------------------------------------------------------------ serving
LIBRARY = (("heat", 16), ("heat", 32), ("heat", 64), ("elastic", 8), ("elastic", 12), ("elastic", 16))


def library_patterns():
    """The resident library of the serving workload: three 2D heat squares (16^2, 32^2, 64^2 Q1, conductivity
    1) and three 3D elastic cubes (8^3, 12^3, 16^3 Q1, E = 1, nu = 0.3)."""
    from .mesh import elastic_pattern, heat_pattern
    return [heat_pattern(m, name=f"lib_heat{m}") if kind == "heat" else elastic_pattern(m, name=f"lib_elastic{m}")
            for kind, m in LIBRARY]


def fill_structure(pattern, n_occ: int, seed: int = 0, k=None, rotate: bool = False, name: str = ""):
    """A structure of n_occ occurrences of one pattern filling a box of side ceil(n_occ^(1/dim)) cell by cell
    in x-fastest order (connected, clamped on x = 0); loads U(0,1) per node (heat) or N(0,1) per dof."""
    dim = pattern.dim
    side = int(np.ceil(n_occ ** (1.0 / dim) - 1e-9))
    while side ** dim < n_occ:
        side += 1
    grid = (side,) * dim
    cp = np.full(side ** dim, -1, dtype=np.int64)
    cp[:n_occ] = 0
    rot_index, rots = None, None
    if rotate and dim == 3:
        rots = cube_rotations()
        rot_index = np.random.default_rng([seed, 5]).integers(len(rots), size=side ** dim)
    load = "uniform" if pattern.physics == "heat" else "normal"
    return build_grid_problem(name or f"fill_{pattern.name}_{n_occ}", [pattern], cp, grid, rot_index, rots,
                              load=load, seed=seed, dirichlet="x0", k=k)


def request_stream(n_requests: int = 1000, rate: float = 50.0, seed: int = 0, n_min: int = 4, n_max: int = 128):
    """Poisson arrivals (mean `rate` per second): (arrival time, library pattern index, occurrence count, seed)."""
    rng = np.random.default_rng([seed, 9])
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    pat = rng.integers(len(LIBRARY), size=n_requests)
    nocc = rng.integers(n_min, n_max + 1, size=n_requests)
    return [(float(t[i]), int(pat[i]), int(nocc[i]), int(seed * 100003 + i)) for i in range(n_requests)]


def merge_structures(problems, name: str = "batch"):
    """Several independent structures as one (block-diagonal dual problem): patterns, occurrences, multiplier
    rows and global nodes are renumbered one structure after the other.  Used to solve uneven batches in
    lockstep (one local-product launch covers every pattern of every structure)."""
    import copy
    from .layout import Problem
    pats, occs, c_rows, kinds, groups, coords, fno, dn, dv = [], [], [], [], [], [], [], [], []
    row0 = node0 = g0 = 0
    dim = problems[0].dim
    dpn = problems[0].dpn
    for pb in problems:
        assert pb.dim == dim and pb.dpn == dpn
        p0 = len(pats)
        pats += pb.patterns
        for o in pb.occs:
            q = copy.copy(o)
            q.pattern = o.pattern + p0
            q.node_map = o.node_map + node0
            q.link_lambda_row = o.link_lambda_row + row0
            occs.append(q)
        c_rows.append(pb.c)
        kinds.append(pb.row_kind)
        groups.append(pb.groups + g0)
        coords.append(pb.global_coords)
        fno.append(pb.f_nodal)
        dn.append(pb.dirichlet_nodes + node0)
        dv.append(pb.dirichlet_values)
        row0 += pb.n_lambda
        node0 += pb.n_global_nodes
        g0 += pb.k
    return Problem(name, dim, dpn, pats, occs, (len(occs),), problems[0].H, problems[0].m, node0,
                   np.concatenate(coords), np.concatenate(fno), np.concatenate(dn), np.concatenate(dv), row0,
                   np.concatenate(c_rows), np.concatenate(kinds), np.concatenate(groups), g0, problems[0].seed)


def batched_uneven(ms=(8, 12, 16, 24), weights=(0.4, 0.3, 0.2, 0.1), n_occ: int = 256, seed: int = 0, k_each=None):
    """Batched uneven 3D elasticity: occurrences of hex patterns of ms[i]^3 elements drawn with the given
    weights; each pattern's occurrences form their own clamped block (box filled x-fastest), the blocks are
    solved together.  Identity rotations, E = 1, nu = 0.3."""
    from .mesh import elastic_pattern
    counts = np.bincount(np.random.default_rng([seed, 8]).choice(len(ms), size=n_occ, p=weights), minlength=len(ms))
    blocks = []
    for i, (m, n) in enumerate(zip(ms, counts)):
        if n == 0:
            continue
        pat = elastic_pattern(int(m), name=f"batch_elastic{m}")
        kk = None if k_each is None else min(k_each, int(n))
        blocks.append(fill_structure(pat, int(n), seed=seed * 31 + i, k=kk))
    return merge_structures(blocks, name="batched_" + "_".join(map(str, ms)))
