"""Occurrence layouts, rigid rotations, signed Boolean links and loads (inputs of Eq. 2).

A structure is a grid of occurrences of patterns that share the same mesh density, so that neighbouring
occurrences meet node to node.  Each occurrence is a rigid rotation (a proper rotation of the square or cube,
global = R local, about the cell centre) plus a translation of its pattern.  This module states the problem
only: which global node every local node lands on, which pairs of interface dofs must agree (the rows of the
signed Boolean B, written in the global frame) and which global dofs carry Dirichlet data (total-FETI rows).

Multiplier rows (one reading of the paper's pairwise rows): at a global node owned by the occurrence set S,
one row per component for each edge of a spanning tree over the face-adjacent pairs of S, pairs taken in
(min, max) order and kept when they join two components (union-find); sign +1 on the lower occurrence index,
-1 on the higher; one Dirichlet row per component on the lowest-index occurrence owning a Dirichlet node.
Rows are ordered by global node, then tree edge, then the Dirichlet row, then component.  B has full row
rank and every gluing row couples two face-adjacent occurrences.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

from .mesh import Pattern


def cube_rotations() -> list[np.ndarray]:
    """The 24 proper rotations of the cube: signed permutation matrices with determinant +1, sorted."""
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                mats.append(R)
    mats.sort(key=lambda R: tuple(R.ravel()))
    return mats


def square_rotations() -> list[np.ndarray]:
    """The 4 rotations of the square about z, embedded as 3x3 (z unchanged)."""
    out = []
    for q in range(4):
        c, s = [1, 0, -1, 0][q], [0, 1, 0, -1][q]
        out.append(np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.int64))
    return out


@dataclass
class Occurrence:
    pattern: int
    rot: np.ndarray              # (3, 3) int, global = R @ local (components and positions)
    cell: tuple                  # grid cell of the occurrence
    node_map: np.ndarray         # (n_nodes,) int64: local node -> global node
    f_global: np.ndarray         # (n_nodes * dpn,) load, pattern node order, GLOBAL-frame components
    link_local_node: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    link_global_comp: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int8))
    link_lambda_row: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    link_sign: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int8))

    @property
    def n_links(self):
        return len(self.link_lambda_row)


@dataclass
class Problem:
    name: str
    dim: int
    dpn: int
    patterns: list
    occs: list
    grid: tuple
    H: float
    m: int
    n_global_nodes: int
    global_coords: np.ndarray
    f_nodal: np.ndarray          # (n_global_nodes * dpn,) assembled global load
    dirichlet_nodes: np.ndarray  # global node ids carrying Dirichlet data
    dirichlet_values: np.ndarray # (len(dirichlet_nodes), dpn)
    n_lambda: int
    c: np.ndarray                # (n_lambda,) right-hand side of B u = c
    row_kind: np.ndarray         # (n_lambda,) 0 = gluing, 1 = Dirichlet
    groups: np.ndarray           # (n_occ,) multivector column of each occurrence
    k: int
    seed: int = 0

    @property
    def n_occ(self):
        return len(self.occs)

    def occ_dofs(self, o):
        """Global dof ids (global frame) of occurrence o's dofs in pattern node order."""
        occ = self.occs[o]
        return (occ.node_map[:, None] * self.dpn + np.arange(self.dpn)[None, :]).ravel()


def _rcb_groups(centres: np.ndarray, k: int) -> np.ndarray:
    """Recursive coordinate bisection of occurrence centres into k groups (ids in traversal order)."""
    groups = np.zeros(len(centres), dtype=np.int32)
    counter = [0]

    def rec(idx, kk):
        if kk == 1:
            groups[idx] = counter[0]
            counter[0] += 1
            return
        pts = centres[idx]
        axis = int(np.argmax(pts.max(0) - pts.min(0)))
        order = idx[np.lexsort((idx, pts[:, axis]))]
        k1 = kk // 2
        cut = int(round(len(idx) * k1 / kk))
        rec(order[:cut], k1)
        rec(order[cut:], kk - k1)

    rec(np.arange(len(centres)), k)
    return groups


def build_grid_problem(name: str, patterns: list, cell_pattern: np.ndarray, grid: tuple,
                       rot_index=None, rotations=None, load: str = "uniform", seed: int = 0,
                       dirichlet: str = "x0", dirichlet_fn=None, k: int | None = None,
                       load_scale: float = 1.0) -> Problem:
    """Place occurrences of `patterns` on a grid of cells (x fastest) and build links, loads, groups.

    cell_pattern: pattern id per cell (len prod(grid)); rot_index: rotation id per cell (into `rotations`).
    load: "uniform" (U(0,1) per global node and component), "normal" (N(0,1) per global dof) or "zero".
    dirichlet: "x0" (global nodes on x = 0) or "all" (every node on the outer boundary).
    dirichlet_fn: coords (n, dim) -> values (n, dpn); default zero.
    """
    dim = len(grid)
    p0 = patterns[0]
    m, H, dpn = p0.m, p0.m * p0.h, p0.dpn
    for p in patterns:
        assert p.m == m and p.dim == dim and p.dpn == dpn and abs(p.m * p.h - H) < 1e-12
    h = H / m
    n_cells = int(np.prod(grid))
    cell_pattern = np.asarray(cell_pattern, dtype=np.int64)
    assert len(cell_pattern) == n_cells
    if rot_index is None:
        rot_index = np.zeros(n_cells, dtype=np.int64)
        rotations = [np.eye(3, dtype=np.int64)]
    nper = [g * m + 1 for g in grid]
    strides = [1, nper[0], nper[0] * (nper[1] if dim > 1 else 1)]
    n_gn = int(np.prod(nper))
    gidx = np.stack(np.meshgrid(*[np.arange(n) for n in nper], indexing="ij"), axis=-1).reshape(-1, dim, order="F")
    gcoords = gidx * h

    occs = []
    for cidx in range(n_cells):
        cell = []
        rem = cidx
        for d in range(dim):
            cell.append(rem % grid[d])
            rem //= grid[d]
        pat = patterns[cell_pattern[cidx]]
        R = np.asarray(rotations[rot_index[cidx]], dtype=np.int64)
        Rd = R[:dim, :dim]
        ctr = np.full(dim, H / 2)
        pos = (pat.coords - ctr) @ Rd.T + ctr + np.array(cell) * H
        gi = np.rint(pos / h).astype(np.int64)
        assert np.all(gi >= 0) and np.all(gi < np.array(nper))
        nmap = np.zeros(len(gi), dtype=np.int64)
        for d in range(dim):
            nmap += gi[:, d] * strides[d]
        occs.append(Occurrence(int(cell_pattern[cidx]), R, tuple(cell), nmap, None))

    # multiplicity of every global node
    mult = np.zeros(n_gn, dtype=np.int64)
    for o in occs:
        mult[o.node_map] += 1
    assert np.all(mult >= 1)

    rng = np.random.default_rng([seed, 1])
    if load == "uniform":
        f_nodal = rng.random(n_gn * dpn) * load_scale
    elif load == "normal":
        f_nodal = rng.standard_normal(n_gn * dpn) * load_scale
    elif load == "zero":
        f_nodal = np.zeros(n_gn * dpn)
    else:
        raise ValueError(load)
    for o in occs:
        dofs = (o.node_map[:, None] * dpn + np.arange(dpn)[None, :]).ravel()
        o.f_global = f_nodal[dofs] / np.repeat(mult[o.node_map], dpn)

    # Dirichlet nodes
    if dirichlet == "x0":
        dnodes = np.nonzero(gidx[:, 0] == 0)[0]
    elif dirichlet == "all":
        dnodes = np.nonzero(np.any((gidx == 0) | (gidx == np.array(nper) - 1), axis=1))[0]
    elif dirichlet == "none":
        dnodes = np.zeros(0, dtype=np.int64)
    else:
        raise ValueError(dirichlet)
    dvals = np.zeros((len(dnodes), dpn)) if dirichlet_fn is None else np.asarray(
        dirichlet_fn(gcoords[dnodes]), dtype=float).reshape(len(dnodes), dpn)
    dmap = {int(g): i for i, g in enumerate(dnodes)}

    # owners of every global node that sits on some occurrence's boundary
    gs, os_, ls = [], [], []
    for oi, o in enumerate(occs):
        b = patterns[o.pattern].bnd_nodes
        gs.append(o.node_map[b])
        os_.append(np.full(len(b), oi, dtype=np.int64))
        ls.append(b.astype(np.int64))
    gs, os_, ls = np.concatenate(gs), np.concatenate(os_), np.concatenate(ls)
    order = np.lexsort((os_, gs))
    gs, os_, ls = gs[order], os_[order], ls[order]
    ug, start, cnt = np.unique(gs, return_index=True, return_counts=True)
    cells = np.array([o.cell for o in occs])

    link_o, link_l, link_c, link_r, link_s = [], [], [], [], []
    c_rows, kinds = [], []
    row = 0
    for g, st, ct in zip(ug, start, cnt):
        g = int(g)
        S = os_[st:st + ct]
        L = ls[st:st + ct]
        if ct >= 2:
            parent = list(range(ct))

            def find(x):
                while parent[x] != x:
                    parent[x] = parent[parent[x]]
                    x = parent[x]
                return x
            for a in range(ct):
                for b in range(a + 1, ct):
                    if np.abs(cells[S[a]] - cells[S[b]]).sum() != 1:
                        continue
                    ra, rb = find(a), find(b)
                    if ra == rb:
                        continue
                    parent[rb] = ra
                    for comp in range(dpn):
                        link_o += [S[a], S[b]]
                        link_l += [L[a], L[b]]
                        link_c += [comp, comp]
                        link_r += [row, row]
                        link_s += [1, -1]
                        c_rows.append(0.0)
                        kinds.append(0)
                        row += 1
        if g in dmap:
            for comp in range(dpn):
                link_o.append(S[0]); link_l.append(L[0]); link_c.append(comp)
                link_r.append(row); link_s.append(1)
                c_rows.append(dvals[dmap[g], comp])
                kinds.append(1)
                row += 1
    # Dirichlet nodes that are on no occurrence boundary cannot occur on a grid (x = 0 is a surface).
    link_o = np.array(link_o, dtype=np.int64)
    link_l = np.array(link_l, dtype=np.int32)
    link_c = np.array(link_c, dtype=np.int8)
    link_r = np.array(link_r, dtype=np.int32)
    link_s = np.array(link_s, dtype=np.int8)
    for oi, o in enumerate(occs):
        sel = link_o == oi
        o.link_local_node = link_l[sel]
        o.link_global_comp = link_c[sel]
        o.link_lambda_row = link_r[sel]
        o.link_sign = link_s[sel]

    centres = cells + 0.5
    if k is None:
        k = min(n_cells, 32)
    k = min(k, n_cells)
    groups = _rcb_groups(centres.astype(float), k)
    return Problem(name, dim, dpn, patterns, occs, tuple(grid), H, m, n_gn, gcoords, f_nodal,
                   dnodes, dvals, row, np.array(c_rows), np.array(kinds, dtype=np.int8), groups, k, seed)


def dense_B(prob: Problem) -> list:
    """Per occurrence, B(s) as a dense (n_lambda, n_dofs) array in the GLOBAL frame (tiny problems only)."""
    out = []
    for o in prob.occs:
        nd = prob.patterns[o.pattern].n_dofs
        B = np.zeros((prob.n_lambda, nd))
        for ln, gc, r, s in zip(o.link_local_node, o.link_global_comp, o.link_lambda_row, o.link_sign):
            B[r, ln * prob.dpn + gc] += s
        out.append(B)
    return out


def set_nodal_load(prob: Problem, f_nodal: np.ndarray) -> Problem:
    """Replace the load by a given assembled nodal load, split over the owners of every node."""
    f_nodal = np.asarray(f_nodal, dtype=float)
    mult = np.zeros(prob.n_global_nodes, dtype=np.int64)
    for o in prob.occs:
        mult[o.node_map] += 1
    for o in prob.occs:
        dofs = (o.node_map[:, None] * prob.dpn + np.arange(prob.dpn)[None, :]).ravel()
        o.f_global = f_nodal[dofs] / np.repeat(mult[o.node_map], prob.dpn)
    prob.f_nodal = f_nodal.copy()
    return prob
