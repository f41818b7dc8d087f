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
        if cell_pattern[cidx] < 0:        # empty cell (partially filled box)
            continue
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

    # multiplicity of every global node (0 for nodes of empty cells only)
    mult = np.zeros(n_gn, dtype=np.int64)
    for o in occs:
        mult[o.node_map] += 1
    assert np.all(mult[np.concatenate([o.node_map for o in occs])] >= 1)

    rng = np.random.default_rng([seed, 1])
    if load == "uniform":
        f_nodal = rng.random(n_gn * dpn) * load_scale
    elif load == "normal":
        f_nodal = rng.standard_normal(n_gn * dpn) * load_scale
    elif load == "zero":
        f_nodal = np.zeros(n_gn * dpn)
    else:
        raise ValueError(load)
    f_nodal[np.repeat(mult == 0, dpn)] = 0.0
    for o in occs:
        dofs = (o.node_map[:, None] * dpn + np.arange(dpn)[None, :]).ravel()
        o.f_global = f_nodal[dofs] / np.repeat(mult[o.node_map], dpn)

    # Dirichlet nodes (only nodes some occurrence owns)
    if dirichlet == "x0":
        dnodes = np.nonzero((gidx[:, 0] == 0) & (mult > 0))[0]
    elif dirichlet == "all":
        dnodes = np.nonzero(np.any((gidx == 0) | (gidx == np.array(nper) - 1), axis=1) & (mult > 0))[0]
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

    # Multiplier rows, in the order (global node, tree edge, Dirichlet row, component).  Nodes owned by two
    # occurrences carry exactly one tree edge (vectorised); nodes with more owners take the union-find loop.
    # Per node: its list of "row items" (a, b, la, lb) with b = -1 for a Dirichlet item, laid out in order.
    is_dir = np.zeros(n_gn, dtype=bool)
    is_dir[dnodes] = True
    item_node, item_a, item_b, item_la, item_lb, item_rank = [], [], [], [], [], []
    two = cnt == 2
    if np.any(two):
        st2 = start[two]
        item_node.append(ug[two]); item_a.append(os_[st2]); item_b.append(os_[st2 + 1])
        item_la.append(ls[st2]); item_lb.append(ls[st2 + 1]); item_rank.append(np.zeros(int(two.sum()), np.int64))
    multi = np.nonzero(cnt > 2)[0]
    ma, mb, mla, mlb, mn, mr = [], [], [], [], [], []
    for t in multi:
        g, st, ct = int(ug[t]), int(start[t]), int(cnt[t])
        S = os_[st:st + ct]
        Lc = ls[st:st + ct]
        parent = list(range(ct))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        rank = 0
        for a in range(ct):
            for b in range(a + 1, ct):
                if np.abs(cells[S[a]] - cells[S[b]]).sum() != 1:
                    continue
                ra, rb = find(a), find(b)
                if ra == rb:
                    continue
                parent[rb] = ra
                mn.append(g); ma.append(S[a]); mb.append(S[b]); mla.append(Lc[a]); mlb.append(Lc[b]); mr.append(rank)
                rank += 1
    if mn:
        item_node.append(np.array(mn)); item_a.append(np.array(ma)); item_b.append(np.array(mb))
        item_la.append(np.array(mla)); item_lb.append(np.array(mlb)); item_rank.append(np.array(mr))
    # Dirichlet items: lowest-index owner of a Dirichlet node, ranked after the node's tree edges
    dmask = is_dir[ug]
    if np.any(dmask):
        std = start[dmask]
        item_node.append(ug[dmask]); item_a.append(os_[std]); item_b.append(np.full(int(dmask.sum()), -1))
        item_la.append(ls[std]); item_lb.append(np.full(int(dmask.sum()), -1))
        item_rank.append(np.full(int(dmask.sum()), 1 << 30))
    item_node = np.concatenate(item_node) if item_node else np.zeros(0, np.int64)
    item_a = np.concatenate(item_a) if item_a else np.zeros(0, np.int64)
    item_b = np.concatenate(item_b) if item_b else np.zeros(0, np.int64)
    item_la = np.concatenate(item_la) if item_la else np.zeros(0, np.int64)
    item_lb = np.concatenate(item_lb) if item_lb else np.zeros(0, np.int64)
    item_rank = np.concatenate(item_rank) if item_rank else np.zeros(0, np.int64)
    order = np.lexsort((item_rank, item_node))
    item_node, item_a, item_b = item_node[order], item_a[order], item_b[order]
    item_la, item_lb, item_rank = item_la[order], item_lb[order], item_rank[order]
    n_items = len(item_node)
    rows = (np.arange(n_items)[:, None] * dpn + np.arange(dpn)[None, :])          # row of (item, comp)
    comp = np.broadcast_to(np.arange(dpn)[None, :], rows.shape)
    glue = item_b >= 0
    # gluing rows: +1 on a, -1 on b; Dirichlet rows: +1 on a
    link_o = np.concatenate([np.repeat(item_a, dpn), np.repeat(item_b[glue], dpn)])
    link_l = np.concatenate([np.repeat(item_la, dpn), np.repeat(item_lb[glue], dpn)]).astype(np.int32)
    link_c = np.concatenate([comp.ravel(), comp[glue].ravel()]).astype(np.int8)
    link_r = np.concatenate([rows.ravel(), rows[glue].ravel()]).astype(np.int32)
    link_s = np.concatenate([np.ones(n_items * dpn), -np.ones(int(glue.sum()) * dpn)]).astype(np.int8)
    row = n_items * dpn
    c_rows = np.zeros(row)
    kinds = np.repeat((~glue).astype(np.int8), dpn)
    if np.any(~glue):
        dvals_full = np.zeros((n_gn, dpn))
        dvals_full[dnodes] = dvals
        dr = rows[~glue]
        c_rows[dr.ravel()] = dvals_full[item_node[~glue]].ravel()
    # (Dirichlet nodes lie on x = 0, a boundary surface of every occurrence that owns them.)
    by_row = np.argsort(link_r, kind="stable")     # every occurrence's links in increasing row order
    link_o, link_l, link_c, link_r, link_s = link_o[by_row], link_l[by_row], link_c[by_row], link_r[by_row], link_s[by_row]
    for oi, o in enumerate(occs):
        sel = link_o == oi
        o.link_local_node = link_l[sel]
        o.link_global_comp = link_c[sel]
        o.link_lambda_row = link_r[sel]
        o.link_sign = link_s[sel]

    centres = cells + 0.5
    n_occ = len(occs)
    if k is None:
        k = min(n_occ, 32)
    k = min(k, n_occ)
    groups = _rcb_groups(centres.astype(float), k)
    return Problem(name, dim, dpn, patterns, occs, tuple(grid), H, m, n_gn, gcoords, f_nodal,
                   dnodes, dvals, row, c_rows, kinds, groups, k, seed)


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
