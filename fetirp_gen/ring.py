"""A truly periodic structure for the permutation multivector (Section 3.1, Eq. 8): n identical annulus sectors
(2D heat, isoparametric Q1 on a polar grid) arranged in a ring, every occurrence the pattern rotated by
2 pi k / n.  Dirichlet rows sit on every sector's inner arc (and optionally its outer arc), so the dual
operator is periodic; the loads are random and non-periodic, as in the paper's donut tests.

Multiplier rows: one gluing row per node of each radial interface line (the line at angle (k + 1) theta is
shared by sectors k and k + 1; +1 on the lower occurrence index, as everywhere in this generator), and one
Dirichlet row per constrained node.  A constrained node at the end of a radial line carries its Dirichlet row
on the sector for which that line is the side at angle theta (sector k for the line between k and k + 1), a rule
that is invariant under the rotation of the ring.

`ring_permutation` returns the map of multiplier rows under the rotation by one sector, with the sign that
makes it commute with the dual operator (the wrap-around line has its +1 on the other side).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .layout import Occurrence, Problem
from .mesh import GAUSS2, Pattern, _shape_grads


def q1_laplace_quad(xy: np.ndarray, kappa: float = 1.0) -> np.ndarray:
    """Conductivity matrix kappa * int grad N_a . grad N_b of one isoparametric bilinear quadrilateral with
    corners xy[a] (a = i + 2 j, the reference corner (2i - 1, 2j - 1)), 2 x 2 Gauss."""
    K = np.zeros((4, 4))
    for xi in itertools.product(GAUSS2, repeat=2):
        dNdxi = _shape_grads(np.array(xi), 2)          # (4, 2)
        J = xy.T @ dNdxi                                # J[d, e] = d x_d / d xi_e
        dNdx = dNdxi @ np.linalg.inv(J)
        K += kappa * (dNdx @ dNdx.T) * abs(np.linalg.det(J))   # the area element (orientation-free)
    return K


def plane_strain_D(E: float, nu: float) -> np.ndarray:
    """Isotropic plane-strain constitutive matrix, Voigt order (xx, yy, xy), engineering shear strain."""
    c = E / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return c * np.array([[1.0 - nu, nu, 0.0], [nu, 1.0 - nu, 0.0], [0.0, 0.0, 0.5 - nu]])


def q1_plane_strain_quad(xy: np.ndarray, E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """Stiffness int eps(N_a)^T D eps(N_b) (unit thickness) of one isoparametric bilinear quadrilateral, dof =
    corner * 2 + component, 2 x 2 Gauss."""
    D = plane_strain_D(E, nu)
    K = np.zeros((8, 8))
    for xi in itertools.product(GAUSS2, repeat=2):
        dNdxi = _shape_grads(np.array(xi), 2)
        J = xy.T @ dNdxi
        dNdx = dNdxi @ np.linalg.inv(J)
        Bm = np.zeros((3, 8))
        Bm[0, 0::2] = dNdx[:, 0]
        Bm[1, 1::2] = dNdx[:, 1]
        Bm[2, 0::2] = dNdx[:, 1]
        Bm[2, 1::2] = dNdx[:, 0]
        K += Bm.T @ D @ Bm * abs(np.linalg.det(J))
    return K


def sector_pattern(n_sectors: int, m_t: int, m_r: int, r_in: float = 1.0, r_out: float = 2.0,
                   kappa: float = 1.0, physics: str = "heat", E: float = 1.0, nu: float = 0.3) -> Pattern:
    """The annulus sector 0 <= phi <= 2 pi / n_sectors, r_in <= r <= r_out, m_t x m_r polar Q1 elements;
    node = i + (m_t + 1) j with phi_i = i theta / m_t and r_j = r_in + j (r_out - r_in) / m_r.  physics "heat"
    (conductivity kappa, one dof per node) or "elastic" (plane strain, E, nu, two dofs per node)."""
    theta = 2.0 * np.pi / n_sectors
    phi = np.arange(m_t + 1) * theta / m_t
    rad = r_in + np.arange(m_r + 1) * (r_out - r_in) / m_r
    P, R = np.meshgrid(phi, rad, indexing="xy")        # rows j (radius), columns i (angle)
    coords = np.stack([(R * np.cos(P)).ravel(), (R * np.sin(P)).ravel()], axis=1)
    n1 = m_t + 1
    rows, cols, vals = [], [], []
    dpn = 1 if physics == "heat" else 2
    for j in range(m_r):
        for i in range(m_t):
            nodes = np.array([i + n1 * j, i + 1 + n1 * j, i + n1 * (j + 1), i + 1 + n1 * (j + 1)])
            if dpn == 1:
                Ke = q1_laplace_quad(coords[nodes], kappa)
                dofs = nodes
            else:
                Ke = q1_plane_strain_quad(coords[nodes], E, nu)
                dofs = (nodes[:, None] * 2 + np.arange(2)[None, :]).ravel()
            rows.append(np.repeat(dofs, len(dofs))); cols.append(np.tile(dofs, len(dofs))); vals.append(Ke.ravel())
    n = coords.shape[0]
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n * dpn, n * dpn)).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    ii, jj = np.arange(n) % n1, np.arange(n) // n1
    bnd = np.nonzero((ii == 0) | (ii == m_t) | (jj == 0) | (jj == m_r))[0].astype(np.int32)
    material = {"kappa": kappa} if dpn == 1 else {"E": E, "nu": nu}
    pat = Pattern(f"sector{n_sectors}_{physics}_{m_t}x{m_r}", 2, m_t, theta / m_t, dpn, physics, material, coords,
                  K, bnd, 1 if dpn == 1 else 3)
    pat.ring = {"n_sectors": n_sectors, "m_t": m_t, "m_r": m_r, "r_in": r_in, "r_out": r_out}
    return pat


def _rot(angle):
    c, s = np.cos(angle), np.sin(angle)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def ring_structure(n_sectors: int = 5, m_t: int = 4, m_r: int = 4, r_in: float = 1.0, r_out: float = 2.0,
                   physics: str = "heat", kappa: float = 1.0, E: float = 1.0, nu: float = 0.3, seed: int = 0,
                   dirichlet: str = "inner", dirichlet_fn=None, load: str = "random") -> Problem:
    """The ring of n_sectors rotated copies of sector_pattern.  dirichlet: "inner" (inner arcs) or "both"
    (inner and outer arcs); dirichlet_fn: coords (n, 2) -> values (n, dpn), default 0; load: "random" (heat
    U(0,1) per global node, elasticity N(0,1) per global dof, split over the owners) or "zero".  Multiplier rows
    follow the order (global node, gluing before Dirichlet, component); vector components are global-frame."""
    if n_sectors < 3:
        raise ValueError("a ring needs at least 3 sectors")
    pat = sector_pattern(n_sectors, m_t, m_r, r_in, r_out, kappa, physics, E, nu)
    dpn = pat.dpn
    theta = 2.0 * np.pi / n_sectors
    n1 = m_t + 1
    # global nodes: positions of every occurrence's nodes, merged where they coincide
    pos = np.concatenate([pat.coords @ _rot(k * theta)[:2, :2].T for k in range(n_sectors)])
    key = np.round(pos / (1e-9 * r_out)).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.ravel()
    n_gn = len(first)
    gcoords = pos[first]
    nmaps = [inv[k * pat.n_nodes:(k + 1) * pat.n_nodes].astype(np.int64) for k in range(n_sectors)]
    mult = np.bincount(np.concatenate(nmaps), minlength=n_gn)

    rng = np.random.default_rng([seed, 1])
    if load == "zero":
        f_nodal = np.zeros(n_gn * dpn)
    elif dpn == 1:
        f_nodal = rng.random(n_gn)
    else:
        f_nodal = rng.standard_normal(n_gn * dpn)
    occs = []
    for k in range(n_sectors):
        dofs = (nmaps[k][:, None] * dpn + np.arange(dpn)[None, :]).ravel()
        occs.append(Occurrence(0, _rot(k * theta), (k,), nmaps[k], f_nodal[dofs] / np.repeat(mult[nmaps[k]], dpn)))

    # local node sets of the sector
    ii, jj = np.arange(pat.n_nodes) % n1, np.arange(pat.n_nodes) // n1
    side0 = np.nonzero(ii == 0)[0]          # radial side at phi = 0 (ordered by radius)
    side1 = np.nonzero(ii == m_t)[0]        # radial side at phi = theta (ordered by radius)
    inner = np.nonzero(jj == 0)[0]
    outer = np.nonzero(jj == m_r)[0]
    dset = inner if dirichlet == "inner" else np.concatenate([inner, outer])
    # row items: (global node, kind 0 gluing / 1 Dirichlet, [(occurrence, local node, sign)])
    items = []
    for k in range(n_sectors):
        kn = (k + 1) % n_sectors
        for a, b in zip(side1, side0):      # line between sectors k (its phi = theta side) and k + 1
            g = int(nmaps[k][a])
            assert g == int(nmaps[kn][b])
            lo, hi = (k, a), (kn, b)
            if kn < k:
                lo, hi = hi, lo
            items.append((g, 0, [(lo[0], lo[1], 1), (hi[0], hi[1], -1)]))
    owner_done = set()
    for k in range(n_sectors):
        for a in dset:
            g = int(nmaps[k][a])
            if g in owner_done:
                continue
            # a node on the phi = 0 side belongs to the previous sector's phi = theta side
            if ii[a] == 0:
                kp = (k - 1) % n_sectors
                owner = (kp, int(side1[np.nonzero(side0 == a)[0][0]]))
            else:
                owner = (k, int(a))
            owner_done.add(g)
            items.append((g, 1, [(owner[0], owner[1], 1)]))
    items.sort(key=lambda t: (t[0], t[1]))
    n_lambda = len(items) * dpn
    link = [[] for _ in range(n_sectors)]
    row_kind = np.repeat(np.array([kind for _, kind, _ in items], dtype=np.int8), dpn)
    c = np.zeros(n_lambda)
    for it, (g, kind, ents) in enumerate(items):
        if kind == 1 and dirichlet_fn is not None:
            c[it * dpn:(it + 1) * dpn] = np.asarray(dirichlet_fn(gcoords[g][None, :]), dtype=float).reshape(-1)[:dpn]
        for comp in range(dpn):
            for (o, ln, sg) in ents:
                link[o].append((it * dpn + comp, ln, comp, sg))
    for o, occ in enumerate(occs):
        L = sorted(link[o])
        occ.link_lambda_row = np.array([t[0] for t in L], dtype=np.int32)
        occ.link_local_node = np.array([t[1] for t in L], dtype=np.int32)
        occ.link_global_comp = np.array([t[2] for t in L], dtype=np.int8)
        occ.link_sign = np.array([t[3] for t in L], dtype=np.int8)
    dnodes = np.array(sorted({g for g, kind, _ in items if kind == 1}), dtype=np.int64)
    dvals = (np.zeros((len(dnodes), dpn)) if dirichlet_fn is None else
             np.asarray(dirichlet_fn(gcoords[dnodes]), dtype=float).reshape(len(dnodes), dpn))
    prob = Problem(f"ring{n_sectors}_{physics}_{m_t}x{m_r}", 2, dpn, [pat], occs, (n_sectors,), r_out, m_t, n_gn,
                   gcoords, f_nodal, dnodes, dvals, n_lambda, c, row_kind, np.arange(n_sectors, dtype=np.int32),
                   n_sectors, seed)
    prob.ring_items = items
    return prob


def ring_heat(n_sectors: int = 5, m_t: int = 4, m_r: int = 4, r_in: float = 1.0, r_out: float = 2.0,
              kappa: float = 1.0, seed: int = 0, dirichlet: str = "inner", dirichlet_fn=None,
              load: str = "uniform") -> Problem:
    """ring_structure for 2D heat (U(0,1) loads per node unless load = "zero")."""
    return ring_structure(n_sectors, m_t, m_r, r_in, r_out, "heat", kappa=kappa, seed=seed, dirichlet=dirichlet,
                          dirichlet_fn=dirichlet_fn, load="zero" if load == "zero" else "random")


def ring_elastic(n_sectors: int = 5, m_t: int = 4, m_r: int = 4, r_in: float = 1.0, r_out: float = 2.0,
                 E: float = 1.0, nu: float = 0.3, seed: int = 0, dirichlet: str = "inner", dirichlet_fn=None,
                 load: str = "random") -> Problem:
    """ring_structure for plane-strain elasticity (N(0,1) loads per dof unless load = "zero")."""
    return ring_structure(n_sectors, m_t, m_r, r_in, r_out, "elastic", E=E, nu=nu, seed=seed, dirichlet=dirichlet,
                          dirichlet_fn=dirichlet_fn, load=load)


def ring_permutation(prob: Problem) -> sp.csr_matrix:
    """The map of multiplier vectors under the rotation of the ring by one sector, as a sparse n_lambda x
    n_lambda matrix Pi: the value of node item r moves to the item of the rotated node (same kind), its
    global-frame components rotated with the structure, with the orientation sign of the wrap-around line (whose
    +1 sits on sector 0 rather than on the sector for which the line is the side at angle theta)."""
    n = len(prob.occs)
    dpn = prob.dpn
    theta = 2.0 * np.pi / n
    items = prob.ring_items
    R = _rot(theta)[:2, :2]
    Rc = np.ones((1, 1)) if dpn == 1 else R
    scale = 1e-9 * prob.H
    key_of = {}
    for r, (g, kind, ents) in enumerate(items):
        key_of[(tuple(np.round(prob.global_coords[g] / scale).astype(np.int64)), kind)] = r

    def orientation(ents):
        if len(ents) == 1:
            return 1
        (o1, _, s1), (o2, _, s2) = ents
        first = o1 if s1 == 1 else o2          # sector carrying +1
        other = o2 if s1 == 1 else o1
        return 1 if (first + 1) % n == other else -1

    rows, cols, vals = [], [], []
    for r, (g, kind, ents) in enumerate(items):
        p = R @ prob.global_coords[g]
        t = key_of[(tuple(np.round(p / scale).astype(np.int64)), kind)]
        sg = orientation(ents) * orientation(items[t][2])
        for a in range(dpn):
            for b in range(dpn):
                if Rc[a, b] != 0.0:
                    rows.append(t * dpn + a); cols.append(r * dpn + b); vals.append(sg * Rc[a, b])
    m = len(items) * dpn
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))
