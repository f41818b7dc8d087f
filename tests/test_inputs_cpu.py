"""The seeded synthetic workloads follow their stated recipe: sizes, non-redundant multiplier rows with their
sign rule, Dirichlet rows on x = 0, proper cube rotations, the load distributions and their split at shared
nodes, the conductivity checkerboard, the multivector groups, the Poisson request stream and the uneven batch."""
import numpy as np
import pytest

from fetirp_gen import LIBRARY, batched_uneven, config, elastic_grid, request_stream
from fetirp_gen.layout import cube_rotations


def _links(prob):
    """Per link: (row, occurrence, global dof, sign)."""
    rows, occ, gdof, sign = [], [], [], []
    for o, oc in enumerate(prob.occs):
        rows.append(oc.link_lambda_row)
        occ.append(np.full(oc.n_links, o))
        gdof.append(oc.node_map[oc.link_local_node] * prob.dpn + oc.link_global_comp)
        sign.append(oc.link_sign)
    return tuple(np.concatenate(a).astype(np.int64) for a in (rows, occ, gdof, sign))


@pytest.fixture(scope="module")
def c2():
    return config("c2")


@pytest.fixture(scope="module")
def rotated():
    return elastic_grid(3, (3, 2, 2), n_patterns=2, k=4, seed=3)


def test_sizes():
    c1 = config("c1")
    assert (c1.n_lambda, c1.n_occ, c1.k, c1.dpn) == (52, 4, 4, 1)
    c2 = config("c2")
    assert (c2.n_lambda, c2.n_occ, c2.grid, c2.dpn, len(c2.patterns)) == (3904, 64, (8, 8), 1, 2)
    assert all(p.m == 32 for p in c2.patterns) and c2.n_global_nodes == 257 * 257


@pytest.mark.parametrize("which", ["c2", "rotated"])
def test_multiplier_rows(which, c2, rotated):
    """Every row has one link (Dirichlet) or two (gluing) on the same global dof; gluing rows carry +1 on the
    lower occurrence index and -1 on the higher; the row kinds and c agree."""
    prob = c2 if which == "c2" else rotated
    rows, occ, gdof, sign = _links(prob)
    cnt = np.bincount(rows, minlength=prob.n_lambda)
    assert cnt.min() >= 1 and cnt.max() <= 2
    assert np.array_equal(cnt == 1, prob.row_kind == 1)
    order = np.lexsort((occ, rows))
    rows, occ, gdof, sign = rows[order], occ[order], gdof[order], sign[order]
    first = np.r_[0, np.cumsum(cnt)[:-1]]
    two = cnt == 2
    a, b = first[two], first[two] + 1
    assert np.array_equal(gdof[a], gdof[b])
    assert np.all(occ[a] < occ[b]) and np.all(sign[a] == 1) and np.all(sign[b] == -1)
    one = first[cnt == 1]
    assert np.all(sign[one] == 1)
    # Dirichlet rows sit on nodes at x = 0 and carry c = 0 (zero Dirichlet data)
    dnode = gdof[one] // prob.dpn
    assert np.allclose(prob.global_coords[dnode, 0], 0.0)
    assert np.all(prob.c == 0.0)
    # non-redundant: at most one gluing row per (global dof, occurrence pair)
    pairs = set(zip(gdof[a].tolist(), occ[a].tolist(), occ[b].tolist()))
    assert len(pairs) == int(two.sum())


def test_gluing_pairs_are_face_neighbours(rotated):
    rows, occ, gdof, sign = _links(rotated)
    cells = np.array([o.cell for o in rotated.occs])
    order = np.lexsort((occ, rows))
    rows, occ = rows[order], occ[order]
    cnt = np.bincount(rows, minlength=rotated.n_lambda)
    first = np.r_[0, np.cumsum(cnt)[:-1]][cnt == 2]
    d = np.abs(cells[occ[first]] - cells[occ[first + 1]]).sum(axis=1)
    assert np.all(d == 1)


def test_rotations_are_proper_cube_rotations(rotated):
    rots = cube_rotations()
    assert len(rots) == 24 and len({r.tobytes() for r in rots}) == 24
    for r in rots:
        assert np.array_equal(r @ r.T, np.eye(3, dtype=r.dtype)) and round(np.linalg.det(r)) == 1
    assert any(not np.array_equal(o.rot, np.eye(3)) for o in rotated.occs)
    for o in rotated.occs:
        assert any(np.array_equal(o.rot, r) for r in rots)


@pytest.mark.parametrize("which", ["c2", "rotated"])
def test_loads_split_at_shared_nodes(which, c2, rotated):
    """Each occurrence carries f_global / multiplicity on its nodes, so the occurrence loads add up exactly
    to the assembled global load."""
    prob = c2 if which == "c2" else rotated
    acc = np.zeros_like(prob.f_nodal)
    for o in range(prob.n_occ):
        np.add.at(acc, prob.occ_dofs(o), prob.occs[o].f_global)
    assert np.allclose(acc, prob.f_nodal, rtol=1e-14, atol=1e-15)


def test_load_distributions(c2, rotated):
    f = c2.f_nodal
    assert f.min() >= 0.0 and f.max() < 1.0 and abs(f.mean() - 0.5) < 0.01
    g = rotated.f_nodal
    assert abs(g.mean()) < 0.1 and abs(g.std() - 1.0) < 0.1


def test_c2_checkerboard_and_groups(c2):
    pat = {o.cell: o.pattern for o in c2.occs}
    for (i, j), p in pat.items():
        for di, dj in ((1, 0), (0, 1)):
            q = pat.get((i + di, j + dj))
            if q is not None:
                assert q != p
    kap = [float(p.material["kappa"]) for p in c2.patterns]
    assert sorted(kap) == [1.0, 1000.0]
    lo, hi = (c2.patterns[0], c2.patterns[1]) if kap[0] < kap[1] else (c2.patterns[1], c2.patterns[0])
    assert abs(hi.K - 1000.0 * lo.K).max() <= 1e-12 * abs(hi.K).max()   # same mesh, conductivity 1000
    assert c2.k == 32 and np.array_equal(np.unique(c2.groups), np.arange(32))
    assert np.bincount(c2.groups).min() >= 1


def test_request_stream():
    req = request_stream(1000, rate=50.0, seed=0)
    t = np.array([r[0] for r in req])
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(np.r_[0.0, t]).mean() - 1 / 50.0) < 0.1 / 50.0
    pats = np.array([r[1] for r in req])
    nocc = np.array([r[2] for r in req])
    assert pats.min() >= 0 and pats.max() < len(LIBRARY) and len(np.unique(pats)) == len(LIBRARY)
    assert nocc.min() >= 4 and nocc.max() <= 128
    assert request_stream(10, seed=1) == request_stream(10, seed=1)


def test_uneven_batch_recipe():
    """Four cube patterns of 8, 12, 16, 24 elements per side, 256 occurrences drawn with weights
    0.4 / 0.3 / 0.2 / 0.1, each pattern's occurrences in their own block (block-diagonal dual problem)."""
    prob = batched_uneven(ms=(2, 3, 4, 5), n_occ=256, seed=0)   # the recipe on smaller meshes (fast)
    ms = [p.m for p in prob.patterns]
    assert ms == [2, 3, 4, 5]
    counts = np.bincount([o.pattern for o in prob.occs], minlength=4)
    assert counts.sum() == 256
    assert np.all(np.abs(counts / 256 - np.array([0.4, 0.3, 0.2, 0.1])) < 0.08)
    rows, occ, gdof, sign = _links(prob)
    pat_of = np.array([o.pattern for o in prob.occs])
    by_row = {}
    for r, o in zip(rows.tolist(), occ.tolist()):
        by_row.setdefault(r, set()).add(int(pat_of[o]))
    assert all(len(v) == 1 for v in by_row.values())   # no row couples two blocks
