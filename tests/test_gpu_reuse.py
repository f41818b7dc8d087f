"""GPU: a context solves again after a refactorisation (the structure tables are kept, d, the coarse problem and G's
values are rebuilt from the new factors) and after a change of structure (every table rebuilt), each time against
the oracle's direct solve."""
import numpy as np
import pytest

from fetirp_gen import heat_grid, elastic_grid
from oracle.direct import direct

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def check(prob, lam, u):
    us_ref, lam_ref, _, _ = direct(prob)
    assert rel(lam, lam_ref) < 1e-8
    for a, b in zip(F.split_u(prob, u), us_ref):
        assert rel(a, b) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_refactorise_and_solve_again(prec):
    """n_b = 1158: the tensor-core S^dag and the factored FP64 products are formed anew by every factorisation."""
    prob = elastic_grid(8, (2, 2, 1), n_patterns=2, k=4, seed=3)
    ctx = F.fetirp_create(F.fetirp_default_options(precision=prec, tol=1e-10))
    try:
        F.load_problem(ctx, prob)
        lam1, u1, st1 = F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob))
        F.fetirp_factorize(ctx)
        lam2, u2, st2 = F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob))
    finally:
        F.fetirp_destroy(ctx)
    check(prob, lam1, u1)
    check(prob, lam2, u2)
    assert st2["iterations"] == st1["iterations"]
    assert rel(lam2, lam1) < 1e-12 and rel(u2, u1) < 1e-12


def test_structure_change_rebuilds_tables():
    """The same two patterns, first on a 3 x 2 grid, then (occurrences cleared and added again) on a 2 x 3 grid
    with other loads: the second solve must see the new links, groups and loads."""
    a = heat_grid(5, (3, 2), kappas=(1.0, 30.0), checker=True, k=3, seed=7)
    b = heat_grid(5, (2, 3), kappas=(1.0, 30.0), checker=True, k=2, seed=8)
    for pa, pb in zip(a.patterns, b.patterns):
        assert (pa.K != pb.K).nnz == 0 and np.array_equal(pa.bnd_nodes, pb.bnd_nodes)
    ctx = F.fetirp_create(F.fetirp_default_options(precision="fp32", tol=1e-10))
    try:
        F.load_problem(ctx, a)
        lam_a, u_a, _ = F.fetirp_solve(ctx, a.n_lambda, a.c, F.n_u(a))
        check(a, lam_a, u_a)
        F.fetirp_clear_occurrences(ctx)
        for occ in b.occs:
            F.fetirp_add_occurrence(ctx, occ.pattern, occ.rot.astype(float), occ.link_local_node,
                                    occ.link_global_comp, occ.link_lambda_row, occ.link_sign, occ.f_global)
        F.fetirp_set_groups(ctx, b.k, b.groups)
        lam_b, u_b, _ = F.fetirp_solve(ctx, b.n_lambda, b.c, F.n_u(b))
        check(b, lam_b, u_b)
    finally:
        F.fetirp_destroy(ctx)
