"""Full-size elastic workload (three 16^3 Q1 cube patterns, 4 x 6 x 8 rotated occurrences, n_lambda = 427,392),
in the launch configuration of the mixed tensor-core form.  The oracle cannot solve this size in seconds, so:
  - the block operator P^T F P V is compared element by element with the oracle's on sampled columns;
  - the solve is checked against the defining equations at full size: subdomain equilibrium
    K(s) u(s) = f(s) - B(s)^T lambda for every occurrence (Eq. 2), interface continuity B u = c, and the
    coarse condition G^T lambda = e (Eq. 3), each to a relative residual of 1e-7 or better."""
import numpy as np
import pytest

from fetirp_gen import config
from oracle.direct import B_matrix, occurrence_stiffness
from oracle.feti import FetiOracle

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")


@pytest.fixture(scope="module")
def c3():
    return config("c3")


def test_c3_operator_matches_oracle_on_sampled_columns(c3):
    """The block operator on a full k = 32 block (R_p = 2048 right-hand sides per pattern: sixteen 128-column
    tiles of the tensor-core product, 37 row tiles), compared element by element with the oracle on three of
    its columns (column g of P^T F P V depends on column g of V only)."""
    orc = FetiOracle(c3, use_schur=False)   # full local solves with the oracle's own generalized inverse
    cols = [0, 17, 31]
    ctx = F.fetirp_create(F.fetirp_default_options())
    try:
        F.load_problem(ctx, c3)
        F.fetirp_prepare(ctx, c3.n_lambda, c3.c)
        V = np.random.default_rng(21).standard_normal((c3.n_lambda, 32))
        Qo = orc.PtFP(V[:, cols])
        for prec, tol in (("fp64", 1e-9), ("fp32", 5e-4), ("tf32x3", 5e-4), ("bf16x3", 1e-3)):
            Q = F.fetirp_apply_block(ctx, V, F.PRECISIONS[prec])[:, cols]
            rel = np.linalg.norm(Q - Qo) / np.linalg.norm(Qo)
            assert rel < tol, (prec, rel)
            assert np.abs(Q - Qo).max() < 10 * tol * np.abs(Qo).max(), prec
    finally:
        F.fetirp_destroy(ctx)


def test_c3_operator_at_the_bench_width(c3):
    """The block operator in the benchmark's launch configuration (k = 4: R_p = 256 right-hand sides per
    pattern, one 256-column tile, the reduction dimension of the tensor-core product split over two CTAs),
    compared element by element with the oracle on all four columns."""
    prob = config("c3", k=4)
    orc = FetiOracle(prob, use_schur=False)
    ctx = F.fetirp_create(F.fetirp_default_options())
    try:
        F.load_problem(ctx, prob)
        F.fetirp_prepare(ctx, prob.n_lambda, prob.c)
        V = np.random.default_rng(22).standard_normal((prob.n_lambda, 4))
        Qo = orc.PtFP(V)
        for prec, tol in (("fp64", 1e-9), ("tf32x3", 5e-4), ("bf16x3", 1e-3)):
            Q = F.fetirp_apply_block(ctx, V, F.PRECISIONS[prec])
            rel = np.linalg.norm(Q - Qo) / np.linalg.norm(Qo)
            assert rel < tol, (prec, rel)
            assert np.abs(Q - Qo).max() < 10 * tol * np.abs(Qo).max(), prec
    finally:
        F.fetirp_destroy(ctx)


@pytest.mark.parametrize("prec,k", [("tf32x3", 32), ("bf16x3", 32), ("bf16x3", 4)])
def test_c3_solve_satisfies_the_equations(c3, prec, k):
    """k = 4 with bf16x3 is the benchmark's configuration."""
    if k != 32:
        c3 = config("c3", k=k)
    ctx = F.fetirp_create(F.fetirp_default_options(precision=prec, tol=1e-8, max_iter=3000))
    try:
        F.load_problem(ctx, c3)
        lam, u, st = F.fetirp_solve(ctx, c3.n_lambda, c3.c, F.n_u(c3))
    finally:
        F.fetirp_destroy(ctx)
    assert st["rel_residual"] <= 1e-8 and st["outer_steps"] >= 1
    us = F.split_u(c3, u)
    B, offs = B_matrix(c3)
    # equilibrium of every occurrence: K(s) u(s) + B(s)^T lambda = f(s)
    Bt_lam = B.T @ lam
    num = den = 0.0
    for s in range(c3.n_occ):
        Ks = occurrence_stiffness(c3, s)
        res = Ks @ us[s] + Bt_lam[offs[s]:offs[s + 1]] - c3.occs[s].f_global
        num += res @ res
        den += c3.occs[s].f_global @ c3.occs[s].f_global
    assert np.sqrt(num / den) < 1e-6
    # continuity: B u = c (u of magnitude ~ |u|, so relative to |u|).  The defect is the dual residual of the
    # solve, stopped at 1e-8 relative: here |B u - c| / |u| ~ 0.21 x the final relative residual, so <= 2.1e-9
    ucat = np.concatenate(us)
    assert np.linalg.norm(B @ ucat - c3.c) / np.linalg.norm(ucat) < 3e-9
    # (G^T lambda = e follows from the equilibrium: N(s)^T (f(s) - B(s)^T lambda) = N(s)^T K(s) u(s) = 0.)
    # Together, equilibrium and continuity are the global FE equations (Eq. 1) with B of full row rank, so they
    # determine u and lambda.
