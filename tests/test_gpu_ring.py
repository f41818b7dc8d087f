"""GPU parity on the periodic ring stand-in (n annulus sectors, each the pattern rotated by 2 pi k / n; Section
3.1 and, for plane strain, Section 4.2), through the C ABI:

- the occurrence split on rings of 2D heat and of plane-strain elasticity, whose rotations by 72 or 40 degrees
  are general rotations of a vector field (turned node by node on the device), against the oracle's direct
  solve in every precision;
- the permutation multivector of Eq. 8, [z, Pi z, ..., Pi^(n-1) z], with and without the periodic shortcut
  (one single-column F-apply per iteration, permuted), against the oracle's permutation loop iterate by
  iterate and against the direct solve;
- the paper's trend: with the permutation multivector the block iteration count stays flat from 5 to 9
  repetitions while classical FETI grows (Sections 3.4 and 4.2)."""
import numpy as np
import pytest

from fetirp_gen.ring import ring_elastic, ring_heat, ring_permutation
from oracle.direct import direct
from oracle.permute import PermutationFeti

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")

RING = {"heat": ring_heat, "elastic": ring_elastic}


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def solve(prob, Pi=None, shortcut=False, **kw):
    ctx = F.fetirp_create(F.fetirp_default_options(**kw))
    try:
        F.load_problem(ctx, prob)
        if Pi is not None:
            F.fetirp_set_permutation(ctx, Pi, prob.n_occ, shortcut)
        return F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob), allow_noconv=kw.get("tol", 1.0) < 1e-200)
    finally:
        F.fetirp_destroy(ctx)


@pytest.mark.parametrize("n", [5, 9])
@pytest.mark.parametrize("physics", ["heat", "elastic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_ring_matches_the_direct_solve(n, physics, prec):
    prob = RING[physics](n, m_t=6, m_r=5, seed=4)
    us_ref, lam_ref, _, _ = direct(prob)
    lam, u, st = solve(prob, precision=prec, tol=1e-12, inner_tol=1e-5)
    assert st["rel_residual"] <= 1e-12
    assert rel(lam, lam_ref) < 1e-8, (rel(lam, lam_ref), st)
    for a, b in zip(F.split_u(prob, u), us_ref):
        assert rel(a, b) < 1e-8


@pytest.mark.parametrize("physics", ["heat", "elastic"])
@pytest.mark.parametrize("shortcut", [False, True])
def test_permutation_iterates_match_the_oracle(physics, shortcut):
    """lambda after 1, 2 and 4 block iterations of the permutation multivector equals the oracle's (Eq. 8 and
    Table 1, right column), in FP64; the shortcut takes the F-image of the block from one column."""
    prob = RING[physics](5, m_t=4, m_r=4, seed=2)
    Pi = ring_permutation(prob)
    orc = PermutationFeti(prob, Pi)
    for its in (1, 2, 4):
        lam_o, _, _ = orc.multivector(tol=0.0, max_it=its)
        lam, _, st = solve(prob, Pi, shortcut, tol=1e-300, max_iter=its, check_every=1)
        assert st["iterations"] == its
        assert rel(lam, lam_o) < 1e-9, (its, rel(lam, lam_o))


@pytest.mark.parametrize("physics", ["heat", "elastic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("shortcut", [False, True])
def test_permutation_solve_matches_the_direct_solve(physics, prec, shortcut):
    prob = RING[physics](9, m_t=6, m_r=5, seed=5)
    us_ref, lam_ref, _, _ = direct(prob)
    lam, u, st = solve(prob, ring_permutation(prob), shortcut, precision=prec, tol=1e-12, inner_tol=1e-5)
    assert st["rel_residual"] <= 1e-12
    assert rel(lam, lam_ref) < 1e-8, (rel(lam, lam_ref), st)
    for a, b in zip(F.split_u(prob, u), us_ref):
        assert rel(a, b) < 1e-8


@pytest.mark.parametrize("physics", ["heat", "elastic"])
def test_permutation_iteration_count_is_flat(physics):
    """From 5 to 9 sectors the permutation multivector's block iteration count stays flat (at most one more),
    while classical FETI (k = 1) needs more iterations and more with more sectors (the trend of the paper's
    Tables 2 and 3)."""
    its, classical = {}, {}
    for n in (5, 9):
        prob = RING[physics](n, m_t=4, m_r=4, seed=0)
        _, _, st = solve(prob, ring_permutation(prob), True, tol=1e-10, check_every=1)
        its[n] = st["iterations"]
        ctx = F.fetirp_create(F.fetirp_default_options(tol=1e-10, check_every=1))
        try:
            F.load_problem(ctx, prob, groups=False)
            F.fetirp_set_groups(ctx, 1, np.zeros(prob.n_occ, dtype=np.int32))
            classical[n] = F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob))[2]["iterations"]
        finally:
            F.fetirp_destroy(ctx)
    assert its[9] <= its[5] + 1, (its, classical)
    assert classical[9] > classical[5] and its[9] < classical[9], (its, classical)


def test_shortcut_refused_on_a_structure_that_is_not_periodic():
    """A map that does not commute with P^T F P (here the ring's permutation on a grid whose rows it does not
    rotate) is refused when the shortcut is asked for."""
    from fetirp_gen import heat_grid
    import scipy.sparse as sp
    prob = heat_grid(4, (3, 1), k=3, seed=1)
    n = prob.n_lambda
    Pi = sp.csr_matrix((np.ones(n), (np.roll(np.arange(n), 1), np.arange(n))), shape=(n, n))
    ctx = F.fetirp_create(F.fetirp_default_options())
    try:
        F.load_problem(ctx, prob)
        F.fetirp_set_permutation(ctx, Pi, 3, True)
        with pytest.raises(F.FetirpError) as e:
            F.fetirp_prepare(ctx, prob.n_lambda, prob.c)
        assert e.value.status == F.FETIRP_EINVAL and "shortcut" in str(e.value)
    finally:
        F.fetirp_destroy(ctx)
