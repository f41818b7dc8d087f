"""Batched uneven structures: independent clamped blocks of different elastic patterns solved as one
structure (one local-product launch covers every pattern, iterations replayed as one CUDA graph), with the
multivector width picked by the autotuner.  Reduced sizes (2^3 .. 6^3 patterns); the full-size batch
(8^3 .. 24^3, 256 occurrences) uses the same code path."""
import numpy as np
import pytest

from fetirp_gen import batched_uneven
from oracle.direct import direct

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_batched_uneven_matches_oracle_with_autotuned_k(prec):
    prob = batched_uneven(ms=(2, 3, 4, 6), weights=(0.4, 0.3, 0.2, 0.1), n_occ=40, seed=2)
    us_ref, lam_ref, _, _ = direct(prob)
    ctx = F.fetirp_create(F.fetirp_default_options(precision=prec, tol=1e-10))
    try:
        F.load_problem(ctx, prob, groups=False)
        best, times = F.fetirp_autotune_k(ctx, prob.n_lambda, prob.c, (4, 8, 16, 32))
        assert best in (4, 8, 16, 32) and np.isfinite(times).all()
        assert times[[4, 8, 16, 32].index(best)] == times.min()
        lam, u, st = F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob))
    finally:
        F.fetirp_destroy(ctx)
    assert np.linalg.norm(lam - lam_ref) / np.linalg.norm(lam_ref) < 1e-8
    for a, b in zip(F.split_u(prob, u), us_ref):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8
