"""GPU parity on the periodic ring stand-in: annulus sectors of 2D heat (isoparametric Q1) rotated by 72 or 40
degrees, solved through the C ABI and compared with the oracle's direct solve.  Scalar patterns take any
rotation (there are no components to turn)."""
import numpy as np
import pytest

from fetirp_gen.ring import ring_heat
from oracle.direct import direct

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n", [5, 9])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_heat_ring_matches_the_direct_solve(n, prec):
    prob = ring_heat(n, m_t=6, m_r=5, seed=4)
    us_ref, lam_ref, _, _ = direct(prob)
    ctx = F.fetirp_create(F.fetirp_default_options(precision=prec, tol=1e-12, inner_tol=1e-5))
    try:
        F.load_problem(ctx, prob)
        lam, u, st = F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob))
    finally:
        F.fetirp_destroy(ctx)
    assert st["rel_residual"] <= 1e-12
    assert rel(lam, lam_ref) < 1e-8
    for a, b in zip(F.split_u(prob, u), us_ref):
        assert rel(a, b) < 1e-8
