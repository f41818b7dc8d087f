"""Pins of the preconditioned oracle (Eqs. 4-7 and Table 1 with a preconditioner): what the mathematics fixes,
independently of how the oracle writes the formulas down."""
import numpy as np
import pytest

from fetirp_gen import elastic_grid, heat_grid
from oracle.direct import direct
from oracle.feti import FetiOracle
from oracle.precond import KINDS, PreconditionedFeti


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def checker():
    # heat, 1 / 1000 conductivity checkerboard, rotated occurrences, ragged grid
    return heat_grid(4, (3, 3), kappas=(1.0, 1000.0), checker=True, rotate=True, k=3, seed=2)


@pytest.fixture(scope="module")
def elastic():
    return elastic_grid(2, (2, 2, 1), n_patterns=2, k=2, seed=4)


@pytest.mark.parametrize("which", ["checker", "elastic"])
@pytest.mark.parametrize("scaling", ["stiffness", "multiplicity"])
def test_scaling_is_a_partition_of_unity(which, scaling, checker, elastic):
    prob = checker if which == "checker" else elastic
    pf = PreconditionedFeti(prob, "lumped", scaling)
    D, inc = pf.Delta, pf.o.incidence
    assert np.allclose(D.sum(1), 1.0, rtol=0, atol=1e-15)
    assert np.all(D >= 0) and np.all(D[inc == 0] == 0)


def test_stiffness_scaling_closed_form_on_the_checkerboard(checker):
    """Across a 1 / 1000 interface the soft side's share is 1000/1001 and the stiff side's 1/1001: both
    sides see the same local node type (edge or corner), so their diagonal stiffness ratio is the
    conductivity ratio."""
    pf = PreconditionedFeti(checker, "lumped", "stiffness")
    kap = np.array([checker.patterns[o.pattern].material["kappa"] for o in checker.occs])
    inc = pf.o.incidence
    n_checked = 0
    for r in range(checker.n_lambda):
        occ = np.nonzero(inc[r])[0]
        if len(occ) != 2:
            assert pf.Delta[r, occ[0]] == 1.0
            continue
        assert kap[occ[0]] != kap[occ[1]]
        for s, t in ((occ[0], occ[1]), (occ[1], occ[0])):
            assert abs(pf.Delta[r, s] - kap[t] / (kap[s] + kap[t])) < 1e-14
        n_checked += 1
    assert n_checked > 20


def test_identity_preconditioner_reduces_to_the_plain_solver(checker):
    pf = PreconditionedFeti(checker, "identity")
    lam_a, it_a, _ = pf.classical_cg(tol=1e-10)
    lam_b, it_b, _ = FetiOracle(checker).classical_cg(tol=1e-10)
    assert it_a == it_b and rel(lam_a, lam_b) < 1e-13


@pytest.mark.parametrize("kind", ["dirichlet", "lumped", "superlumped"])
def test_projector_and_initialisation(kind, elastic):
    pf = PreconditionedFeti(elastic, kind)
    G = pf.o.G
    V = np.random.default_rng(0).standard_normal((elastic.n_lambda, 3))
    QV = pf.Q(V)
    assert rel(pf.Q(QV), QV) < 1e-12                                   # a projector
    assert np.linalg.norm(G.T @ QV) < 1e-10 * np.linalg.norm(G) * np.linalg.norm(V)   # onto ker(G^T)
    assert np.linalg.norm(pf.Qt(G)) < 1e-10 * np.linalg.norm(G)          # Q^T removes range(G)
    assert rel(G.T @ pf.lambda0(), pf.o.e()) < 1e-12                   # G^T lambda_0 = e


@pytest.mark.parametrize("kind", ["dirichlet", "lumped", "superlumped"])
def test_preconditioner_symmetric_psd(kind, checker):
    pf = PreconditionedFeti(checker, kind)
    M = pf.M(np.eye(checker.n_lambda))
    assert np.linalg.norm(M - M.T) <= 1e-13 * np.linalg.norm(M)
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() >= -1e-12 * ev.max() and ev.max() > 0


def test_dirichlet_operator_is_the_primal_schur_complement(elastic):
    """S(s) annihilates the rigid modes restricted to the boundary and is positive semidefinite of corank 6
    (a floating elastic body): the defining properties of the condensed stiffness."""
    pf = PreconditionedFeti(elastic, "dirichlet")
    for s in range(elastic.n_occ):
        S = pf.X[s]
        Nb = pf.o.Ns[s][pf.bd[s]]
        assert np.linalg.norm(S @ Nb) < 1e-10 * np.linalg.norm(S) * np.linalg.norm(Nb)
        ev = np.linalg.eigvalsh(S)
        assert np.sum(ev < 1e-10 * ev.max()) == 6


@pytest.mark.parametrize("which", ["checker", "elastic"])
@pytest.mark.parametrize("kind", ["dirichlet", "lumped", "superlumped"])
def test_preconditioned_solves_reproduce_the_direct_solve(which, kind, checker, elastic):
    prob = checker if which == "checker" else elastic
    us_ref, lam_ref, _, _ = direct(prob)
    pf = PreconditionedFeti(prob, kind)
    for solver in (pf.classical_cg, pf.multivector):
        lam, it, hist = solver(tol=1e-12)
        assert hist[-1] <= 1e-12
        assert rel(lam, lam_ref) < 1e-8, (kind, solver.__name__)
        _, us = pf.o.recover(lam)
        for a, b in zip(us, us_ref):
            assert rel(a, b) < 1e-8


def test_preconditioners_cut_iterations_on_the_contrast(checker):
    """On the 1 / 1000 checkerboard the scaled preconditioners need fewer classical iterations than the
    identity, the Dirichlet one the fewest (the order of efficiency of Eqs. 4-5)."""
    its = {k: PreconditionedFeti(checker, k).classical_cg(tol=1e-8)[1] for k in KINDS}
    assert its["dirichlet"] <= its["lumped"] < its["identity"]
    assert its["superlumped"] < its["identity"]


def test_planted_one_sided_scaling_is_caught(checker, monkeypatch):
    """Dropping the right-hand scaling Delta(s) in the preconditioner (a plausible slip) makes it
    nonsymmetric: the symmetry pin fails."""
    pf = PreconditionedFeti(checker, "lumped")

    def M_wrong(V):
        V = np.asarray(V, dtype=float)
        out = np.zeros_like(V)
        for s in range(checker.n_occ):
            Bs = pf.o.Bs[s]
            Ds = pf.Delta[:, s][:, None]
            Y = (Bs.T @ V)[pf.bd[s]]
            Z = np.zeros((Bs.shape[1], V.shape[1]))
            Z[pf.bd[s]] = pf.X[s] @ Y
            out += Ds * (Bs @ Z)
        return out

    monkeypatch.setattr(pf, "M", M_wrong)
    M = pf.M(np.eye(checker.n_lambda))
    assert np.linalg.norm(M - M.T) > 1e-3 * np.linalg.norm(M)
