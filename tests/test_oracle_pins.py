"""Pins of the CPU oracle to things other than itself: closed forms, patch tests, an exact 1D reduction,
brute force on tiny meshes, algebraic invariants of Eq. 3 and the projector, and planted mistakes that must
be caught.  CPU only."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from fetirp_gen import (config, heat_grid, elastic_grid, q1_laplace, q1_elastic3d, elastic_D, heat_pattern,
                        elastic_pattern, set_nodal_load)
from oracle.direct import direct, solve_direct, global_stiffness
from oracle.feti import FetiOracle, analytic_kernel, PatternInverse
from oracle.brute import solve_eq3, dual_dense

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- element matrices (closed forms)
def test_q1_laplace_2d_closed_form():
    ref = np.loadtxt(os.path.join(GOLD, "q1_laplace_2d.txt"))
    for h in (1.0, 0.125, 3.0):
        assert np.allclose(q1_laplace(2, h), ref, atol=1e-15)
    assert np.allclose(q1_laplace(2, 1.0, kappa=1000.0), 1000 * ref)


def test_q1_laplace_3d_closed_form():
    ref = np.loadtxt(os.path.join(GOLD, "q1_laplace_3d_row0.txt"))
    assert np.allclose(q1_laplace(3, 1.0)[0], ref, atol=1e-15)
    assert np.allclose(q1_laplace(3, 0.5), 0.5 * q1_laplace(3, 1.0))   # scales with h in 3D


@pytest.mark.parametrize("E,nu,h", [(1.0, 0.3, 1.0), (210.0, 0.25, 0.0625)])
def test_elastic_uniform_strain_energy(E, nu, h):
    """1/2 u^T K u = 1/2 eps:C:eps * vol exactly for an affine field (full Gauss integration)."""
    rng = np.random.default_rng(0)
    Ke = q1_elastic3d(h, E, nu)
    for _ in range(4):
        A = rng.standard_normal((3, 3))
        corners = np.array([[(a >> d) & 1 for d in range(3)] for a in range(8)]) * h
        u = (corners @ A.T).ravel()
        eps = 0.5 * (A + A.T)
        ev = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[1, 2], 2 * eps[0, 2], 2 * eps[0, 1]])
        assert np.isclose(0.5 * u @ Ke @ u, 0.5 * ev @ elastic_D(E, nu) @ ev * h ** 3, rtol=1e-12)
        # lambda/mu split: a pure rotation (skew A) stores no energy
        S = A - A.T
        us = (corners @ S.T).ravel()
        assert abs(us @ Ke @ us) < 1e-12 * np.abs(Ke).max() * (us @ us)


@pytest.mark.parametrize("pat", [heat_pattern(4), heat_pattern(3, kappa=7.0), elastic_pattern(2), elastic_pattern(3)])
def test_kernel_and_rank(pat):
    N = analytic_kernel(pat)
    K = pat.K.toarray()
    assert np.abs(K @ N).max() < 1e-12 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-10 * ev[-1]) == pat.kernel_dim
    assert np.allclose(K, K.T)


def test_generalized_inverse_property():
    """K K^+ y = y for y in range(K) (Sec. 2, floating subdomains)."""
    for pat in (heat_pattern(4), elastic_pattern(2)):
        inv = PatternInverse(pat)
        rng = np.random.default_rng(1)
        y = pat.K @ rng.standard_normal(pat.n_dofs)
        assert rel(pat.K @ inv.solve(y), y) < 1e-12


# ---------------------------------------------------------------- patch tests and exact solutions
def test_patch_heat_linear_field():
    lin = lambda x: 0.3 + 1.7 * x[:, 0] - 0.4 * x[:, 1]
    for rotate in (False, True):
        p = heat_grid(4, (3, 2), kappas=(5.0, 5.0), checker=True, rotate=rotate, dirichlet="all",
                      dirichlet_fn=lambda x: lin(x)[:, None], load="zero")
        u = solve_direct(p)
        assert np.abs(u - lin(p.global_coords)).max() < 1e-12
        o = FetiOracle(p)
        lam, it, _ = o.classical_cg(1e-14)
        _, us = o.recover(lam)
        for s in range(p.n_occ):
            assert np.abs(us[s] - lin(p.global_coords[p.occs[s].node_map])).max() < 1e-10


def test_patch_elastic_affine_field():
    A = np.array([[0.01, 0.02, -0.03], [0.0, -0.02, 0.01], [0.015, 0.0, 0.005]])
    b = np.array([0.1, -0.2, 0.05])
    fld = lambda x: x @ A.T + b
    p = elastic_grid(2, (2, 1, 2), n_patterns=2, dirichlet="all", dirichlet_fn=fld, load="zero")
    u = solve_direct(p).reshape(-1, 3)
    assert np.abs(u - fld(p.global_coords)).max() < 1e-12
    o = FetiOracle(p)
    lam, it, _ = o.multivector(1e-14)
    _, us = o.recover(lam)
    for s in range(p.n_occ):
        assert np.abs(us[s].reshape(-1, 3) - fld(p.global_coords[p.occs[s].node_map])).max() < 1e-10


def test_heat_strip_flux_exact():
    """u = 0 on x = 0 and a uniform flux q on x = L: the Q1 solution is exactly u = q x / kappa (a 1D
    field that Q1 represents), which pins the Dirichlet rows, the load split and the conductivity."""
    q, kappa, m = 2.5, 3.0, 4
    p = heat_grid(m, (3, 2), kappas=(kappa,), load="zero")
    h = 1.0 / m
    X = p.global_coords
    L = X[:, 0].max()
    f = np.zeros(p.n_global_nodes)
    right = np.isclose(X[:, 0], L)
    f[right] = q * h
    f[right & (np.isclose(X[:, 1], 0) | np.isclose(X[:, 1], X[:, 1].max()))] = q * h / 2
    set_nodal_load(p, f)
    u = solve_direct(p)
    assert np.abs(u - q * X[:, 0] / kappa).max() < 1e-12
    o = FetiOracle(p)
    lam, _, _ = o.classical_cg(1e-14)
    _, us = o.recover(lam)
    assert max(np.abs(us[s] - q * X[p.occs[s].node_map, 0] / kappa).max() for s in range(p.n_occ)) < 1e-10
    # the interface flux through every vertical interface carries the applied load (lambda = -q h)
    _, lam_d, _, _ = direct(p)
    assert rel(lam, lam_d) < 1e-10


# ---------------------------------------------------------------- three-way agreement
@pytest.mark.parametrize("make", [
    lambda: config("c1"),
    lambda: heat_grid(4, (3, 3), kappas=(1.0, 100.0), checker=True, rotate=True, k=3),
    lambda: elastic_grid(2, (2, 2, 1), n_patterns=2, k=4),
    lambda: config("c3r"),
])
def test_direct_feti_brute_agree(make):
    p = make()
    us, lam, res, _ = direct(p)
    assert res < 1e-12          # B^T lambda = rho is consistent: lambda exists
    o = FetiOracle(p)
    lam_cg, it_cg, _ = o.classical_cg(1e-13)
    lam_mv, it_mv, _ = o.multivector(1e-13)
    assert rel(lam_cg, lam) < 1e-9
    assert rel(lam_mv, lam) < 1e-9
    _, us_mv = o.recover(lam_mv)
    assert max(rel(a, b) for a, b in zip(us_mv, us)) < 1e-9
    if p.n_lambda <= 1200:
        lam_b, _ = solve_eq3(p)       # Moore-Penrose pseudo-inverses + SVD kernels
        assert rel(lam_b, lam) < 1e-9


def test_schur_identity_in_F():
    """S^+ = t K^+ t^T: F through the boundary block equals F through full local solves."""
    p = elastic_grid(2, (2, 1, 2), n_patterns=1)
    V = np.random.default_rng(3).standard_normal((p.n_lambda, 3))
    a = FetiOracle(p, use_schur=True).F(V)
    b = FetiOracle(p, use_schur=False).F(V)
    assert rel(a, b) < 1e-12


def test_projector_and_coarse_invariants():
    p = config("c3r")
    o = FetiOracle(p)
    rng = np.random.default_rng(4)
    V = rng.standard_normal((p.n_lambda, 5))
    PV = o.project(V)
    assert rel(o.project(PV), PV) < 1e-13                   # idempotent
    assert np.abs(o.G.T @ PV).max() < 1e-11 * np.abs(V).max()   # range(P) = ker(G^T)
    W = rng.standard_normal((p.n_lambda, 5))
    assert np.isclose(np.sum(o.project(W) * V), np.sum(W * o.project(V)))   # symmetric
    assert rel(o.G.T @ o.lambda0(), o.e()) < 1e-12          # G^T lambda_0 = e


def test_PtFP_symmetric_psd_and_choice_of_inverse():
    """P^T F P is symmetric PSD (F inherits SPD from K on range(P)) and does not depend on the choice of
    generalized inverse: the Moore-Penrose F of the brute force gives the same projected operator."""
    p = heat_grid(4, (3, 2), kappas=(1.0, 10.0), checker=True)
    o = FetiOracle(p)
    P = o.project(np.eye(p.n_lambda))
    A = P @ o.dense_F() @ P
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > -1e-12 * np.abs(A).max()
    Fb, Gb, _, _ = dual_dense(p)
    Pb = np.eye(p.n_lambda) - Gb @ np.linalg.solve(Gb.T @ Gb, Gb.T)
    assert np.allclose(P, Pb, atol=1e-12)
    assert rel(Pb @ Fb @ Pb, A) < 1e-10


def test_multivector_invariants_and_iterations():
    """The block form is never slower than classical CG (the CG direction stays in the block span, Section
    3.1): block iterations <= classical iterations; directions are F-orthonormal across blocks and lie in
    ker(G^T)."""
    for p in (config("c1"), heat_grid(4, (4, 2), kappas=(1.0, 50.0), checker=True, k=4), config("c3r")):
        o = FetiOracle(p)
        _, it_cg, _ = o.classical_cg(1e-10)
        _, it_mv, _ = o.multivector(1e-10)
        assert it_mv <= it_cg
    p = config("c1")
    o = FetiOracle(p)
    # rerun the block loop by hand for three steps and check W_i^T P~_j = delta_ij I
    lam = o.lambda0()
    r = o.project(o.d() - o.F(lam))
    Ws, Ps = [], []
    for _ in range(3):
        Wt = o.project(o.split(o.project(r)))
        for Wi, Pi in zip(Ws, Ps):
            Wt = Wt - Wi @ (Pi.T @ Wt)
        Pt = o.project(o.F(Wt))
        ev, V = np.linalg.eigh(0.5 * (Wt.T @ Pt + Pt.T @ Wt))
        keep = ev > 1e-12 * ev.max()
        T = V[:, keep] / np.sqrt(ev[keep])
        Wt, Pt = Wt @ T, Pt @ T
        r = r - Pt @ (Wt.T @ r)
        Ws.append(Wt); Ps.append(Pt)
    Wall, Pall = np.hstack(Ws), np.hstack(Ps)
    assert np.allclose(Wall.T @ Pall, np.eye(Wall.shape[1]), atol=1e-10)
    assert np.abs(o.G.T @ Wall).max() < 1e-12
    assert np.abs(Wall.T @ r).max() < 1e-10 * np.linalg.norm(r) * 10 + 1e-14


def test_split_sums_to_vector():
    p = config("c2", k=8)
    o = FetiOracle(p)
    z = np.random.default_rng(5).standard_normal(p.n_lambda)
    Z = o.split(z)
    assert Z.shape == (p.n_lambda, 8)
    assert rel(Z.sum(1), z) < 1e-15


# ---------------------------------------------------------------- planted mistakes must be caught
def _agree(p, o):
    _, lam, _, _ = direct(p)
    lam_f, _, _ = o.classical_cg(1e-13)
    return rel(lam_f, lam) < 1e-8


def test_planted_sign_error_in_B_is_caught(monkeypatch):
    import oracle.feti as feti
    p = heat_grid(4, (2, 2), kappas=(1.0,), load="uniform")
    assert _agree(p, feti.FetiOracle(p))
    good = feti.B_matrix

    def bad_B(prob):
        B, offs = good(prob)
        B = B.toarray()
        row = prob.occs[1].link_lambda_row[3]
        B[row, offs[1]:offs[2]] *= -1.0
        return sp.csr_matrix(B), offs
    monkeypatch.setattr(feti, "B_matrix", bad_B)   # planted: one wrong sign in one occurrence's B
    assert not _agree(p, feti.FetiOracle(p))


def test_planted_dropped_term_in_d_is_caught():
    p = config("c1")
    o = FetiOracle(p)
    d_ok = o.d
    o.d = lambda: d_ok() + p.c + 0.5 * o.Bs[0] @ o.kplus(0, p.occs[0].f_global) * 0  # neutral change
    assert _agree(p, o)
    o.d = lambda: d_ok() - o.Bs[0] @ o.kplus(0, p.occs[0].f_global)   # planted: one occurrence dropped
    assert not _agree(p, o)


def test_planted_transposed_rotation_is_caught():
    p = elastic_grid(2, (2, 1, 1), n_patterns=1, k=2, seed=0)
    assert any(not np.array_equal(o.rot, np.eye(3)) and not np.array_equal(o.rot, o.rot.T) for o in p.occs)
    assert _agree(p, FetiOracle(p))
    o = FetiOracle(p)
    o.Rh = [R.T.tocsr() for R in o.Rh]   # planted: local <-> global frames swapped
    assert not _agree(p, o)
