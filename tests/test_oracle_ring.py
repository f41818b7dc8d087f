"""Pins of the periodic ring stand-in and of the permutation multivector (Section 3.1, Eq. 8): the
isoparametric element by the patch test, the periodicity of the dual operator under the supplied
permutation, agreement with the direct solve, and the paper's claims that the block iteration cannot be slower
than the classical one and gains more with more repetitions."""
import numpy as np
import pytest

from fetirp_gen.ring import (plane_strain_D, q1_laplace_quad, q1_plane_strain_quad, ring_elastic, ring_heat,
                             ring_permutation, sector_pattern)
from oracle.direct import direct
from oracle.permute import PermutationFeti


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_quad_element_on_a_square_is_the_q1_closed_form():
    """On the unit square the isoparametric element is the Q1 matrix: diagonal 2/3, edge neighbours -1/6,
    opposite corner -1/3 (corner order (0,0), (1,0), (0,1), (1,1)), in either orientation of the corners."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(q1_laplace_quad(xy), ref, atol=1e-15)
    flipped = xy[:, ::-1]           # a left-handed corner order: same matrix
    assert np.allclose(q1_laplace_quad(flipped), ref, atol=1e-15)


def test_sector_stiffness_is_psd_with_constant_kernel():
    pat = sector_pattern(5, 4, 3)
    K = pat.K.toarray()
    assert np.allclose(K, K.T, atol=1e-14)
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-13 and ev[1] > 1e-6 * ev[-1]


def test_patch_test_linear_field_on_the_ring():
    """Zero source, Dirichlet data of a linear field on both arcs: the direct solve reproduces the field at
    every node (isoparametric bilinear elements are linearly complete)."""
    f = lambda x: 0.3 + 1.7 * x[:, 0] - 0.9 * x[:, 1]
    prob = ring_heat(5, m_t=3, m_r=3, dirichlet="both", dirichlet_fn=f, load="zero")
    us, _, _, _ = direct(prob)
    for o, u in enumerate(us):
        assert np.abs(u - f(prob.global_coords[prob.occs[o].node_map])).max() < 1e-12


def test_plane_strain_element_energy_and_rigid_modes():
    """A uniform strain stores (1/2) eps^T D eps per unit area (pins E, nu and plane strain); the element's
    kernel is the two translations and the rotation (rank 8 - 3)."""
    E, nu = 2.0, 0.3
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]) * 0.5
    K = q1_plane_strain_quad(xy, E, nu)
    G = np.array([[0.3, -0.2], [0.5, 0.1]])          # displacement gradient: u = G x
    u = (xy @ G.T).ravel()
    eps = np.array([G[0, 0], G[1, 1], G[0, 1] + G[1, 0]])
    D = np.array([[1 - nu, nu, 0], [nu, 1 - nu, 0], [0, 0, 0.5 - nu]]) * E / ((1 + nu) * (1 - 2 * nu))
    assert abs(0.5 * u @ K @ u - 0.5 * eps @ D @ eps * 0.25) < 1e-14
    assert np.allclose(plane_strain_D(E, nu), D, atol=1e-15)
    N = np.zeros((4, 2, 3))
    N[:, 0, 0] = 1.0
    N[:, 1, 1] = 1.0
    N[:, 0, 2], N[:, 1, 2] = -xy[:, 1], xy[:, 0]
    assert np.abs(K @ N.reshape(8, 3)).max() < 1e-14
    assert np.linalg.matrix_rank(K, tol=1e-10) == 5


def test_elastic_patch_test_affine_field_on_the_ring():
    """Zero body force, an affine displacement imposed on both arcs: the direct solve reproduces it at every
    node, in every rotated sector (the rotation of the vector components is consistent)."""
    A = np.array([[0.02, -0.05], [0.04, 0.01]])
    b = np.array([0.1, -0.2])
    f = lambda x: x @ A.T + b
    prob = ring_elastic(5, m_t=3, m_r=3, dirichlet="both", dirichlet_fn=f, load="zero")
    us, _, _, _ = direct(prob)
    for o, u in enumerate(us):
        assert np.abs(u - f(prob.global_coords[prob.occs[o].node_map]).ravel()).max() < 1e-12


@pytest.mark.parametrize("make,dpn", [(ring_heat, 1), (ring_elastic, 2)])
@pytest.mark.parametrize("n", [3, 5, 9])
def test_ring_sizes_and_periodicity(n, make, dpn):
    m_t, m_r = 4, 3
    prob = make(n, m_t=m_t, m_r=m_r, seed=2)
    assert prob.n_lambda == dpn * (n * (m_r + 1) + n * m_t)   # radial lines + inner-arc Dirichlet nodes
    pf = PermutationFeti(prob, ring_permutation(prob))
    Pi = pf.Pi.toarray()
    assert np.abs(np.linalg.matrix_power(Pi, n) - np.eye(prob.n_lambda)).max() < 1e-13
    Fd = pf.dense_F()
    assert np.abs(Fd @ Pi - Pi @ Fd).max() <= 1e-12 * np.abs(Fd).max()
    V = np.random.default_rng(0).standard_normal(prob.n_lambda)
    assert rel(pf.project(pf.Pi @ V), pf.Pi @ pf.project(V)) < 1e-12


@pytest.mark.parametrize("make", [ring_heat, ring_elastic])
@pytest.mark.parametrize("n", [5, 9])
def test_permutation_multivector_reproduces_the_direct_solve(n, make):
    prob = make(n, m_t=4, m_r=4, seed=1)
    pf = PermutationFeti(prob, ring_permutation(prob))
    us_ref, lam_ref, _, _ = direct(prob)
    lam, it, hist = pf.multivector(tol=1e-12)
    assert hist[-1] <= 1e-12 and rel(lam, lam_ref) < 1e-9
    _, us = pf.recover(lam)
    for a, b in zip(us, us_ref):
        assert rel(a, b) < 1e-9
    lam_c, it_c, _ = pf.classical_cg(tol=1e-12)
    assert it <= it_c


def test_more_repetitions_gain_more():
    """The relative saving of the permutation multivector over classical FETI grows with the number of
    repetitions of the pattern (the trend of the paper's assessments)."""
    saving = {}
    for n in (5, 9):
        prob = ring_heat(n, m_t=4, m_r=4, seed=1)
        pf = PermutationFeti(prob, ring_permutation(prob))
        it_b = pf.multivector(tol=1e-10)[1]
        it_c = pf.classical_cg(tol=1e-10)[1]
        saving[n] = 1.0 - it_b / it_c
    assert saving[9] > saving[5] > 0.3


@pytest.mark.parametrize("make", [ring_heat, ring_elastic])
def test_dirichlet_preconditioned_permutation_block_is_flat_in_the_repetitions(make):
    """With the Dirichlet preconditioner (the setting of the paper's donut assessments) the permutation
    multivector reproduces the direct solve, and its iteration count does not grow from 5 to 9 repetitions while
    the classical count does (the trend of Tables 2-3)."""
    from oracle.permute import PreconditionedPermutationFeti
    its = {}
    for n in (5, 9):
        prob = make(n, m_t=6, m_r=6, seed=3)
        pf = PreconditionedPermutationFeti(prob, ring_permutation(prob), "dirichlet")
        us_ref, lam_ref, _, _ = direct(prob)
        lam, it_b, hist = pf.multivector(tol=1e-10)
        assert hist[-1] <= 1e-10 and rel(lam, lam_ref) < 1e-8
        it_c = pf.classical_cg(tol=1e-10)[1]
        its[n] = (it_c, it_b)
        assert it_b < it_c
    assert its[9][1] <= its[5][1] + 1 and its[9][0] > its[5][0]
