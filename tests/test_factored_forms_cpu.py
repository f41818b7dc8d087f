"""The algebra of two reformulations the GPU path makes with the factor (neither is in the paper, which forms S^+
and solves the local problems on a CPU).  Plain numpy on small patterns, independent of the oracle and of the
GPU code.  CPU only.

1. The large patterns' S^dag (formed as a Gram on the tensor cores): S is the boundary Schur complement of a
   floating pattern, L its Cholesky factor with every zero pivot's column cleared and a unit diagonal put in its
   place (the generalized inverse of Sec. 2), Lam = L^{-1} with the zero-pivot rows cleared, N_b the kernel traces
   and Pi = I - N_b (N_b^T N_b)^{-1} N_b^T.  Then Lam^T Lam is a reflexive generalized inverse of S and
   (Lam Pi)^T (Lam Pi) its Moore-Penrose inverse, numpy's SVD pinv; a dropped kernel vector must be caught.
2. The recovery's forward sweep of f - B^T lambda as the sweep of f minus a sweep of B^T lambda that starts at
   the boundary block (boundary dofs ordered last)."""
import numpy as np
import pytest
import scipy.linalg as sla

from fetirp_gen import heat_pattern, elastic_pattern


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def schur(pat):
    K = pat.K.toarray()
    bd = (pat.bnd_nodes[:, None] * pat.dpn + np.arange(pat.dpn)).ravel()
    it = np.setdiff1d(np.arange(pat.n_dofs), bd)
    return K[np.ix_(bd, bd)] - K[np.ix_(bd, it)] @ np.linalg.solve(K[np.ix_(it, it)], K[np.ix_(it, bd)])


def zero_pivot_factor(S, tol=1e-9):
    """Right-looking Cholesky; a pivot <= tol * its original diagonal is a zero pivot: its column is cleared."""
    A = S.copy()
    d0 = np.diag(S).copy()
    L = np.zeros_like(S)
    zp = []
    for j in range(S.shape[0]):
        if A[j, j] <= tol * d0[j]:
            zp.append(j)
            continue
        col = A[j:, j] / np.sqrt(A[j, j])
        L[j:, j] = col
        A[j:, j:] -= np.outer(col, col)
    return L, zp


@pytest.mark.parametrize("make", [lambda: heat_pattern(6, kappa=3.0), lambda: elastic_pattern(3, E=2.0, nu=0.3)],
                         ids=["heat2d_6", "elastic3d_3"])
def test_gram_of_the_projected_factor_inverse_is_the_moore_penrose_inverse(make):
    pat = make()
    S = schur(pat)
    L, zp = zero_pivot_factor(S)
    assert len(zp) == pat.kernel_dim
    Lu = L.copy()
    Lu[zp, zp] = 1.0
    Lam = sla.solve_triangular(Lu, np.eye(S.shape[0]), lower=True)
    Lam[zp, :] = 0.0
    Splus = Lam.T @ Lam
    assert rel(S @ Splus @ S, S) < 1e-10                 # a generalized inverse
    assert rel(Splus @ S @ Splus, Splus) < 1e-10         # reflexive
    Nb = sla.null_space(S, rcond=1e-9)
    assert Nb.shape[1] == pat.kernel_dim
    Pi = np.eye(S.shape[0]) - Nb @ np.linalg.solve(Nb.T @ Nb, Nb.T)
    Y = Lam @ Pi
    Sdag = Y.T @ Y
    ref = np.linalg.pinv(S, rcond=1e-10, hermitian=True)
    assert rel(Sdag, ref) < 1e-9
    assert rel(Pi @ Splus @ Pi, ref) < 1e-9
    # the projected operator is the same for every generalized inverse: on range(S), S^+ and S^dag agree
    x = S @ np.random.default_rng(0).standard_normal(S.shape[0])
    assert rel(Pi @ (Splus @ x), Sdag @ x) < 1e-9
    # a planted mistake: one kernel vector left out of the projector leaves S^dag off by far more
    Nb1 = Nb[:, 1:]
    Pi1 = np.eye(S.shape[0])
    if Nb1.shape[1] > 0:
        Pi1 -= Nb1 @ np.linalg.solve(Nb1.T @ Nb1, Nb1.T)
    Y1 = Lam @ Pi1
    assert rel(Y1.T @ Y1, ref) > 1e-3


def forward_zp(L, zp, B):
    """Forward substitution with the zero-pivot convention of the factor: those rows of the solution are 0."""
    X = np.array(B, dtype=float)
    z = set(zp)
    for j in range(L.shape[0]):
        X[j] = 0.0 if j in z else X[j] / L[j, j]
        X[j + 1:] -= np.outer(L[j + 1:, j], X[j])
    return X


def test_recovery_sweep_splits_into_the_loads_and_a_boundary_only_sweep():
    """The recovery applies the forward sweep to f - B^T lambda as the sweep of f (kept from d) minus the sweep of
    B^T lambda, which lives on the boundary rows (ordered last) and so starts at the boundary block: the interior
    rows of its result are zero and the boundary rows are the sweep with L_S alone."""
    pat = elastic_pattern(3)
    K = pat.K.toarray()
    bd = (pat.bnd_nodes[:, None] * pat.dpn + np.arange(pat.dpn)).ravel()
    it = np.setdiff1d(np.arange(pat.n_dofs), bd)
    order = np.concatenate([it, bd])                     # interior first, boundary last
    Kp = K[np.ix_(order, order)]
    L, zp = zero_pivot_factor(Kp)
    ni = len(it)
    assert len(zp) == pat.kernel_dim and min(zp) >= ni   # zero pivots only in the boundary block
    rng = np.random.default_rng(1)
    f = rng.standard_normal((Kp.shape[0], 3))
    b = np.zeros_like(f)
    b[ni:] = rng.standard_normal((len(bd), 3))           # B^T lambda: boundary rows only
    full = forward_zp(L, zp, f - b)
    tb = forward_zp(L, zp, b)
    assert np.abs(tb[:ni]).max() == 0.0
    LS = L[ni:, ni:]
    tb_s = forward_zp(LS, [z - ni for z in zp], b[ni:])
    assert rel(tb[ni:], tb_s) < 1e-13
    split = forward_zp(L, zp, f)
    split[ni:] -= tb_s
    assert rel(split, full) < 1e-12
