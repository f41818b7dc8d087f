"""Brute force for tiny meshes (test infrastructure only): Moore-Penrose pseudo-inverses of every K(s), a
kernel basis from the SVD, and a dense solve of the saddle-point system of Eq. 3.  Nothing here is shared
with oracle.feti: a different generalized inverse and a different kernel basis give the same lambda."""
from __future__ import annotations

import numpy as np

from .direct import occurrence_stiffness, B_matrix


def dual_dense(prob, tol=1e-10):
    B, offs = B_matrix(prob)
    B = B.toarray()
    F = np.zeros((prob.n_lambda, prob.n_lambda))
    d = -prob.c.copy()
    Gc, e = [], []
    for o in range(prob.n_occ):
        K = occurrence_stiffness(prob, o).toarray()
        Bs = B[:, offs[o]:offs[o + 1]]
        Kp = np.linalg.pinv(K, rcond=tol, hermitian=True)
        U, sv, _ = np.linalg.svd(K)
        N = U[:, sv < tol * sv[0]]
        f = prob.occs[o].f_global
        F += Bs @ Kp @ Bs.T
        d += Bs @ Kp @ f
        Gc.append(Bs @ N)
        e.append(N.T @ f)
    return F, np.hstack(Gc), d, np.concatenate(e)


def solve_eq3(prob):
    """lambda from the dense saddle-point system [F G; G^T 0][lambda; alpha] = [d; e] (Eq. 3)."""
    F, G, d, e = dual_dense(prob)
    n, m = F.shape[0], G.shape[1]
    A = np.block([[F, G], [G.T, np.zeros((m, m))]])
    sol = np.linalg.solve(A, np.concatenate([d, e]))
    return sol[:n], sol[n:]
