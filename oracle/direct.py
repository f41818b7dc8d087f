"""Plain definition of the solution: assemble the global stiffness, solve K u = f directly (Eq. 1), then
recover the interface reactions lambda from the subdomain equilibria (Eq. 2).  FP64, scipy sparse LU.
Test infrastructure only (see oracle/__init__.py)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def rotation_blocks(prob, o):
    """R-hat for occurrence o: the per-node rotation acting on dof vectors (global = R-hat local).
    Scalar problems (dpn = 1) have no components to rotate."""
    occ = prob.occs[o]
    n = prob.patterns[occ.pattern].n_nodes
    if prob.dpn == 1:
        return sp.identity(n, format="csr")
    R = occ.rot[:prob.dpn, :prob.dpn].astype(float)
    return sp.kron(sp.identity(n), sp.csr_matrix(R), format="csr")


def occurrence_stiffness(prob, o):
    """K(s) in the global frame: R-hat K_pattern R-hat^T (the pattern is meshed once, Sec. 4.2)."""
    Rh = rotation_blocks(prob, o)
    Kp = prob.patterns[prob.occs[o].pattern].K
    return (Rh @ Kp @ Rh.T).tocsr()


def global_stiffness(prob):
    """K^Omega = sum_s of the occurrence stiffnesses placed on global dofs (Eq. 1)."""
    n = prob.n_global_nodes * prob.dpn
    rows, cols, vals = [], [], []
    for o in range(prob.n_occ):
        Ks = occurrence_stiffness(prob, o).tocoo()
        dofs = prob.occ_dofs(o)
        rows.append(dofs[Ks.row]); cols.append(dofs[Ks.col]); vals.append(Ks.data)
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return K.tocsr()


def global_load(prob):
    """f^Omega = sum_s f(s) (each shared nodal load was split over its owners, so the sum restores it)."""
    f = np.zeros(prob.n_global_nodes * prob.dpn)
    for o in range(prob.n_occ):
        np.add.at(f, prob.occ_dofs(o), prob.occs[o].f_global)
    return f


def dirichlet_dofs(prob):
    dofs = (prob.dirichlet_nodes[:, None] * prob.dpn + np.arange(prob.dpn)[None, :]).ravel()
    return dofs, prob.dirichlet_values.ravel()


def solve_direct(prob):
    """u^Omega with the Dirichlet dofs eliminated: K_ff u_f = f_f - K_fd u_d (Eq. 1)."""
    K = global_stiffness(prob)
    f = global_load(prob)
    n = K.shape[0]
    dd, dv = dirichlet_dofs(prob)
    used = np.unique(np.concatenate([prob.occ_dofs(o) for o in range(prob.n_occ)]))   # nodes of occupied cells
    free = np.setdiff1d(used, dd)
    u = np.zeros(n)
    u[dd] = dv
    rhs = f[free] - K[free][:, dd] @ dv
    lu = spla.splu(K[free][:, free].tocsc())
    u[free] = lu.solve(rhs)
    return u


def B_matrix(prob):
    """The signed Boolean B = [B(1) ... B(n)] in the global frame, columns = concatenated occurrence dofs."""
    offs = np.concatenate([[0], np.cumsum([prob.patterns[o.pattern].n_dofs for o in prob.occs])])
    rows, cols, vals = [], [], []
    for oi, o in enumerate(prob.occs):
        rows.append(o.link_lambda_row.astype(np.int64))
        cols.append(offs[oi] + o.link_local_node.astype(np.int64) * prob.dpn + o.link_global_comp)
        vals.append(o.link_sign.astype(float))
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(prob.n_lambda, offs[-1])).tocsr()
    return B, offs


def split_u(prob, u_global):
    """u(s) for every occurrence: the global field read on its dofs (global frame)."""
    return [u_global[prob.occ_dofs(o)] for o in range(prob.n_occ)]


def reactions_lambda(prob, u_global):
    """lambda from Eq. 2: B(s)^T lambda = f(s) - K(s) u(s) for all s, solved as (B B^T) lambda = B rho
    (B has full row rank, so lambda is unique)."""
    B, offs = B_matrix(prob)
    us = split_u(prob, u_global)
    rho = np.concatenate([prob.occs[o].f_global - occurrence_stiffness(prob, o) @ us[o] for o in range(prob.n_occ)])
    lam = spla.splu((B @ B.T).tocsc()).solve(B @ rho)
    return lam, np.linalg.norm(B.T @ lam - rho) / max(np.linalg.norm(rho), 1e-300)


def direct(prob):
    """(u per occurrence in the global frame, lambda, consistency residual of B^T lambda = rho)."""
    u = solve_direct(prob)
    lam, res = reactions_lambda(prob, u)
    return split_u(prob, u), lam, res, u
