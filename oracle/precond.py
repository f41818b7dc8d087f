"""Preconditioned FETI: the Dirichlet, lumped and superlumped preconditioners of Eqs. 4-5 with their diagonal
scaling, the preconditioner-weighted projector and initialisation of Eqs. 6-7, and the classical and multivector
solvers of Table 1 with a preconditioner.  Plain FP64 numpy/scipy, restated from the paper; test infrastructure
only (see oracle/__init__.py), built on FetiOracle for F, G, d, e.

The paper states the scaling only as a diagonal operator per occurrence on the interface with
sum_s Delta(s) = I.  Two choices are provided:
  - "multiplicity": each of the r occurrences of a row gets 1 / r (FetiOracle.Delta);
  - "stiffness": on a gluing row between occurrences s and t at global dof i, Delta(s) = K(t)_ii /
    (K(s)_ii + K(t)_ii) (the other side's share of the diagonal stiffness; each side's diagonal taken in the
    global frame), and 1 on a Dirichlet row.  This is the stiffness scaling that keeps heterogeneous
    coefficients (the 1 / 1000 checkerboard) from degrading the preconditioner.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .direct import occurrence_stiffness
from .feti import FetiOracle

KINDS = ("identity", "dirichlet", "lumped", "superlumped")


class PreconditionedFeti:
    def __init__(self, prob, kind="lumped", scaling="stiffness", base: FetiOracle | None = None):
        if kind not in KINDS:
            raise ValueError(kind)
        self.prob = prob
        self.kind = kind
        self.o = base if base is not None else FetiOracle(prob)
        o = self.o
        n_occ = prob.n_occ
        # boundary dofs of every occurrence (global frame, occurrence dof numbering) and the boundary blocks
        self.bd = [o.inv[prob.occs[s].pattern].bnd_dofs for s in range(n_occ)]
        self.Kg = [occurrence_stiffness(prob, s) for s in range(n_occ)]
        self.Delta = self._scaling(scaling)
        self.X = [self._local_operator(s) for s in range(n_occ)] if kind != "identity" else None
        # Gram of the coarse space in the preconditioner's metric (Eqs. 6-7)
        MG = self.M(o.G)
        self.MG = MG
        self.GtMG = o.G.T @ MG
        self.GtMG_inv = np.linalg.inv(self.GtMG)

    # ---- scaling and local operators (Eqs. 4-5) ------------------------------------------------------------
    def _scaling(self, scaling):
        o, prob = self.o, self.prob
        if scaling == "multiplicity":
            return o.Delta.copy()
        if scaling != "stiffness":
            raise ValueError(scaling)
        # diagonal stiffness of each occurrence at the dof of each of its links (global frame)
        kd = np.zeros((prob.n_lambda, prob.n_occ))
        for s in range(prob.n_occ):
            Bs = o.Bs[s].tocoo()           # rows = lambda rows, cols = occurrence dofs
            diag = self.Kg[s].diagonal()
            kd[Bs.row, s] = diag[Bs.col]
        inc = o.incidence
        D = np.zeros_like(kd)
        cnt = inc.sum(1)
        for r in range(prob.n_lambda):
            occ = np.nonzero(inc[r])[0]
            if cnt[r] == 1:
                D[r, occ[0]] = 1.0
            else:
                tot = kd[r, occ].sum()
                for s in occ:   # the share of the other occurrences' stiffness
                    D[r, s] = (tot - kd[r, s]) / ((len(occ) - 1) * tot)
        return D

    def _local_operator(self, s):
        """X(s) on the boundary dofs of occurrence s: the primal Schur complement S(s) = K_bb - K_bi K_ii^{-1}
        K_ib (Dirichlet), K_bb (lumped) or diag(K_bb) (superlumped), global frame."""
        K = self.Kg[s]
        bd = self.bd[s]
        if self.kind == "lumped":
            return K[bd][:, bd].toarray()
        if self.kind == "superlumped":
            return np.diag(K.diagonal()[bd])
        inner = np.setdiff1d(np.arange(K.shape[0]), bd)
        Kii = K[inner][:, inner].tocsc()
        Kib = K[inner][:, bd].toarray()
        return K[bd][:, bd].toarray() - Kib.T @ spla.splu(Kii).solve(Kib)

    def M(self, V):
        """The preconditioner tilde-F^{-1} V = sum_s Delta(s) B(s) X(s) B(s)^T Delta(s) V (Eqs. 4-5)."""
        V = np.asarray(V, dtype=float)
        if self.kind == "identity":
            return V.copy()
        one = V.ndim == 1
        V2 = V[:, None] if one else V
        out = np.zeros_like(V2)
        for s in range(self.prob.n_occ):
            Bs = self.o.Bs[s]
            Ds = self.Delta[:, s][:, None]
            Y = (Bs.T @ (Ds * V2))[self.bd[s]]
            Z = np.zeros((Bs.shape[1], V2.shape[1]))
            Z[self.bd[s]] = self.X[s] @ Y
            out += Ds * (Bs @ Z)
        return out[:, 0] if one else out

    # ---- coarse problem with the preconditioner (Eqs. 6-7) -------------------------------------------------
    def Q(self, V):
        """Q V = V - tilde-F^{-1} G (G^T tilde-F^{-1} G)^{-1} G^T V."""
        G = self.o.G
        return V - self.MG @ (self.GtMG_inv @ (G.T @ V))

    def Qt(self, V):
        """Q^T V = V - G (G^T tilde-F^{-1} G)^{-1} G^T tilde-F^{-1} V."""
        G = self.o.G
        return V - G @ (self.GtMG_inv @ (self.MG.T @ V))

    def lambda0(self):
        """lambda_0 = tilde-F^{-1} G (G^T tilde-F^{-1} G)^{-1} e (Table 1's initialisation, lambda_00 = 0)."""
        return self.MG @ (self.GtMG_inv @ self.o.e())

    # ---- Table 1 with a preconditioner ---------------------------------------------------------------------
    def classical_cg(self, tol=1e-8, max_it=10000):
        """Classical FETI (Table 1, left): r = Q^T (d - F lambda), z = Q tilde-F^{-1} r, p = Q^T F w."""
        o = self.o
        lam = self.lambda0()
        r = self.Qt(o.d() - o.F(lam))
        r0 = np.linalg.norm(r)
        hist = [1.0]
        z = self.Q(self.M(r))
        w = z.copy()
        it = 0
        while hist[-1] > tol and it < max_it:
            p = self.Qt(o.F(w))
            wp = w @ p
            alpha = (w @ r) / wp
            lam = lam + alpha * w
            r = r - alpha * p
            z = self.Q(self.M(r))
            beta = -(p @ z) / wp
            w = z + beta * w
            it += 1
            hist.append(np.linalg.norm(r) / r0)
        return lam, it, np.array(hist)

    def split(self, z, groups=None, k=None):
        """Occurrence split of z with this preconditioner's scaling: column g = sum over the occurrences c of
        group g of Delta(c) z (the columns sum to z because sum_c Delta(c) = I)."""
        prob = self.prob
        groups = prob.groups if groups is None else groups
        k = prob.k if k is None else k
        onehot = np.zeros((prob.n_occ, k))
        onehot[np.arange(prob.n_occ), groups] = 1.0
        return (self.Delta * z[:, None]) @ onehot

    def multivector(self, tol=1e-8, max_it=1000, eps_eta=1e-12, groups=None, k=None):
        """Multivector FETI (Table 1, right) with the preconditioner, full reorthogonalisation and the
        F-normalisation of the numerical-issues subsection (eta^{-1/2} from an eigendecomposition, eigenvalues
        below eps_eta * max dropped).  Directions: the split of z = Q tilde-F^{-1} r, each column made
        admissible by Q."""
        o = self.o
        lam = self.lambda0()
        r = self.Qt(o.d() - o.F(lam))
        r0 = np.linalg.norm(r)
        hist = [1.0]
        Ws, Ps = [], []
        Wt = self.Q(self.split(self.Q(self.M(r)), groups, k))
        it = 0
        while hist[-1] > tol and it < max_it:
            for Wi, Pi in zip(Ws, Ps):
                Wt = Wt - Wi @ (Pi.T @ Wt)
            # Wt is already admissible in exact arithmetic; near the attainable residual the subtraction above
            # cancels almost everything and leaves the earlier directions' rounding in range(G), which the
            # F-normalisation would magnify, so Q is applied once more
            Wt = self.Q(Wt)
            Pt = self.Qt(o.F(Wt))
            eta = Wt.T @ Pt
            eta = 0.5 * (eta + eta.T)
            ev, V = np.linalg.eigh(eta)
            keep = ev > eps_eta * max(ev.max(), 0.0)
            if not np.any(keep):
                break
            T = V[:, keep] / np.sqrt(ev[keep])[None, :]
            Wt, Pt = Wt @ T, Pt @ T
            alpha = Wt.T @ r
            lam = lam + Wt @ alpha
            r = r - Pt @ alpha
            Ws.append(Wt); Ps.append(Pt)
            it += 1
            hist.append(np.linalg.norm(r) / r0)
            Wt = self.Q(self.split(self.Q(self.M(r)), groups, k))
        return lam, it, np.array(hist)
