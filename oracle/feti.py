"""FETI dual interface problem and its Krylov solvers, restated from the paper in plain FP64 numpy/scipy.
Test infrastructure only (see oracle/__init__.py).

Notation follows the paper: K(s), K(s)^+, N(s) (kernel), B(s) = A(s) t(s) (signed Boolean assembly of the
trace), F, G, d, e (Eq. 3), the projector written Q in Table 1 (called P here: P = I - G (G^T G)^{-1} G^T,
the identity preconditioner reading), lambda_0, and the multivector blocks W, P~ of Table 1 (right).
The oracle's generalized inverse fixes a statically determinate set of dofs and takes the kernel from the
mesh coordinates (constants for heat, the 6 rigid modes for elasticity); it never detects zero pivots, so it
is independent of the CUDA library's factorisation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .direct import B_matrix, rotation_blocks


def analytic_kernel(pat):
    """N(s) of a floating pattern in its own frame (Sec. 2, floating subdomains): constants for heat; the
    2 translations and the rotation for plane elasticity; the 3 translations and 3 infinitesimal rotations
    about the centroid for 3D elasticity."""
    n = pat.n_nodes
    if pat.dpn == 1:
        return np.ones((n, 1))
    x = pat.coords - pat.coords.mean(0)
    if pat.dpn == 2:   # plane elasticity: 2 translations and the in-plane rotation (-y, x) about the centroid
        N = np.zeros((n, 2, 3))
        N[:, 0, 0] = 1.0
        N[:, 1, 1] = 1.0
        N[:, 0, 2], N[:, 1, 2] = -x[:, 1], x[:, 0]
        return N.reshape(n * 2, 3)
    N = np.zeros((n, 3, 6))
    for c in range(3):
        N[:, c, c] = 1.0
    # rotation about z: (-y, x, 0); about x: (0, -z, y); about y: (z, 0, -x)
    N[:, 0, 3], N[:, 1, 3] = -x[:, 1], x[:, 0]
    N[:, 1, 4], N[:, 2, 4] = -x[:, 2], x[:, 1]
    N[:, 0, 5], N[:, 2, 5] = x[:, 2], -x[:, 0]
    return N.reshape(n * 3, 6)


def fixed_dofs(pat):
    """Dofs whose removal leaves a nonsingular stiffness: one node for heat; for plane elasticity both
    components of node 0 and the y component of node m (the far end of the first grid line); the 3-2-1 set on
    three corner nodes (0,0,0), (H,0,0), (0,H,0) for 3D elasticity."""
    if pat.dpn == 1:
        return np.array([0])
    if pat.dpn == 2:   # both components of node 0, the y component of node m (first grid line, x differs)
        return np.array([0, 1, 2 * pat.m + 1])
    m1 = pat.m + 1
    a, b, c = 0, pat.m, pat.m * m1
    return np.array([3 * a, 3 * a + 1, 3 * a + 2, 3 * b + 1, 3 * b + 2, 3 * c + 2])


class PatternInverse:
    """A generalized inverse K^+ of the floating pattern stiffness with K K^+ y = y for y in range(K)
    (Sec. 2): K^+ = [K_ff^{-1} 0; 0 0] over the free/fixed split of `fixed_dofs`."""

    def __init__(self, pat):
        self.pat = pat
        n = pat.n_dofs
        self.fixed = fixed_dofs(pat)
        self.free = np.setdiff1d(np.arange(n), self.fixed)
        self.lu = spla.splu(pat.K[self.free][:, self.free].tocsc())
        self.N = analytic_kernel(pat)
        bd = (pat.bnd_nodes[:, None].astype(np.int64) * pat.dpn + np.arange(pat.dpn)[None, :]).ravel()
        self.bnd_dofs = bd
        self._Sp = None

    def solve(self, Y):
        Y = np.asarray(Y, dtype=float)
        one = Y.ndim == 1
        Y2 = Y[:, None] if one else Y
        X = np.zeros_like(Y2)
        X[self.free] = self.lu.solve(np.ascontiguousarray(Y2[self.free]))
        return X[:, 0] if one else X

    def schur_pinv(self):
        """S^+ = t K^+ t^T, the boundary block of K^+ (the identity stated after Eq. 3)."""
        if self._Sp is None:
            n, nb = self.pat.n_dofs, len(self.bnd_dofs)
            E = np.zeros((n, nb))
            E[self.bnd_dofs, np.arange(nb)] = 1.0
            self._Sp = self.solve(E)[self.bnd_dofs]
        return self._Sp


class FetiOracle:
    """The dual interface problem (Eq. 3) of a Problem from fetirp_gen, in the global frame."""

    def __init__(self, prob, use_schur=True):
        self.prob = prob
        self.inv = [PatternInverse(p) for p in prob.patterns]
        self.B, self.offs = B_matrix(prob)
        self.Bs = [self.B[:, self.offs[o]:self.offs[o + 1]].tocsr() for o in range(prob.n_occ)]
        self.Rh = [rotation_blocks(prob, o) for o in range(prob.n_occ)]
        self.use_schur = use_schur
        # G = [ ... B(s) N(s) ... ] (Eq. 3), N(s) = R-hat N_pattern in the global frame
        self.Ns = [self.Rh[o] @ self.inv[prob.occs[o].pattern].N for o in range(prob.n_occ)]
        self.G = np.hstack([self.Bs[o] @ self.Ns[o] for o in range(prob.n_occ)])
        self.nz = [N.shape[1] for N in self.Ns]
        self.GtG = self.G.T @ self.G
        self.GtG_inv = np.linalg.inv(self.GtG)
        # multiplicity scaling Delta(s) (the diagonal scaling of Eqs. 4-5, sum_s Delta(s) = I) restricted to lambda rows
        inc = np.zeros((prob.n_lambda, prob.n_occ))
        for o, occ in enumerate(prob.occs):
            inc[occ.link_lambda_row, o] = 1.0
        self.incidence = inc
        self.Delta = inc / inc.sum(1, keepdims=True)

    # ---- local operators -------------------------------------------------------------------------
    def kplus(self, o, Y):
        """K(s)^+ Y in the global frame: R-hat K_pattern^+ R-hat^T Y."""
        inv = self.inv[self.prob.occs[o].pattern]
        return self.Rh[o] @ inv.solve(self.Rh[o].T @ Y)

    def F(self, V):
        """F V = sum_s B(s) K(s)^+ B(s)^T V (Eq. 3); with use_schur the local product is taken through
        the boundary block S^+ = t K^+ t^T (same value, the identity after Eq. 3)."""
        V = np.asarray(V, dtype=float)
        one = V.ndim == 1
        V2 = V[:, None] if one else V
        out = np.zeros_like(V2)
        for o in range(self.prob.n_occ):
            Bs = self.Bs[o]
            Y = Bs.T @ V2
            if self.use_schur:
                inv = self.inv[self.prob.occs[o].pattern]
                bd = inv.bnd_dofs
                Rb = self.Rh[o][bd][:, bd]
                X = np.zeros_like(Y)
                X[bd] = Rb @ (inv.schur_pinv() @ (Rb.T @ Y[bd]))
            else:
                X = self.kplus(o, Y)
            out += Bs @ X
        return out[:, 0] if one else out

    def d(self):
        """d = sum_s B(s) K(s)^+ f(s) - c (Eq. 3, with the total-FETI right-hand side B u = c)."""
        out = -self.prob.c.copy()
        for o in range(self.prob.n_occ):
            out += self.Bs[o] @ self.kplus(o, self.prob.occs[o].f_global)
        return out

    def e(self):
        """e^T = ( ... f(s)^T N(s) ... ) (Eq. 3)."""
        return np.concatenate([self.Ns[o].T @ self.prob.occs[o].f_global for o in range(self.prob.n_occ)])

    # ---- coarse problem (projector paragraph, identity preconditioner) ------------------------------
    def project(self, V):
        """P V = V - G (G^T G)^{-1} G^T V; P is symmetric, so P^T = P."""
        return V - self.G @ (self.GtG_inv @ (self.G.T @ V))

    def lambda0(self):
        """lambda_0 = G (G^T G)^{-1} e (the initialisation of Table 1 with lambda_00 = 0)."""
        return self.G @ (self.GtG_inv @ self.e())

    def PtFP(self, V):
        """The block interface operator P^T F P V applied to a block of directions."""
        return self.project(self.F(self.project(V)))

    # ---- Krylov solvers (Table 1) ---------------------------------------------------------------
    def classical_cg(self, tol=1e-8, max_it=10000):
        """Classical FETI (Table 1, left column) with the identity preconditioner."""
        d = self.d()
        lam = self.lambda0()
        r = self.project(d - self.F(lam))
        r0 = np.linalg.norm(r)
        hist = [1.0]
        z = self.project(r)
        w = z.copy()
        it = 0
        while hist[-1] > tol and it < max_it:
            p = self.project(self.F(w))
            wp = w @ p
            alpha = (w @ r) / wp
            lam = lam + alpha * w
            r = r - alpha * p
            z = self.project(r)
            beta = -(p @ z) / wp
            w = z + beta * w
            it += 1
            hist.append(np.linalg.norm(r) / r0)
        return lam, it, np.array(hist)

    def split(self, z, groups=None, k=None):
        """Multivector from one interface vector: column g = sum over occurrences c of group g of
        Delta(c) z (the occurrence split; the columns sum to z)."""
        groups = self.prob.groups if groups is None else groups
        k = self.prob.k if k is None else k
        onehot = np.zeros((self.prob.n_occ, k))
        onehot[np.arange(self.prob.n_occ), groups] = 1.0
        return (self.Delta * z[:, None]) @ onehot

    def multivector(self, tol=1e-8, max_it=1000, eps_eta=1e-12, groups=None, k=None, reorth_depth=None):
        """Multivector FETI (Table 1, right column) with full reorthogonalisation and F-normalisation
        (numerical-issues subsection): eta = W^T P~ is replaced by I through W <- W eta^{-1/2},
        reorth_depth = number of previous blocks orthogonalised against (None = all; 1 = the short recurrence
        of Table 1, where beta = -(W^T P~)^{-1} P~^T Z = -P~^T Z after normalisation);
        P~ <- P~ eta^{-1/2}, eta^{-1/2} taken from a symmetric eigendecomposition in which eigenvalues below
        eps_eta * max are dropped (the pseudo-inverse that handles redundant directions)."""
        d = self.d()
        lam = self.lambda0()
        r = self.project(d - self.F(lam))
        r0 = np.linalg.norm(r)
        hist = [1.0]
        Ws, Ps = [], []
        Wt = self.project(self.split(self.project(r), groups, k))
        it = 0
        while hist[-1] > tol and it < max_it:
            hist_blocks = list(zip(Ws, Ps)) if reorth_depth is None else list(zip(Ws, Ps))[-reorth_depth:]
            for Wi, Pi in hist_blocks:       # (full) reorthogonalisation against previous blocks
                Wt = Wt - Wi @ (Pi.T @ Wt)
            Pt = self.project(self.F(Wt))    # F-image of the directions (Table 1)
            eta = Wt.T @ Pt
            eta = 0.5 * (eta + eta.T)
            ev, V = np.linalg.eigh(eta)
            keep = ev > eps_eta * max(ev.max(), 0.0)
            if not np.any(keep):
                break
            T = V[:, keep] / np.sqrt(ev[keep])[None, :]
            Wt, Pt = Wt @ T, Pt @ T
            alpha = Wt.T @ r                  # step length, with W^T P~ = I
            lam = lam + Wt @ alpha            # iterate update
            r = r - Pt @ alpha                # residual update
            Ws.append(Wt); Ps.append(Pt)
            it += 1
            hist.append(np.linalg.norm(r) / r0)
            Wt = self.project(self.split(self.project(r), groups, k))   # new directions from the residual, split
        return lam, it, np.array(hist)

    # ---- recovery -------------------------------------------------------------------------------
    def recover(self, lam):
        """alpha from the first row of Eq. 3 (F lam + G alpha = d, projected on range(G)) and
        u(s) = K(s)^+ (f(s) - B(s)^T lam) - N(s) alpha(s) (Eq. 2 with the kernel term)."""
        alpha = self.GtG_inv @ (self.G.T @ (self.d() - self.F(lam)))
        us, off = [], 0
        for o in range(self.prob.n_occ):
            a = alpha[off:off + self.nz[o]]
            off += self.nz[o]
            us.append(self.kplus(o, self.prob.occs[o].f_global - self.Bs[o].T @ lam) - self.Ns[o] @ a)
        return alpha, us

    def dense_F(self):
        return self.F(np.eye(self.prob.n_lambda))
