"""The permutation multivector of Section 3.1 (Eq. 8) for a truly periodic structure: the block of search
directions is made of the interface vector and its images under the rotation of the structure by one, two, ...
occurrences, z -> [z, Pi z, Pi^2 z, ..., Pi^(n-1) z], Pi being the permutation of the interface partitions (with
the orientation signs of the multiplier rows).  The rest is the multivector FETI of Table 1 (right) as in
FetiOracle.multivector.  Plain FP64 numpy/scipy; test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .feti import FetiOracle


class PermutationFeti(FetiOracle):
    """Pi: the n_lambda x n_lambda map of interface vectors under the rotation of the structure by one
    occurrence (a signed permutation of the rows, with the rotation of vector components; the map a periodic
    structure's user supplies)."""

    def __init__(self, prob, Pi, n_images=None):
        super().__init__(prob)
        self.Pi = sp.csr_matrix(Pi)
        self.n_images = prob.n_occ if n_images is None else n_images

    def split(self, z, groups=None, k=None):
        """[z, Pi z, ..., Pi^(m-1) z] with m = n_images (Eq. 8: the permuted interface partitions)."""
        cols = [np.asarray(z, dtype=float)]
        for _ in range(self.n_images - 1):
            cols.append(self.Pi @ cols[-1])
        return np.stack(cols, axis=1)


class PreconditionedPermutationFeti:
    """The permutation multivector with a preconditioner of Eqs. 4-5 (the setting of the paper's donut
    assessments, which use the Dirichlet one): PreconditionedFeti's operators and loop, the split replaced by
    [z, Pi z, ..., Pi^(m-1) z] with z = Q tilde-F^{-1} r."""

    def __new__(cls, prob, Pi, kind="dirichlet", scaling="stiffness", n_images=None):
        from .precond import PreconditionedFeti
        pf = PreconditionedFeti(prob, kind, scaling)
        Pi = sp.csr_matrix(Pi)
        m = prob.n_occ if n_images is None else n_images

        def split(z, groups=None, k=None):
            cols = [np.asarray(z, dtype=float)]
            for _ in range(m - 1):
                cols.append(Pi @ cols[-1])
            return np.stack(cols, axis=1)

        pf.split = split
        pf.Pi = Pi
        return pf
