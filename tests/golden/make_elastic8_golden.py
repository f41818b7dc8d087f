"""Writes elastic8_3x4x4.npz: the oracle's direct solution (oracle.direct: global assembly, sparse LU of Eq. 1,
lambda from the subdomain equilibria of Eq. 2) of the medium elastic structure used by tests/test_gpu_medium.py
(three 8^3 Q1 cube patterns on a 3 x 4 x 4 grid of rotated occurrences, 16 per pattern, k = 30, clamped x = 0,
N(0,1) loads, seed 3).  The direct solve takes minutes on the host, so its result is stored; the file also holds
the sizes and a checksum of the inputs, which the test compares with the generator's current output.

    python tests/golden/make_elastic8_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from fetirp_gen import elastic_grid  # noqa: E402
from oracle.direct import direct  # noqa: E402


def medium_problem():
    return elastic_grid(8, (3, 4, 4), n_patterns=3, k=30, seed=3)


def input_checksum(prob):
    f = np.concatenate([o.f_global for o in prob.occs])
    rows = np.concatenate([o.link_lambda_row for o in prob.occs]).astype(np.float64)
    return np.array([prob.n_lambda, prob.n_occ, f.sum(), (f * f).sum(), rows.sum(), prob.c.sum()])


def main():
    prob = medium_problem()
    us, lam, res, _ = direct(prob)
    assert res < 1e-10, res
    np.savez_compressed(os.path.join(HERE, "elastic8_3x4x4.npz"), lam=lam, u=np.concatenate(us),
                        checksum=input_checksum(prob))
    print("n_lambda", prob.n_lambda, "consistency residual", res)


if __name__ == "__main__":
    main()
