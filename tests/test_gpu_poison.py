"""Reads of device memory the library never wrote.  With FETIRP_POISON=1 every new device allocation of the
library is filled with NaN bytes, so such a read turns the solution into NaN (fresh driver memory is usually
zero, which would hide it).  Both iteration paths, both local-product precisions, heat (one kernel mode) and
elasticity (six modes), must still reproduce the direct solve."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
import paper_1208_6387_gb300.fetirp as F
from fetirp_gen import config, heat_grid, elastic_grid
from oracle.direct import direct
cases = [heat_grid(5, (3, 2), kappas=(1.0, 30.0), checker=True, rotate=True, k=4, seed=7),
         elastic_grid(3, (2, 2, 1), n_patterns=2, k=4, seed=1), config("c1")]
worst = 0.0
for prob in cases:
    _, lam_ref, _, _ = direct(prob)
    for prec in ("fp64", "fp32"):
        for pers in (1, 0):
            ctx = F.fetirp_create(F.fetirp_default_options(precision=prec, tol=1e-12, inner_tol=1e-5,
                                                           persistent=pers))
            F.load_problem(ctx, prob)
            lam, u, st = F.fetirp_solve(ctx, prob.n_lambda, prob.c, F.n_u(prob))
            F.fetirp_destroy(ctx)
            err = np.linalg.norm(lam - lam_ref) / np.linalg.norm(lam_ref)
            assert np.isfinite(err) and err < 1e-8, (prob.name, prec, pers, err, st)
            worst = max(worst, err)
print("worst", worst)
"""


def test_poisoned_allocations_do_not_reach_results():
    env = dict(os.environ, FETIRP_POISON="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
