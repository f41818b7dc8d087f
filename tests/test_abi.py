"""The C ABI: every function declared in include/fetirp.h is exported by libfetirp.so and bound by the
Python binding; the library loads without a GPU.  No compute calls (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "fetirp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fetirp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1208_6387_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = declared()
    for must in ("fetirp_create", "fetirp_create_pattern", "fetirp_add_occurrence", "fetirp_solve",
                 "fetirp_apply_block", "fetirp_destroy", "fetirp_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fetirp_[a-z_0-9]+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol(libpath):
    import paper_1208_6387_gb300.fetirp as F
    L = F.lib()
    for n in declared():
        assert hasattr(L, n)
        assert n in F._SIGS, f"binding has no signature for {n}"
        assert hasattr(F, n), f"binding has no function {n}"


def test_defaults_and_status_strings(libpath):
    import paper_1208_6387_gb300.fetirp as F
    o = F.fetirp_default_options()
    assert o.tol == 1e-8 and o.block_k == 32 and o.precision == F.FETIRP_PREC_FP64
    assert o.inner_tol == 0.0   # per-precision inner tolerance
    assert F.lib().fetirp_status_string(4) == b"FETIRP_ENOCONV"


def test_create_without_gpu_fails_loudly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1208_6387_gb300.fetirp as F
    with pytest.raises(F.FetirpError):
        F.fetirp_create()
