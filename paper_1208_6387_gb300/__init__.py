"""Repeated-pattern (multivector) FETI on one GB300 (sm_103a).

The compute path is libfetirp.so (hand-written CUDA, C ABI in include/fetirp.h); `fetirp` is its ctypes
binding.  Build with paper_1208_6387_gb300._build.build() (or __graft_entry__.build()).
"""
from . import fetirp  # noqa: F401
from .fetirp import *  # noqa: F401,F403
