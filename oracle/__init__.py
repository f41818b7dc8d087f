"""CPU FP64 oracle for repeated-pattern FETI (Gosselet, Rixen & Rey, arXiv 1208.6387).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this package: only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline leg (and its `--impl reference` arm) use it.  It shares no
code with the CUDA library; both read the seeded inputs made by fetirp_gen.

Contents
  direct  -- the plain definition: global assembly and direct solve of K u = f (Eq. 1), interface reactions
             lambda from the local equilibria (Eq. 2).
  feti    -- the dual interface problem (Eq. 3) built from the definitions of F, G, d, e with the oracle's own
             generalized inverse (fixed dofs + analytic kernel), the coarse projector and lambda_0 (Sec. 2,
             projector paragraph), classical FETI-CG (Table 1, left) and multivector FETI (Table 1, right) with
             full reorthogonalisation and F-normalisation (Sec. 3.3), and the block operator P^T F P V.
  brute   -- brute force for tiny meshes: Moore-Penrose pseudo-inverses and a dense solve of Eq. 3.
  precond -- the Dirichlet, lumped and superlumped preconditioners (Eqs. 4-5) with multiplicity or stiffness
             scaling, the preconditioner-weighted projector and lambda_0, and Table 1 with a preconditioner.

Parity pins live in tests/test_oracle_*.py.  Parity against the paper's printed numbers (Tables 2-4) is
unpinned: the donut meshes they were measured on are not available, so only trends can be compared.
"""
