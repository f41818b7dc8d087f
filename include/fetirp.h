/*
 * fetirp.h -- repeated-pattern FETI on one GB300 (sm_103a): C ABI.
 *
 * Method: Gosselet, Rixen & Rey, "A domain decomposition strategy to efficiently solve structures
 * containing repeated patterns" (arXiv 1208.6387).  A structure is a set of occurrences of a few meshed
 * patterns.  Each occurrence s carries its pattern's stiffness K(s) in the pattern frame, a rigid rotation
 * and a signed Boolean assembly B(s) = A(s) t(s) (Eq. 2).  The library solves the dual interface problem
 *     [F G; G^T 0] [lambda; alpha] = [d; e],   F = sum_s B(s) K(s)^+ B(s)^T   (Eq. 3)
 * with multivector (block) FETI (Table 1, right column; full reorthogonalisation and F-normalisation of
 * the numerical-issues subsection), every occurrence of a pattern sharing that pattern's one factorisation
 * (the multi-right-hand-side product of the efficient-implementation subsection).  Dirichlet data enter
 * as total-FETI multiplier rows (Dirichlet-conditions subsection), so every occurrence is floating.
 *
 * Conventions shared by every entry point
 *  - Status: every call returns a fetirp_status and never throws; on error fetirp_last_error(ctx) holds
 *    a message owned by the context, and no output buffer has been written.
 *  - Ownership: every input array is copied (to host and device memory owned by the context) before the
 *    call returns; the caller may free or reuse it.  Outputs go to caller-allocated buffers whose sizes
 *    follow from the arguments.  "_device" entry points take device pointers allocated by the caller and
 *    run on the context's stream; they return once the work is enqueued unless stated otherwise.
 *  - Threading: a context is used by one host thread at a time.
 *  - Indices are 0-based.  dof = node * dofs_per_node + component.
 *  - Sizes that overflow int32 where an int32 is taken, negative sizes, NULL required pointers, non-finite
 *    values, or indices out of range return FETIRP_EINVAL.
 */
#ifndef FETIRP_H
#define FETIRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fetirp_ctx_s* fetirp_ctx;

typedef enum {
  FETIRP_OK = 0,
  FETIRP_EINVAL = 1,     /* bad argument */
  FETIRP_ENOMEM = 2,     /* device or host allocation failed */
  FETIRP_ESINGULAR = 3,  /* detected kernel dimension differs from the expected one, or G^T G singular */
  FETIRP_ENOCONV = 4,    /* tolerance not reached within the iteration caps (outputs hold the last iterate) */
  FETIRP_ECUDA = 5,      /* a CUDA call failed */
  FETIRP_ESTATE = 6,     /* call out of order (e.g. solve before any occurrence) */
  FETIRP_ETIMEOUT = 7    /* a bounded device-side wait gave up */
} fetirp_status;

/* Arithmetic of the local multi-right-hand-side products S^+ Y (the hot contraction). */
enum {
  FETIRP_PREC_FP64 = 0, /* plain FP64 form */
  FETIRP_PREC_FP32 = 1, /* FP32 products wrapped in FP64 outer refinement (defect correction) */
  FETIRP_PREC_TF32X3 = 2, /* tensor cores (tcgen05 kind::tf32), operands split hi+lo, 3 products, FP32
                             accumulation in TMEM; wrapped in FP64 outer refinement */
  FETIRP_PREC_AUTO = 3,   /* solves only (fetirp_options.precision): per structure, FP32 for latency-bound ones
                             (every used pattern with n_b <= 512 and n_lambda <= 262144, which then run the
                             persistent iteration), TF32X3 otherwise; both inside the FP64 refinement */
  FETIRP_PREC_BF16X3 = 4  /* tensor cores (tcgen05 kind::f16 with bf16 operands, twice the tf32 rate), operands
                             split into bf16 pairs (16 significant bits), 3 products, FP32 accumulation in TMEM;
                             operator accurate to ~1e-5 relative; wrapped in FP64 outer refinement.  Rotations of
                             vector fields in 90-degree steps only; not taken by fetirp_apply_split or
                             fetirp_apply_block_device_noalloc */
};

typedef struct {
  int32_t precision;   /* FETIRP_PREC_* of the solves, default FP64 */
  double tol;          /* target ||r_j|| / ||r_0||, r = P^T (d - F lambda) (the residual of Table 1); default 1e-8 */
  int32_t max_iter;    /* cap on block iterations over the whole solve; default 2000 */
  int32_t block_k;     /* multivector width k; 1 = classical FETI-CG; default 32 (clamped to the number
                          of occurrences; fetirp_set_groups overrides) */
  int32_t max_outer;   /* cap on FP64 refinement steps of the mixed forms; default 30 */
  double inner_tol;    /* relative tolerance of each inner (low-precision) solve; 0 (the default) = 1e-6 with FP32
                          local products, 1e-5 with TF32X3 and 1e-4 with BF16X3, each above the operator's
                          accuracy (a tighter inner target only adds stagnating iterations) */
  double pivot_tol;    /* zero pivot when pivot <= pivot_tol * original diagonal; default 1e-9 */
  double eig_trunc;    /* a direction is dropped when its normalisation pivot <= eig_trunc * largest;
                          default 1e-12 */
  void* cuda_stream;   /* cudaStream_t used for all device work; NULL = a stream created and owned by the
                          context (the legacy default stream cannot be captured into CUDA graphs) */
  int32_t device;      /* CUDA device ordinal; default 0 */
  int32_t check_every; /* block iterations per convergence read-back (and per captured graph); default 4 */
  int32_t timing;      /* 1: bracket every phase with CUDA events and fill the phase_* statistics; default 0 */
  double eig_trunc_inner; /* truncation threshold of the low-precision inner solves of the mixed forms, where
                             the operator is only accurate to ~1e-7; default 1e-6 */
  int32_t use_graphs;  /* 1: the check_every iterations between read-backs are captured once as a CUDA graph
                          and replayed; 0: launched one by one; default 1 */
  int32_t timing_mask; /* with timing = 1: bit p set -> phase p is bracketed with events; 0 = every phase */
  int64_t history_bytes; /* cap on the two direction-history arrays (a full history restarts the recurrence);
                            0 = half of the free device memory */
  int32_t persistent;  /* 1: structures small enough to be latency-bound (n_lambda <= 262144, k <= 32, FP64 or
                          FP32 local products) run whole block iterations in one cooperative persistent
                          launch with bounded grid barriers, stopping on the device at convergence; 0: CUDA
                          graphs of per-phase kernels; default 1 */
  /* Caller-supplied device allocator (for example a framework's caching allocator); both NULL (the default)
     = cudaMalloc / cudaFree.  Set both or neither.  alloc(bytes, stream, alloc_user) returns device memory
     on options.device, 256-byte aligned, usable on `stream` (the context's stream), or NULL (the call then
     returns FETIRP_ENOMEM); free(ptr, alloc_user) releases one pointer that alloc returned, after the library
     has synchronised the device.  The library calls them from the host thread of the call (server calls:
     from its worker threads), only while one of its entry points runs or the context (or a context sharing
     its patterns) is destroyed; they must stay valid until then. */
  void* (*alloc)(size_t bytes, void* stream, void* alloc_user);
  void (*free)(void* ptr, void* alloc_user);
  void* alloc_user;
} fetirp_options;

/* Phases of a solve, for the per-phase statistics. */
enum {
  FETIRP_PHASE_FACTOR = 0,   /* pattern factorisation (fetirp_factorize / fetirp_create_pattern) */
  FETIRP_PHASE_COARSE = 1,   /* G^T G, its inverse, e, lambda_0, d */
  FETIRP_PHASE_LOCAL = 2,    /* local multi-RHS products S^+ Y (the hot contraction) */
  FETIRP_PHASE_GATHER = 3,   /* signed gather B(s)^T V into pattern-frame traces */
  FETIRP_PHASE_SCATTER = 4,  /* signed scatter-add of the local solutions */
  FETIRP_PHASE_PROJECT = 5,  /* projector P = I - G (G^T G)^{-1} G^T */
  FETIRP_PHASE_GRAM = 6,     /* block Gram products (reorthogonalisation coefficients, eta, W^T r) */
  FETIRP_PHASE_REORTH = 7,   /* W -= W_hist C */
  FETIRP_PHASE_UPDATE = 8,   /* split of r, W T, P~ T, lambda and residual updates, norms */
  FETIRP_PHASE_RECOVER = 9,  /* alpha and u(s) */
  FETIRP_PHASE_NORMALISE = 10, /* F-normalisation of eta (pivoted Cholesky, one CTA) */
  FETIRP_PHASE_ITERATE = 11,   /* whole block iterations in one persistent launch (options.persistent) */
  FETIRP_PHASE_OUTER = 12,     /* FP64 residual evaluations r = P^T (d - F lambda) (initial residual and every
                                  outer refinement step; their F-apply is not booked under local/gather/scatter) */
  FETIRP_NPHASE = 13
};

typedef struct {
  int32_t iterations;         /* block iterations (all outer steps) */
  int32_t outer_steps;        /* FP64 residual evaluations after the first (0 for the plain FP64 form) */
  int32_t f_applies;          /* block F-applies P^T F P W */
  int32_t dropped_directions; /* directions removed by the normalisation (redundant information) */
  int32_t kernel_dim_total;   /* columns of G */
  double rel_residual;        /* final ||P^T (d - F lambda)|| / ||r_0|| evaluated in FP64 */
  double setup_ms;            /* host wall time of the structure set-up (tables, coarse problem, d, lambda_0) */
  double solve_ms;            /* device time of iterations + recovery (CUDA events on the context stream) */
  int64_t launches;           /* kernels launched by the call */
  /* with options.timing = 1: per phase (FETIRP_PHASE_*) device time, launches, and the algorithmic work
     counted from the sizes (flops and compulsory bytes, not hardware counters) */
  double phase_ms[FETIRP_NPHASE];
  int64_t phase_launches[FETIRP_NPHASE];
  double phase_flops[FETIRP_NPHASE];
  double phase_bytes[FETIRP_NPHASE];
} fetirp_stats;

/* Test hook of the bounded device waits (the method has no counterpart): the next solve that uses the
 * persistent iteration launches it with a grid barrier that waits for one CTA more than the grid has and a
 * 0.2 s limit, so every wait expires; the solve returns FETIRP_ETIMEOUT and the context stays usable (the
 * following solve runs normally).  Nothing faults or hangs: each CTA stops waiting at the limit and returns. */
fetirp_status fetirp_inject_barrier_stall(fetirp_ctx ctx);

/* Fill *opt with the defaults listed above. */
void fetirp_default_options(fetirp_options* opt);

/* Human-readable name of a status code (static storage). */
const char* fetirp_status_string(fetirp_status s);

/* Create a context on opt->device (opt may be NULL for defaults).  *out receives the handle. */
fetirp_status fetirp_create(const fetirp_options* opt, fetirp_ctx* out);

/*
 * A context that shares the patterns (factors) of `parent` read-only, with its own stream, occurrences and
 * work buffers (opt NULL: the parent's options).  Patterns added to the parent later are not seen.  Several
 * children may solve different structures concurrently from different host threads; the parent must outlive
 * its children and must not be refactorised while they run.  fetirp_create_pattern and fetirp_factorize on a
 * child return FETIRP_ESTATE.  (Serving pattern: a library of resident factors, one child per request slot.)
 */
fetirp_status fetirp_create_child(fetirp_ctx parent, const fetirp_options* opt, fetirp_ctx* out);

/* Message of the last failed call on ctx (owned by ctx, valid until the next call); "" if none. */
const char* fetirp_last_error(fetirp_ctx ctx);

/* Release every host and device resource of ctx.  NULL is a no-op. */
void fetirp_destroy(fetirp_ctx ctx);

/*
 * Register a pattern and factorise it on the device in FP64 (Sec. 2: K(s)^+ with K K^+ y = y on range(K),
 * kernel N; Schur complement S = K_bb - K_bi K_ii^{-1} K_ib and S^+ = t K^+ t^T, stated after Eq. 3).
 *  n_nodes, dofs_per_node: mesh size; dofs_per_node is 1 (heat) or 2..3 (elasticity).
 *  rowptr[n+1], col[nnz], val[nnz]: the FULL symmetric CSR of the free (unconstrained) pattern stiffness,
 *     n = n_nodes * dofs_per_node, pattern frame.  Symmetry is assumed, not checked.
 *  n_bnd, bnd_nodes[n_bnd]: the trace t: distinct nodes that may carry multipliers.  Their dofs are
 *     ordered last (boundary-last), in the order given, so the trailing factor block is chol(S).
 *  expected_kernel_dim: -1 to accept the detected kernel dimension; otherwise FETIRP_ESINGULAR when the
 *     number of zero pivots differs.
 *  *pattern_id receives the id (0, 1, ...).
 * Device memory: a dense FP64 factor of (n rounded up to 64)^2 doubles, L_S^{-1} and S^+ in FP64, S^dag in FP32
 * and as tf32 and bf16 pairs.  Patterns with n_b >= 1024 form the bf16 pair of S^dag on the tensor cores and
 * compute S^+ and the FP32 and tf32 forms of S^dag only on the first call that needs them (a solve, an apply
 * or fetirp_get_pattern in FP64, FP32 or TF32X3; that call waits for them): a BF16X3 solve needs none of them
 * and applies S^+ in its FP64 refinement through L_S^{-1}.
 */
fetirp_status fetirp_create_pattern(fetirp_ctx ctx, int32_t n_nodes, int32_t dofs_per_node,
                                    const int64_t* rowptr, const int32_t* col, const double* val,
                                    int32_t n_bnd, const int32_t* bnd_nodes, int32_t expected_kernel_dim,
                                    int32_t* pattern_id);

/*
 * Add an occurrence of a pattern (Eq. 2 with the rotation of the elasticity subsection).
 *  rot[9]: row-major R with global = R * local, or NULL for the identity.  R must be a proper rotation:
 *     finite, R R^T = I and det R = +1, both to 1e-12 (FETIRP_EINVAL otherwise).  With one dof per node the
 *     field has no components to turn, so the rotation is not used.  With two dofs per node R may not couple
 *     z with x or y (entries above 1e-12 there: FETIRP_EINVAL).  Vector fields: a signed permutation (the
 *     rotations of the cube, of the square) is folded into the links, so the hot path stays a signed
 *     gather/scatter; any other rotation keeps the links in the global frame and the gathered traces are turned
 *     into the pattern frame node by node (R^T) on the device, and the local solutions back (R), before the
 *     scatter.  Such occurrences use the per-phase iteration and are not accepted by fetirp_apply_split.
 *  n_links and the four link arrays: the rows of B(s) in the GLOBAL frame: entry sign[i] (+1 or -1) in
 *     multiplier row lambda_row[i] on component global_comp[i] of pattern node local_node[i], which must
 *     be one of the pattern's boundary nodes.  Every multiplier row must end up with one or two entries in
 *     total over all occurrences (a Dirichlet row or a pairwise gluing row).
 *  f_global[n_nodes * dofs_per_node]: the occurrence's load, pattern node order, global-frame components.
 *  *occ_id receives the occurrence id (0, 1, ... in call order).
 */
fetirp_status fetirp_add_occurrence(fetirp_ctx ctx, int32_t pattern_id, const double* rot, int32_t n_links,
                                    const int32_t* local_node, const int8_t* global_comp,
                                    const int32_t* lambda_row, const int8_t* sign, const double* f_global,
                                    int32_t* occ_id);

/* Remove every occurrence (and the multivector groups) so that the context can take the next structure;
 * patterns and device buffers are kept, so a reused context does not allocate again for a structure of
 * the same size or smaller. */
fetirp_status fetirp_clear_occurrences(fetirp_ctx ctx);

/*
 * Multivector columns (the block of search directions of Table 1, right): occurrence s contributes its
 * share Delta(s) z of the preconditioned residual z to column group_of_occ[s] in [0, k), where
 * Delta(s) = 1/(number of occurrences in the row) on the multiplier rows s appears in (sum_s Delta(s) = I).
 * Without this call the occurrences are split into min(block_k, n_occ) contiguous groups by id.
 */
fetirp_status fetirp_set_groups(fetirp_ctx ctx, int32_t k, const int32_t* group_of_occ);

/*
 * The permutation multivector of Section 3.1 (Eq. 8) for a periodic structure: the block of search directions
 * built from the residual z is [z, Pi z, Pi^2 z, ..., Pi^(n_images-1) z] instead of the occurrence split, Pi
 * being the map of interface vectors under the rotation of the structure by one occurrence (a signed
 * permutation of the multiplier rows, with the rotation of vector components by the structure's rotation).
 *  n_lambda, rowptr[n_lambda + 1], col[nnz], val[nnz]: Pi as a CSR matrix (row i of Pi z = sum val z[col]).
 *     Every power Pi^g (g < n_images) may have at most 8 entries per row (FETIRP_EINVAL otherwise).
 *     rowptr = NULL switches back to the occurrence split.
 *  n_images: the block width k, 1..64 (n_images = number of occurrences for a ring of them).
 *  shortcut: 1 = the periodic shortcut of Table 1 (right): since F commutes with Pi on such a structure, the
 *     F-image of the block is [p, Pi p, ...] with one single-column F-apply p = P^T F P z, and the image of the
 *     reorthogonalised block follows by the same linear combination of the stored images (no F-apply of k
 *     columns).  The next fetirp_prepare / fetirp_solve checks P^T F P Pi v = Pi P^T F P v on a seeded vector in
 *     FP64 (relative 1e-9) and returns FETIRP_EINVAL when the structure is not periodic under Pi.
 *     0 = the F-apply of the whole block, as for any multivector.
 * The setting stays until fetirp_set_groups, fetirp_clear_occurrences or a call with rowptr = NULL.  Solves
 * with a permutation use the per-phase iteration (CUDA graphs), not the persistent kernel.  fetirp_apply_split
 * needs the occurrence split and returns FETIRP_EINVAL meanwhile.  Every input is copied.
 */
fetirp_status fetirp_set_permutation(fetirp_ctx ctx, int64_t n_lambda, const int64_t* rowptr, const int32_t* col,
                                     const double* val, int32_t n_images, int32_t shortcut);

/* Preconditioners of Eqs. 4-5 and their scaling (fetirp_set_preconditioner). */
enum {
  FETIRP_PRECOND_NONE = 0,        /* identity (the default): P = I - G (G^T G)^{-1} G^T */
  FETIRP_PRECOND_DIRICHLET = 1,   /* X(s) = S(s) = K_bb - K_bi K_ii^{-1} K_ib, the primal Schur complement */
  FETIRP_PRECOND_LUMPED = 2,      /* X(s) = K_bb, the boundary block of the stiffness */
  FETIRP_PRECOND_SUPERLUMPED = 3  /* X(s) = diag(K_bb) */
};
enum {
  FETIRP_SCALING_MULTIPLICITY = 0, /* Delta(s) = 1 / (occurrences sharing the row) */
  FETIRP_SCALING_STIFFNESS = 1     /* on a gluing row between s and t at dof i: Delta(s) = K(t)_ii / (K(s)_ii +
                                      K(t)_ii), the diagonals in the global frame; 1 on a Dirichlet row */
};

/*
 * The preconditioner of the solves of this context (Eqs. 4-5): tilde-F^{-1} = sum_s Delta(s) B(s) X(s) B(s)^T
 * Delta(s), with sum_s Delta(s) = I on the multiplier rows, and the projector of Eqs. 6-7 in its metric,
 * Q = I - tilde-F^{-1} G (G^T tilde-F^{-1} G)^{-1} G^T, lambda_0 = tilde-F^{-1} G (G^T tilde-F^{-1} G)^{-1} e.
 * The iteration is Table 1 (right column) with the preconditioner: the block is the split (by Delta, or the
 * permutation images of fetirp_set_permutation) of z = Q tilde-F^{-1} r, r = Q^T (d - F lambda), and the stopping
 * rule is ||r_j|| / ||r_0|| <= tol on that r.  X(s) is the pattern's operator in the pattern frame, formed at the
 * next fetirp_prepare / fetirp_solve in FP64 (Dirichlet: n_b right-hand sides through the interior block of the
 * pattern factor); tilde-F^{-1} and Q are applied in FP64 in every precision, and the direction history is kept
 * in FP64.  With the mixed forms the inner operator carries the ~1e-7 rounding of the low-precision local
 * products; on strongly heterogeneous structures (the 1 / 1000 checkerboard) that rounding of the soft
 * occurrences exceeds what the preconditioner resolves on the stiff ones and the solve does not converge
 * (FETIRP_ENOCONV): use FETIRP_PREC_FP64 there.  A preconditioned solve uses the per-phase iteration (CUDA graphs)
 * and the full F-apply of the block (no periodic shortcut).  The setting stays until changed.
 * fetirp_apply_block and fetirp_apply_split keep the unpreconditioned projector P.
 * Errors: FETIRP_EINVAL for an unknown kind or scaling; the next prepare returns FETIRP_EINVAL when stiffness
 * scaling meets a non-positive diagonal.
 */
fetirp_status fetirp_set_preconditioner(fetirp_ctx ctx, int32_t kind, int32_t scaling);

/*
 * Declare the structure a union of independent sub-structures (the batching of the serving loop): block b owns
 * the multiplier rows [row_offset[b], row_offset[b + 1]) and nothing couples the blocks.  The next solves then
 * stop when ||r|| <= tol * min_b ||r0_b|| (r restricted to block b), so that every block meets the relative
 * tolerance on its own, and fetirp_stats.rel_residual reports the worst block's ||r_b|| / ||r0_b||.  With
 * multivector groups that do not mix blocks, the block iteration of the union is the blocks' own iterations
 * carried out together (F, P and the block Gram matrices are block diagonal), so one local-product launch per
 * iteration serves every block.  n_blocks = 0 (or row_offset = NULL) removes the setting; so does
 * fetirp_clear_occurrences.  row_offset[n_blocks] must equal the n_lambda of the solve (FETIRP_EINVAL otherwise).
 */
fetirp_status fetirp_set_row_blocks(fetirp_ctx ctx, int32_t n_blocks, const int64_t* row_offset);

/*
 * Solve for lambda and the displacements (Table 1 and the recovery u(s) = K^+ (f - B^T lambda) + N alpha).
 *  n_lambda: number of multiplier rows (max lambda_row + 1 over all occurrences).
 *  c[n_lambda]: right-hand side of B u = c (Dirichlet values on Dirichlet rows, 0 on gluing rows), or NULL
 *     for zero.
 *  lambda_out[n_lambda]; u_out[sum_s n_nodes(s) * dofs_per_node]: occurrences concatenated in id order,
 *     pattern node order, global-frame components.  Host memory.
 *  stats: may be NULL.
 * Blocks until done.  FETIRP_ENOCONV still writes the last iterate.
 */
fetirp_status fetirp_solve(fetirp_ctx ctx, int64_t n_lambda, const double* c, double* lambda_out,
                           double* u_out, fetirp_stats* stats);

/*
 * Autotuner of the multivector width: for every candidate k (1..64) the structure is solved once with k
 * contiguous occurrence groups (by id) and timed with CUDA events; the fastest k is then set as the context's
 * grouping (as fetirp_set_groups would) and returned in *best_k.  times_ms[n_cand] (may be NULL) receives the
 * measured solve times (device time, FETIRP_ENOCONV solves count as +infinity).  Block iterations trade
 * against the FP64 Gram work, which grows as k^2 per stored block, so the best k depends on the structure
 * and on the precision.
 */
fetirp_status fetirp_autotune_k(fetirp_ctx ctx, int64_t n_lambda, const double* c, int32_t n_cand,
                                const int32_t* candidates, int32_t* best_k, double* times_ms);

/* As fetirp_solve with caller-allocated DEVICE buffers (c may be NULL); blocks until done. */
fetirp_status fetirp_solve_device(fetirp_ctx ctx, int64_t n_lambda, const double* d_c, double* d_lambda,
                                  double* d_u, fetirp_stats* stats);

/*
 * The block interface operator Q = P^T F P V on a block of k directions (the F-apply of Table 1), with
 * P = I - G (G^T G)^{-1} G^T.  V and Q are n_lambda x k, row-major (k contiguous), FP64, host memory.
 * precision: FETIRP_PREC_* for the local products.  Blocks until done.  Requires n_lambda to have been
 * fixed by a previous fetirp_solve or fetirp_prepare.
 */
fetirp_status fetirp_apply_block(fetirp_ctx ctx, int32_t k, const double* V, double* Q, int32_t precision);

/* As fetirp_apply_block on DEVICE buffers; enqueued on the context's stream, returns without waiting, except
 * that the first call after a factorisation in FP64, FP32 or TF32X3 on a structure with a pattern of
 * n_b >= 1024 first forms that pattern's S^+ and FP32 / tf32 forms of S^dag (see fetirp_create_pattern) and
 * waits for them: make that call before any stream capture.  A bounded wait of the tensor-core pipeline
 * (FETIRP_PREC_TF32X3) that expired is reported only through fetirp_device_status, since the call returns
 * before the kernel has run. */
fetirp_status fetirp_apply_block_device(fetirp_ctx ctx, int32_t k, const double* d_V, double* d_Q,
                                        int32_t precision);

/*
 * Completion status of the device work enqueued by the asynchronous "_device" entry points
 * (fetirp_apply_block_device, fetirp_apply_split_device, fetirp_apply_block_device_noalloc): waits for the
 * context's stream, then returns FETIRP_ETIMEOUT (and clears the flag) when a bounded wait inside the
 * tensor-core pipeline expired since the last check, in which case the outputs of those calls are not valid;
 * FETIRP_OK otherwise.  The blocking entry points (fetirp_solve, fetirp_apply_block, fetirp_apply_split) make
 * this check themselves.
 */
fetirp_status fetirp_device_status(fetirp_ctx ctx);

/* Q = P^T F P S(r) for the k split columns of one interface vector r (the multivector of Section 3.1:
 * column g holds r on the rows of the occurrences of group g, scaled by 1 / the row's occurrence count),
 * computed in the sparse-column form.  F acts on S(r) only where a split column touches an occurrence (its own
 * group and its neighbours' groups: at most seven right-hand sides per occurrence in 3D instead of k), and
 * F G X with X = (G^T G)^{-1} G^T S(r) comes from precomputed local coarse responses
 * M_s = S^+(s) B(s)^T G restricted to the kernel modes of s and its neighbours (by linearity of the
 * F-apply of Table 1).  The result equals fetirp_apply_block on the dense S(r) in the same precision.
 *   r: n_lambda doubles; Q: n_lambda x k row-major doubles (k = the structure's multivector width), caller
 *      owned.  _device: device pointers, asynchronous on the context's stream; otherwise host buffers.
 *   The first call for a structure builds the pair lists and M (FP64 products, kept in FP64 and FP32).
 * Errors: FETIRP_ESTATE before a structure is prepared; FETIRP_EINVAL for NULL buffers, an unknown precision,
 * or more than 48 coarse columns touching one occurrence. */
fetirp_status fetirp_apply_split(fetirp_ctx ctx, const double* r, double* Q, int32_t precision);
fetirp_status fetirp_apply_split_device(fetirp_ctx ctx, const double* d_r, double* d_Q, int32_t precision);

/*
 * Allocation-free variant of fetirp_apply_block_device (this entry point has no counterpart in the paper; it
 * exists for callers of the library).  Some callers cannot let a library allocate device memory while they
 * run: for example an application that provisions every byte of GPU memory once at start-up through its own
 * allocator and forbids later cudaMalloc/cudaFree calls, whose implicit device synchronisation and failure
 * modes it cannot accept.  This call computes the same Q = P^T F P V (same arguments and layout) but keeps
 * its scratch (the gathered traces, local products and coarse vectors) in one fixed array compiled into the
 * library, FETIRP_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - Limit: a call needing more scratch than FETIRP_NOALLOC_SCRATCH_BYTES (about 8 bytes x k x (n_lambda +
 *    2 x sum over occurrences of the boundary dof count) in FP64) returns FETIRP_EINVAL with the sizes in
 *    fetirp_last_error; nothing is written.
 *  - Set-up: the first call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 *    device current) and caches it, and the first call after a factorisation forms the operators of large
 *    patterns as fetirp_apply_block_device does (into buffers sized at factorisation: no allocation); make
 *    those first calls before any stream capture.
 *  - Sharing: every call on a device uses the same array and it keeps the previous call's contents; the
 *    call overwrites every scratch entry it reads, so nothing has to start at zero.  Calls that overlap on the
 *    GPU (other streams, other host threads, other contexts on the same device) race on the array and must
 *    be serialised by the caller.  The partial sums of G^T V and of the coarse product (G^T G)^{-1} X use
 *    small buffers of the context itself, allocated by fetirp_prepare, so two overlapping calls on one
 *    context race on those as well.
 *  - Requires fetirp_prepare (or a solve) on ctx first; enqueued on the context's stream.
 */
#define FETIRP_NOALLOC_SCRATCH_BYTES (32u << 20)
fetirp_status fetirp_apply_block_device_noalloc(fetirp_ctx ctx, int32_t k, const double* d_V, double* d_Q,
                                                int32_t precision);

/*
 * Build the coarse problem (G, G^T G and its inverse, e, lambda_0) and d for n_lambda rows and the given
 * c (host, may be NULL) without iterating.  fetirp_solve calls it itself.
 */
fetirp_status fetirp_prepare(fetirp_ctx ctx, int64_t n_lambda, const double* c);

/* Re-run the FP64 factorisation of every pattern from its resident stiffness (the setup of the method);
 * blocks until done. */
fetirp_status fetirp_factorize(fetirp_ctx ctx);

/*
 * Read back a pattern's operators (test hook).  Any output may be NULL.
 *  n_b_out, kernel_dim_out: boundary dof count (n_bnd * dofs_per_node) and detected kernel dimension.
 *  splus[n_b * n_b]: S^+ (row-major, boundary dofs in bnd_nodes order, dof-major within a node).
 *  kernel[n * kernel_dim]: N (row-major over the pattern's ORIGINAL dof numbering), K N = 0.
 * Call once with splus = kernel = NULL to learn the sizes.
 */
fetirp_status fetirp_get_pattern(fetirp_ctx ctx, int32_t pattern_id, int32_t* n_b_out, int32_t* kernel_dim_out,
                                 double* splus, double* kernel);

/* ------------------------------------------------------------------------------------------- serving
 * Continuous batching of whole structures over a resident pattern library.  A server owns max_slots worker
 * threads, each driving a child context (own stream) of the library context.  Submitted structures queue in
 * arrival order; a slot takes the next structure as soon as it is free and the structure's device-memory
 * estimate fits in what the other active structures leave of mem_budget_bytes (a structure is always
 * admitted when nothing else runs).  Structures solved at the same time overlap on the GPU through their
 * streams.  Each result is computed with the same kernels and buffers it would get alone, so it does not
 * depend on what else is in flight.
 */
typedef struct fetirp_server_s* fetirp_server;

/* A structure: occurrences of library patterns (arrays as in fetirp_add_occurrence, concatenated). */
typedef struct {
  int32_t n_occ;
  const int32_t* pattern_id;     /* [n_occ] ids in the library context */
  const double* rot;             /* [9 n_occ] row-major rotations, or NULL for identities */
  const int32_t* link_offset;    /* [n_occ + 1] prefix offsets into the link arrays */
  const int32_t* local_node;     /* links, concatenated over occurrences */
  const int8_t* global_comp;
  const int32_t* lambda_row;
  const int8_t* sign;
  const int64_t* f_offset;       /* [n_occ + 1] prefix offsets into f_global (each occurrence's n_dofs) */
  const double* f_global;        /* loads, concatenated over occurrences */
  int64_t n_lambda;
  const double* c;               /* [n_lambda] or NULL */
  int32_t k;                     /* multivector width; 0 = options default */
  const int32_t* group_of_occ;   /* [n_occ] or NULL (contiguous groups) */
} fetirp_structure;

/* library: a context holding the patterns (not a child).  slot_opt: options of every slot's context (NULL:
 * the library's options).  Every input is copied. */
fetirp_status fetirp_server_create(fetirp_ctx library, const fetirp_options* slot_opt, int32_t max_slots,
                                   int64_t mem_budget_bytes, fetirp_server* out);
/* Continuous batching of F-applies across requests: a slot that takes the next structure also takes, up to
 * max_structures in all, queued structures made of the same single library pattern while the union stays within
 * 64 multivector columns and the memory budget, and solves them together as independent blocks of one structure
 * (fetirp_set_row_blocks): every local-product launch then serves all of them, and each result meets the
 * relative tolerance on its own (the same solution as alone, to that tolerance; not bitwise).  1 (the default)
 * = one structure per solve.  FETIRP_EINVAL outside 1..64. */
fetirp_status fetirp_server_set_batching(fetirp_server srv, int32_t max_structures);
/* Queue a structure (copied) and return its ticket. */
fetirp_status fetirp_server_submit(fetirp_server srv, const fetirp_structure* st, int64_t* ticket);
/* Wait up to timeout_s seconds (0: just poll; < 0: forever) for a ticket.  *done = 1 when finished; then the
 * outputs (host buffers of n_lambda and sum n_dofs doubles, may be NULL), stats and, through the return value,
 * the solve's own status are delivered and the ticket is released.  latency_ms (may be NULL): submit -> done. */
fetirp_status fetirp_server_wait(fetirp_server srv, int64_t ticket, double timeout_s, int32_t* done,
                                 double* lambda_out, double* u_out, fetirp_stats* stats, double* latency_ms);
/* Non-blocking check of a ticket: fetirp_server_wait with timeout_s = 0 (same outputs, same release of the
 * ticket once *done = 1). */
fetirp_status fetirp_server_poll(fetirp_server srv, int64_t ticket, int32_t* done, double* lambda_out,
                                 double* u_out, fetirp_stats* stats, double* latency_ms);
/* Finish queued work, join the slots and release everything. */
void fetirp_server_destroy(fetirp_server srv);

#ifdef __cplusplus
}
#endif
#endif /* FETIRP_H */
