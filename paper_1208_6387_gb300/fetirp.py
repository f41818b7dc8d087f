"""Thin Python binding of include/fetirp.h (ctypes): the same entry points, argument marshalling only.

Every step of the method runs in libfetirp.so on the GPU.  There is no CPU fallback: importing works without
a GPU (so the exported symbols can be checked), but every call needs the compiled library and a CUDA device,
and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libfetirp.so")

FETIRP_OK, FETIRP_EINVAL, FETIRP_ENOMEM, FETIRP_ESINGULAR, FETIRP_ENOCONV, FETIRP_ECUDA, FETIRP_ESTATE, \
    FETIRP_ETIMEOUT = range(8)
FETIRP_PREC_FP64, FETIRP_PREC_FP32, FETIRP_PREC_TF32X3, FETIRP_PREC_AUTO, FETIRP_PREC_BF16X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FETIRP_PREC_FP64, "fp32": FETIRP_PREC_FP32, "tf32x3": FETIRP_PREC_TF32X3,
              "auto": FETIRP_PREC_AUTO, "bf16x3": FETIRP_PREC_BF16X3}


# device allocator hooks of fetirp_options: alloc(bytes, stream, user) -> device pointer; free(ptr, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class fetirp_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32), ("block_k", C.c_int32),
                ("max_outer", C.c_int32), ("inner_tol", C.c_double), ("pivot_tol", C.c_double),
                ("eig_trunc", C.c_double), ("cuda_stream", C.c_void_p), ("device", C.c_int32),
                ("check_every", C.c_int32), ("timing", C.c_int32), ("eig_trunc_inner", C.c_double),
                ("use_graphs", C.c_int32), ("timing_mask", C.c_int32), ("history_bytes", C.c_int64),
                ("persistent", C.c_int32), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


def caching_allocator_hooks(device: int = 0):
    """(alloc, free) hooks for fetirp_options that take device memory from PyTorch's caching allocator on the
    given device and the context's stream.  Keep the returned objects alive while any context that uses them
    exists."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device, stream=int(stream or 0))
        except Exception:
            return None   # the library reports FETIRP_ENOMEM

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free)


PHASES = ["factor", "coarse", "local", "gather", "scatter", "project", "gram", "reorth", "update", "recover",
          "normalise", "iterate", "outer"]


class fetirp_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("outer_steps", C.c_int32), ("f_applies", C.c_int32),
                ("dropped_directions", C.c_int32), ("kernel_dim_total", C.c_int32), ("rel_residual", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("launches", C.c_int64),
                ("phase_ms", C.c_double * 13), ("phase_launches", C.c_int64 * 13),
                ("phase_flops", C.c_double * 13), ("phase_bytes", C.c_double * 13)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name.startswith("phase_") else v
        return d


class fetirp_structure(C.Structure):
    _fields_ = [("n_occ", C.c_int32), ("pattern_id", C.c_void_p), ("rot", C.c_void_p), ("link_offset", C.c_void_p),
                ("local_node", C.c_void_p), ("global_comp", C.c_void_p), ("lambda_row", C.c_void_p),
                ("sign", C.c_void_p), ("f_offset", C.c_void_p), ("f_global", C.c_void_p), ("n_lambda", C.c_int64),
                ("c", C.c_void_p), ("k", C.c_int32), ("group_of_occ", C.c_void_p)]


class FetirpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_STATUS = {0: "FETIRP_OK", 1: "FETIRP_EINVAL", 2: "FETIRP_ENOMEM", 3: "FETIRP_ESINGULAR", 4: "FETIRP_ENOCONV",
           5: "FETIRP_ECUDA", 6: "FETIRP_ESTATE", 7: "FETIRP_ETIMEOUT"}

_lib = None
P = C.c_void_p
_SIGS = {
    "fetirp_default_options": (None, [C.POINTER(fetirp_options)]),
    "fetirp_status_string": (C.c_char_p, [C.c_int]),
    "fetirp_create": (C.c_int, [C.POINTER(fetirp_options), C.POINTER(P)]),
    "fetirp_last_error": (C.c_char_p, [P]),
    "fetirp_destroy": (None, [P]),
    "fetirp_create_pattern": (C.c_int, [P, C.c_int32, C.c_int32, P, P, P, C.c_int32, P, C.c_int32,
                                        C.POINTER(C.c_int32)]),
    "fetirp_add_occurrence": (C.c_int, [P, C.c_int32, P, C.c_int32, P, P, P, P, P, C.POINTER(C.c_int32)]),
    "fetirp_set_groups": (C.c_int, [P, C.c_int32, P]),
    "fetirp_clear_occurrences": (C.c_int, [P]),
    "fetirp_autotune_k": (C.c_int, [P, C.c_int64, P, C.c_int32, P, C.POINTER(C.c_int32), P]),
    "fetirp_create_child": (C.c_int, [P, C.POINTER(fetirp_options), C.POINTER(P)]),
    "fetirp_server_create": (C.c_int, [P, C.POINTER(fetirp_options), C.c_int32, C.c_int64, C.POINTER(P)]),
    "fetirp_server_submit": (C.c_int, [P, C.POINTER(fetirp_structure), C.POINTER(C.c_int64)]),
    "fetirp_server_wait": (C.c_int, [P, C.c_int64, C.c_double, C.POINTER(C.c_int32), P, P, C.POINTER(fetirp_stats),
                                     C.POINTER(C.c_double)]),
    "fetirp_server_poll": (C.c_int, [P, C.c_int64, C.POINTER(C.c_int32), P, P, C.POINTER(fetirp_stats),
                                     C.POINTER(C.c_double)]),
    "fetirp_server_destroy": (None, [P]),
    "fetirp_server_set_batching": (C.c_int, [P, C.c_int32]),
    "fetirp_solve": (C.c_int, [P, C.c_int64, P, P, P, C.POINTER(fetirp_stats)]),
    "fetirp_solve_device": (C.c_int, [P, C.c_int64, P, P, P, C.POINTER(fetirp_stats)]),
    "fetirp_apply_block": (C.c_int, [P, C.c_int32, P, P, C.c_int32]),
    "fetirp_apply_block_device": (C.c_int, [P, C.c_int32, P, P, C.c_int32]),
    "fetirp_apply_block_device_noalloc": (C.c_int, [P, C.c_int32, P, P, C.c_int32]),
    "fetirp_prepare": (C.c_int, [P, C.c_int64, P]),
    "fetirp_factorize": (C.c_int, [P]),
    "fetirp_inject_barrier_stall": (C.c_int, [P]),
    "fetirp_device_status": (C.c_int, [P]),
    "fetirp_set_permutation": (C.c_int, [P, C.c_int64, P, P, P, C.c_int32, C.c_int32]),
    "fetirp_set_preconditioner": (C.c_int, [P, C.c_int32, C.c_int32]),
    "fetirp_set_row_blocks": (C.c_int, [P, C.c_int32, P]),
    "fetirp_apply_split": (C.c_int, [P, C.c_void_p, C.c_void_p, C.c_int]),
    "fetirp_apply_split_device": (C.c_int, [P, C.c_void_p, C.c_void_p, C.c_int]),
    "fetirp_get_pattern": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), P, P]),
}


def lib():
    """The loaded libfetirp.so (built by __graft_entry__.build() / paper_1208_6387_gb300._build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfetirp.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, st):
    if st != FETIRP_OK:
        msg = lib().fetirp_last_error(ctx).decode() if ctx else ""
        raise FetirpError(st, msg)


def fetirp_default_options(**kw) -> fetirp_options:
    o = fetirp_options()
    lib().fetirp_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


def fetirp_create(opts: fetirp_options | None = None):
    h = C.c_void_p()
    st = lib().fetirp_create(C.byref(opts) if opts is not None else None, C.byref(h))
    if st != FETIRP_OK:
        raise FetirpError(st, "fetirp_create failed (no CUDA device or bad options)")
    return h


def fetirp_status_string(status: int) -> str:
    return lib().fetirp_status_string(int(status)).decode()


def fetirp_destroy(ctx):
    lib().fetirp_destroy(ctx)


def fetirp_last_error(ctx) -> str:
    return lib().fetirp_last_error(ctx).decode()


def fetirp_create_pattern(ctx, n_nodes, dofs_per_node, rowptr, col, val, bnd_nodes, expected_kernel_dim=-1) -> int:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    bnd = np.ascontiguousarray(bnd_nodes, dtype=np.int32)
    pid = C.c_int32()
    _check(ctx, lib().fetirp_create_pattern(ctx, int(n_nodes), int(dofs_per_node), _ptr(rowptr), _ptr(col), _ptr(val),
                                            len(bnd), _ptr(bnd), int(expected_kernel_dim), C.byref(pid)))
    return pid.value


def fetirp_add_occurrence(ctx, pattern_id, rot, local_node, global_comp, lambda_row, sign, f_global) -> int:
    rot = None if rot is None else np.ascontiguousarray(rot, dtype=np.float64).reshape(9)
    ln = np.ascontiguousarray(local_node, dtype=np.int32)
    gc = np.ascontiguousarray(global_comp, dtype=np.int8)
    lr = np.ascontiguousarray(lambda_row, dtype=np.int32)
    sg = np.ascontiguousarray(sign, dtype=np.int8)
    f = np.ascontiguousarray(f_global, dtype=np.float64)
    oid = C.c_int32()
    _check(ctx, lib().fetirp_add_occurrence(ctx, int(pattern_id), _ptr(rot), len(lr), _ptr(ln), _ptr(gc), _ptr(lr),
                                            _ptr(sg), _ptr(f), C.byref(oid)))
    return oid.value


def fetirp_set_groups(ctx, k, group_of_occ):
    g = np.ascontiguousarray(group_of_occ, dtype=np.int32)
    _check(ctx, lib().fetirp_set_groups(ctx, int(k), _ptr(g)))


def fetirp_autotune_k(ctx, n_lambda, c, candidates=(4, 8, 16, 32)):
    """Returns (best k, solve times in ms per candidate); the context keeps the best grouping."""
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    times = np.zeros(len(cand))
    bk = C.c_int32()
    _check(ctx, lib().fetirp_autotune_k(ctx, int(n_lambda), _ptr(c), len(cand), _ptr(cand), C.byref(bk), _ptr(times)))
    return bk.value, times


def fetirp_clear_occurrences(ctx):
    _check(ctx, lib().fetirp_clear_occurrences(ctx))


def fetirp_create_child(parent, opts: fetirp_options | None = None):
    h = C.c_void_p()
    st = lib().fetirp_create_child(parent, C.byref(opts) if opts is not None else None, C.byref(h))
    if st != FETIRP_OK:
        raise FetirpError(st, "fetirp_create_child failed")
    return h


def structure_of(prob, pattern_ids=None):
    """Marshal a fetirp_gen.Problem into a fetirp_structure (the arrays are kept alive on the returned
    object).  pattern_ids maps the problem's pattern indices to library ids (default: identity)."""
    pid = np.array([o.pattern if pattern_ids is None else pattern_ids[o.pattern] for o in prob.occs], dtype=np.int32)
    rot = np.concatenate([o.rot.astype(np.float64).ravel() for o in prob.occs])
    lo = np.concatenate([[0], np.cumsum([o.n_links for o in prob.occs])]).astype(np.int32)
    cat = lambda f, dt: np.ascontiguousarray(np.concatenate([f(o) for o in prob.occs]).astype(dt))
    ln, gc = cat(lambda o: o.link_local_node, np.int32), cat(lambda o: o.link_global_comp, np.int8)
    lr, sg = cat(lambda o: o.link_lambda_row, np.int32), cat(lambda o: o.link_sign, np.int8)
    fo = np.concatenate([[0], np.cumsum([len(o.f_global) for o in prob.occs])]).astype(np.int64)
    fg = cat(lambda o: o.f_global, np.float64)
    c = np.ascontiguousarray(prob.c, dtype=np.float64)
    grp = np.ascontiguousarray(prob.groups, dtype=np.int32)
    s = fetirp_structure(len(prob.occs), _ptr(pid), _ptr(rot), _ptr(lo), _ptr(ln), _ptr(gc), _ptr(lr), _ptr(sg),
                         _ptr(fo), _ptr(fg), int(prob.n_lambda), _ptr(c), int(prob.k), _ptr(grp))
    s._keep = (pid, rot, lo, ln, gc, lr, sg, fo, fg, c, grp)
    return s


def fetirp_server_create(library, slot_opts: fetirp_options | None, max_slots, mem_budget_bytes):
    h = C.c_void_p()
    st = lib().fetirp_server_create(library, C.byref(slot_opts) if slot_opts is not None else None, int(max_slots),
                                    int(mem_budget_bytes), C.byref(h))
    if st != FETIRP_OK:
        raise FetirpError(st, "fetirp_server_create failed")
    return h


def fetirp_server_set_batching(srv, max_structures):
    st = lib().fetirp_server_set_batching(srv, int(max_structures))
    if st != FETIRP_OK:
        raise FetirpError(st, "fetirp_server_set_batching")


def fetirp_server_submit(srv, structure):
    t = C.c_int64()
    st = lib().fetirp_server_submit(srv, C.byref(structure), C.byref(t))
    if st != FETIRP_OK:
        raise FetirpError(st, "fetirp_server_submit failed")
    return t.value


def fetirp_server_wait(srv, ticket, n_lambda, n_u, timeout_s=-1.0, allow_noconv=False):
    """Returns None if not done within timeout_s, else (lambda, u, stats dict, latency_ms)."""
    done = C.c_int32()
    lam = np.zeros(int(n_lambda))
    u = np.zeros(int(n_u))
    stt = fetirp_stats()
    lat = C.c_double()
    s = lib().fetirp_server_wait(srv, int(ticket), float(timeout_s), C.byref(done), _ptr(lam), _ptr(u), C.byref(stt),
                                 C.byref(lat))
    if not done.value:
        if s != FETIRP_OK:
            raise FetirpError(s, "fetirp_server_wait failed")
        return None
    if s != FETIRP_OK and not (allow_noconv and s == FETIRP_ENOCONV):
        raise FetirpError(s, "structure failed in the server")
    return lam, u, stt.as_dict(), lat.value


def fetirp_server_poll(srv, ticket, n_lambda, n_u, allow_noconv=False):
    """Non-blocking: None while the structure is not done, else (lambda, u, stats dict, latency_ms)."""
    done = C.c_int32()
    lam = np.zeros(int(n_lambda))
    u = np.zeros(int(n_u))
    stt = fetirp_stats()
    lat = C.c_double()
    s = lib().fetirp_server_poll(srv, int(ticket), C.byref(done), _ptr(lam), _ptr(u), C.byref(stt), C.byref(lat))
    if not done.value:
        if s != FETIRP_OK:
            raise FetirpError(s, "fetirp_server_poll failed")
        return None
    if s != FETIRP_OK and not (allow_noconv and s == FETIRP_ENOCONV):
        raise FetirpError(s, "structure failed in the server")
    return lam, u, stt.as_dict(), lat.value


def fetirp_server_destroy(srv):
    lib().fetirp_server_destroy(srv)


def fetirp_prepare(ctx, n_lambda, c=None):
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    _check(ctx, lib().fetirp_prepare(ctx, int(n_lambda), _ptr(c)))


def fetirp_solve(ctx, n_lambda, c, n_u, allow_noconv=False):
    """Returns (lambda, u, stats dict); u concatenates the occurrences (global frame)."""
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    lam = np.zeros(int(n_lambda))
    u = np.zeros(int(n_u))
    st = fetirp_stats()
    s = lib().fetirp_solve(ctx, int(n_lambda), _ptr(c), _ptr(lam), _ptr(u), C.byref(st))
    if not (allow_noconv and s == FETIRP_ENOCONV):
        _check(ctx, s)
    return lam, u, st.as_dict()


def fetirp_solve_device(ctx, n_lambda, c_ptr, lambda_ptr, u_ptr, allow_noconv=False):
    """Device pointers (ints, e.g. torch tensor .data_ptr()); c_ptr may be 0 / None."""
    st = fetirp_stats()
    s = lib().fetirp_solve_device(ctx, int(n_lambda), C.c_void_p(c_ptr) if c_ptr else None, C.c_void_p(lambda_ptr),
                                  C.c_void_p(u_ptr), C.byref(st))
    if not (allow_noconv and s == FETIRP_ENOCONV):
        _check(ctx, s)
    return st.as_dict()


def fetirp_apply_block(ctx, V, precision=FETIRP_PREC_FP64):
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Q = np.zeros_like(V)
    _check(ctx, lib().fetirp_apply_block(ctx, V.shape[1], _ptr(V), _ptr(Q), int(precision)))
    return Q


def fetirp_apply_split(ctx, r, k, precision=FETIRP_PREC_FP64):
    """Q = P^T F P S(r) (n_lambda x k) by the sparse-column form; r: host vector."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    Q = np.zeros((r.shape[0], int(k)))
    _check(ctx, lib().fetirp_apply_split(ctx, _ptr(r), _ptr(Q), int(precision)))
    return Q


def fetirp_apply_split_device(ctx, r_ptr, Q_ptr, precision=FETIRP_PREC_FP64):
    _check(ctx, lib().fetirp_apply_split_device(ctx, C.c_void_p(r_ptr), C.c_void_p(Q_ptr), int(precision)))


def fetirp_apply_block_device(ctx, k, V_ptr, Q_ptr, precision=FETIRP_PREC_FP64):
    _check(ctx, lib().fetirp_apply_block_device(ctx, int(k), C.c_void_p(V_ptr), C.c_void_p(Q_ptr), int(precision)))


FETIRP_NOALLOC_SCRATCH_BYTES = 32 << 20


def fetirp_apply_block_device_noalloc(ctx, k, V_ptr, Q_ptr, precision=FETIRP_PREC_FP64):
    """Same operator as fetirp_apply_block_device with the scratch in the library's fixed device array (no
    device allocation in the call; see include/fetirp.h for the size limit and the sharing rules)."""
    _check(ctx, lib().fetirp_apply_block_device_noalloc(ctx, int(k), C.c_void_p(V_ptr), C.c_void_p(Q_ptr),
                                                         int(precision)))


def fetirp_set_permutation(ctx, Pi, n_images, shortcut=False):
    """The permutation multivector [z, Pi z, ...] (Pi: scipy sparse n_lambda x n_lambda, or None for the
    occurrence split); argument marshalling only."""
    if Pi is None:
        _check(ctx, lib().fetirp_set_permutation(ctx, 0, None, None, None, 1, 0))
        return
    import scipy.sparse as sp
    M = sp.csr_matrix(Pi)
    M.sort_indices()
    rowptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
    col = np.ascontiguousarray(M.indices, dtype=np.int32)
    val = np.ascontiguousarray(M.data, dtype=np.float64)
    _check(ctx, lib().fetirp_set_permutation(ctx, int(M.shape[0]), _ptr(rowptr), _ptr(col), _ptr(val),
                                             int(n_images), 1 if shortcut else 0))


PRECONDITIONERS = {"identity": 0, "dirichlet": 1, "lumped": 2, "superlumped": 3}
SCALINGS = {"multiplicity": 0, "stiffness": 1}


def fetirp_set_preconditioner(ctx, kind="identity", scaling="stiffness"):
    """The preconditioner of Eqs. 4-5 by name (identity, dirichlet, lumped, superlumped) and its scaling
    (multiplicity, stiffness); argument marshalling only."""
    _check(ctx, lib().fetirp_set_preconditioner(ctx, PRECONDITIONERS[kind], SCALINGS[scaling]))


def fetirp_set_row_blocks(ctx, row_offsets):
    """Independent sub-structures owning the multiplier rows [row_offsets[b], row_offsets[b + 1]) (None: one)."""
    if row_offsets is None:
        _check(ctx, lib().fetirp_set_row_blocks(ctx, 0, None))
        return
    ro = np.ascontiguousarray(row_offsets, dtype=np.int64)
    _check(ctx, lib().fetirp_set_row_blocks(ctx, len(ro) - 1, _ptr(ro)))


def fetirp_device_status(ctx):
    """Waits for the context's stream; raises FetirpError(FETIRP_ETIMEOUT) if a bounded tensor-core wait of an
    asynchronous _device call expired since the last check."""
    _check(ctx, lib().fetirp_device_status(ctx))


def fetirp_factorize(ctx):
    _check(ctx, lib().fetirp_factorize(ctx))


def fetirp_inject_barrier_stall(ctx):
    """Test hook: the next persistent launch waits for a CTA that never arrives (0.2 s limit) -> ETIMEOUT."""
    _check(ctx, lib().fetirp_inject_barrier_stall(ctx))


def fetirp_get_pattern(ctx, pattern_id, n_dofs=None):
    """Returns (n_b, kernel_dim, S^+ (n_b x n_b), N (n_dofs x kernel_dim) or None)."""
    nb, kd = C.c_int32(), C.c_int32()
    _check(ctx, lib().fetirp_get_pattern(ctx, int(pattern_id), C.byref(nb), C.byref(kd), None, None))
    S = np.zeros((nb.value, nb.value))
    N = np.zeros((n_dofs, kd.value)) if n_dofs is not None else None
    _check(ctx, lib().fetirp_get_pattern(ctx, int(pattern_id), None, None, _ptr(S), _ptr(N)))
    return nb.value, kd.value, S, N


# ------------------------------------------------------------------------------------------------ marshalling
def load_problem(ctx, prob, expected_kernel=True, groups=True):
    """Register every pattern and occurrence of a fetirp_gen.Problem (argument marshalling only)."""
    pids = []
    for pat in prob.patterns:
        K = pat.K.tocsr()
        pids.append(fetirp_create_pattern(ctx, pat.n_nodes, pat.dpn, K.indptr, K.indices, K.data, pat.bnd_nodes,
                                          pat.kernel_dim if expected_kernel else -1))
    for occ in prob.occs:
        fetirp_add_occurrence(ctx, pids[occ.pattern], occ.rot.astype(float), occ.link_local_node,
                              occ.link_global_comp, occ.link_lambda_row, occ.link_sign, occ.f_global)
    if groups:
        fetirp_set_groups(ctx, prob.k, prob.groups)
    return pids


def n_u(prob):
    return sum(prob.patterns[o.pattern].n_dofs for o in prob.occs)


def split_u(prob, u):
    out, off = [], 0
    for o in prob.occs:
        n = prob.patterns[o.pattern].n_dofs
        out.append(u[off:off + n])
        off += n
    return out
