"""Serving: structures submitted to a server over a resident pattern library are solved by child contexts
in concurrent slots.  Each result must be the same alone and in a mix (bitwise: every structure runs on its
own stream and buffers with deterministic kernels) and must match the oracle."""
import numpy as np
import pytest

from fetirp_gen import library_patterns, fill_structure, LIBRARY
from oracle.direct import direct

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")

SMALL_LIBRARY = [0, 1, 3]   # heat 16^2, heat 32^2, elastic 8^3 from the serving library


@pytest.fixture(scope="module")
def library():
    pats = library_patterns()
    ctx = F.fetirp_create(F.fetirp_default_options())
    pids = {}
    for i in SMALL_LIBRARY:
        p = pats[i]
        K = p.K.tocsr()
        pids[i] = F.fetirp_create_pattern(ctx, p.n_nodes, p.dpn, K.indptr, K.indices, K.data, p.bnd_nodes,
                                          p.kernel_dim)
    yield ctx, pats, pids
    F.fetirp_destroy(ctx)


def _requests(pats, n=9):
    rng = np.random.default_rng(5)
    out = []
    for i in range(n):
        li = SMALL_LIBRARY[i % len(SMALL_LIBRARY)]
        prob = fill_structure(pats[li], int(rng.integers(4, 20)), seed=100 + i, k=8, rotate=(li == 3))
        out.append((li, prob))
    return out


def _serve(ctx, pids, reqs, slots, budget):
    opts = F.fetirp_default_options(precision="fp32", tol=1e-10, history_bytes=256 << 20)
    srv = F.fetirp_server_create(ctx, opts, slots, budget)
    try:
        structs = [F.structure_of(prob, {0: pids[li]}) for li, prob in reqs]
        tickets = [F.fetirp_server_submit(srv, s) for s in structs]
        res = [F.fetirp_server_wait(srv, t, prob.n_lambda, F.n_u(prob)) for t, (_, prob) in zip(tickets, reqs)]
    finally:
        F.fetirp_server_destroy(srv)
    return res


def test_results_same_alone_and_in_the_mix(library):
    ctx, pats, pids = library
    reqs = _requests(pats)
    mixed = _serve(ctx, pids, reqs, slots=4, budget=8 << 30)
    for i in (0, 4, 7):
        alone = _serve(ctx, pids, [reqs[i]], slots=1, budget=8 << 30)[0]
        assert np.array_equal(alone[0], mixed[i][0]) and np.array_equal(alone[1], mixed[i][1])
    for (li, prob), (lam, u, st, lat) in zip(reqs, mixed):
        us_ref, lam_ref, _, _ = direct(prob)
        assert np.linalg.norm(lam - lam_ref) / np.linalg.norm(lam_ref) < 1e-8
        for a, b in zip(F.split_u(prob, u), us_ref):
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8
        assert st["rel_residual"] <= 1e-10 and lat > 0


def test_admission_by_memory_budget(library):
    """With a budget below one structure's estimate, structures still run (one at a time) and all finish."""
    ctx, pats, pids = library
    reqs = _requests(pats, n=4)
    res = _serve(ctx, pids, reqs, slots=4, budget=1)
    assert all(r is not None for r in res)
    lat = [r[3] for r in res]
    assert max(lat) > min(lat)          # queued behind one another


def test_poll_delivers_the_same_results(library):
    """fetirp_server_poll never blocks: polling every ticket until it is done (bounded on the host) delivers
    the results that fetirp_server_wait delivers, bitwise."""
    import time
    ctx, pats, pids = library
    reqs = _requests(pats, n=3)
    waited = _serve(ctx, pids, reqs, slots=2, budget=8 << 30)
    opts = F.fetirp_default_options(precision="fp32", tol=1e-10, history_bytes=256 << 20)
    srv = F.fetirp_server_create(ctx, opts, 2, 8 << 30)
    try:
        tickets = [F.fetirp_server_submit(srv, F.structure_of(prob, {0: pids[li]})) for li, prob in reqs]
        polled = [None] * len(reqs)
        deadline = time.monotonic() + 120.0
        while any(p is None for p in polled) and time.monotonic() < deadline:
            for i, (t, (_, prob)) in enumerate(zip(tickets, reqs)):
                if polled[i] is None:
                    polled[i] = F.fetirp_server_poll(srv, t, prob.n_lambda, F.n_u(prob))
            time.sleep(0.001)
    finally:
        F.fetirp_server_destroy(srv)
    assert all(p is not None for p in polled)
    for a, b in zip(waited, polled):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_batched_structures_match_the_direct_solve(library, prec):
    """Continuous batching across requests: structures of the same library pattern queued together are solved
    as independent blocks of one structure (one local-product launch per iteration for all of them).  Every
    result meets the tolerance on its own and matches the direct solve and the structure solved alone to 1e-8
    (the same solution; the iterates are not bitwise those of the lone solve)."""
    ctx, pats, pids = library
    rng = np.random.default_rng(12)
    reqs = [(3, fill_structure(pats[3], int(rng.integers(4, 12)), seed=300 + i, k=8, rotate=True)) for i in range(5)]
    reqs += [(1, fill_structure(pats[1], int(rng.integers(4, 20)), seed=400 + i, k=8)) for i in range(3)]
    opts = F.fetirp_default_options(precision=prec, tol=1e-10, history_bytes=256 << 20)
    srv = F.fetirp_server_create(ctx, opts, 1, 8 << 30)   # one slot: the queue builds up behind the first solve
    try:
        F.fetirp_server_set_batching(srv, 4)
        structs = [F.structure_of(prob, {0: pids[li]}) for li, prob in reqs]
        tickets = [F.fetirp_server_submit(srv, st) for st in structs]
        res = [F.fetirp_server_wait(srv, t, prob.n_lambda, F.n_u(prob)) for t, (_, prob) in zip(tickets, reqs)]
    finally:
        F.fetirp_server_destroy(srv)
    batched_iters = set()
    for (li, prob), (lam, u, st, lat) in zip(reqs, res):
        us_ref, lam_ref, _, _ = direct(prob)
        assert st["rel_residual"] <= 1e-10
        assert np.linalg.norm(lam - lam_ref) / np.linalg.norm(lam_ref) < 1e-8
        for a, b in zip(F.split_u(prob, u), us_ref):
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8
        batched_iters.add(st["iterations"])
    # several structures shared a solve (identical statistics), so at least one batch held more than one
    assert len(batched_iters) < len(reqs)
