"""fetirp_apply_block_device_noalloc: the allocation-free variant of fetirp_apply_block_device, for callers that
cannot let the library allocate device memory during a call.  Its scratch is a fixed array compiled into
the library, shared by every call on a device; each result must match the allocating entry point's, on two
calls in a row (the second call sees the first call's leftovers in the shared array).  This file is named
so that pytest collects it last."""
import numpy as np
import pytest

from fetirp_gen import config, elastic_grid

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_1208_6387_gb300.fetirp")
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 2e-4, "tf32x3": 2e-4}   # the tolerances of the operator parity tests


def _ctx(prob):
    ctx = F.fetirp_create(F.fetirp_default_options())
    F.load_problem(ctx, prob)
    F.fetirp_prepare(ctx, prob.n_lambda, prob.c)
    return ctx


@pytest.mark.parametrize("name", ["c1", "c2"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_noalloc_matches_allocating_entry_point(name, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prob = config(name)
    ctx = _ctx(prob)
    try:
        gen = torch.Generator(device="cuda").manual_seed(3)
        for call in range(2):   # two calls in a row, different inputs
            k = prob.k if call == 0 else max(1, prob.k // 2)
            V = torch.randn(prob.n_lambda, k, dtype=torch.float64, device="cuda", generator=gen)
            Q_ref = torch.empty_like(V)
            Q = torch.full_like(V, float("nan"))
            F.fetirp_apply_block_device(ctx, k, V.data_ptr(), Q_ref.data_ptr(), F.PRECISIONS[prec])
            F.fetirp_apply_block_device_noalloc(ctx, k, V.data_ptr(), Q.data_ptr(), F.PRECISIONS[prec])
            F.fetirp_device_status(ctx)   # no bounded tensor-core wait expired in either call
            torch.cuda.synchronize()
            a, b = Q.cpu().numpy(), Q_ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL[prec], (call, prec)
    finally:
        F.fetirp_destroy(ctx)


def test_noalloc_rejects_oversize_requests():
    """A block whose scratch exceeds the fixed array is refused with FETIRP_EINVAL and Q is left untouched."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prob = elastic_grid(8, (4, 4, 2), n_patterns=1, k=32, rotate=False)
    n_b = prob.patterns[0].n_b
    k = 64
    need = 8 * k * (prob.n_lambda + 2 * prob.n_occ * (n_b + 3) // 4 * 4)
    assert need > F.FETIRP_NOALLOC_SCRATCH_BYTES
    ctx = _ctx(prob)
    try:
        V = torch.ones(prob.n_lambda, k, dtype=torch.float64, device="cuda")
        Q = torch.full_like(V, 7.0)
        with pytest.raises(F.FetirpError) as e:
            F.fetirp_apply_block_device_noalloc(ctx, k, V.data_ptr(), Q.data_ptr(), F.FETIRP_PREC_FP64)
        assert e.value.status == F.FETIRP_EINVAL and "scratch" in str(e.value)
        torch.cuda.synchronize()
        assert bool((Q == 7.0).all())
    finally:
        F.fetirp_destroy(ctx)
