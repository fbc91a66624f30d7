"""maxsat_eval_noalloc: the allocation-free evaluation for callers that cannot
call cudaMalloc (stream-capturing code, frameworks whose allocator owns the
device memory, latency-critical loops). Through the C ABI it must give the
same weighted costs as maxsat_eval, call after call, while its scratch lives
in one static device array shared by every call.

Collected last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_02101_gb300 as m
    return m


def test_eval_noalloc_matches_eval_on_consecutive_calls(ms):
    import torch
    stream = torch.cuda.Stream()
    n, off, lits, w = workloads.mixed_length(n=2000, m=9000, cap=5, seed=7)
    params = ms.maxsat_default_params(n_buckets=2, fit_iters=2000)
    ctx = ms.maxsat_create(n, off, lits, w, params, stream)
    with torch.cuda.stream(stream):
        off_d = torch.from_numpy(off).cuda()
        lits_d = torch.from_numpy(lits).cuda()
        w_d = torch.from_numpy(w).cuda()
    rng = np.random.default_rng(0)
    for B in (300, 1000):  # two calls in a row, different sizes and inputs
        X = rng.integers(0, 2, size=(B, n)).astype(np.uint8)
        with torch.cuda.stream(stream):
            x_d = torch.from_numpy(X).cuda()
            ref = torch.zeros(B, dtype=torch.int64, device="cuda")
            out = torch.full((B,), -1, dtype=torch.int64, device="cuda")
        ms.maxsat_eval(ctx, x_d, ref)
        ms.maxsat_eval_noalloc(n, off_d, lits_d, w_d, x_d, out, stream)
        stream.synchronize()
        assert torch.equal(out.cpu(), ref.cpu())
        assert int(out.min()) >= 0
    ms.maxsat_destroy(ctx)


def test_eval_noalloc_rejects_requests_beyond_its_scratch(ms):
    import torch
    n, B = 20000, 4096  # 20000 x 4096 transposed bytes alone exceed the array
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    lits = torch.ones(1, dtype=torch.int32, device="cuda")
    x = torch.zeros((B, n), dtype=torch.uint8, device="cuda")
    cost = torch.zeros(B, dtype=torch.int64, device="cuda")
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_eval_noalloc(n, off, lits, None, x, cost)
    assert e.value.code == ms.MAXSAT_EINVAL
    assert "MAXSAT_NOALLOC_SCRATCH_BYTES" in str(e.value)
