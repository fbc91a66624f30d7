"""maxsat_eval_noalloc: the allocation-free evaluation for callers that cannot
call cudaMalloc (frameworks whose own allocator owns the device memory budget,
latency-critical loops that cannot take an allocation's implicit
synchronisation). Through the C ABI it must give the same weighted costs as
maxsat_eval and as the oracle's literal-by-literal evaluation, call after
call, while its scratch lives in one static device array shared by every call.

Collected last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

import oracle
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


def _dev(torch, a, stream):
    with torch.cuda.stream(stream):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_eval_noalloc_matches_eval_on_consecutive_calls(ms):
    import torch
    stream = torch.cuda.Stream()
    n, off, lits, w = workloads.mixed_length(n=2000, m=9000, cap=5, seed=7)
    params = ms.maxsat_default_params(n_buckets=2, fit_iters=2000)
    ctx = ms.maxsat_create(n, off, lits, w, params, stream)
    off_d, lits_d, w_d = (_dev(torch, a, stream) for a in (off, lits, w))
    inst = oracle.Instance(n, off, lits, w)
    rng = np.random.default_rng(0)
    for B in (300, 1000):  # two calls in a row, different sizes and inputs
        X = rng.integers(0, 2, size=(B, n)).astype(np.uint8)
        x_d = _dev(torch, X, stream)
        with torch.cuda.stream(stream):
            ref = torch.zeros(B, dtype=torch.int64, device="cuda")
            out = torch.full((B,), -1, dtype=torch.int64, device="cuda")
        ms.maxsat_eval(ctx, x_d, ref)
        ms.maxsat_eval_noalloc(n, off_d, lits_d, w_d, x_d, out, stream)
        stream.synchronize()
        assert torch.equal(out.cpu(), ref.cpu())
        assert np.array_equal(out.cpu().numpy(), oracle.evaluate(inst, X))
    ms.maxsat_destroy(ctx)


def test_eval_noalloc_unweighted_equals_unit_weights(ms):
    """weights_dev = None scores every clause 1, as a context whose weights
    are all 1 (twice in a row)."""
    import torch
    stream = torch.cuda.Stream()
    n, off, lits, _ = workloads.random_ksat(300, 1300, 3, seed=2)
    ones = np.ones(len(off) - 1, np.int64)
    ctx = ms.maxsat_create(n, off, lits, ones,
                           ms.maxsat_default_params(n_buckets=1, fit_iters=2000), stream)
    off_d, lits_d = _dev(torch, off, stream), _dev(torch, lits, stream)
    rng = np.random.default_rng(1)
    for B in (256, 77):
        X = rng.integers(0, 2, size=(B, n)).astype(np.uint8)
        x_d = _dev(torch, X, stream)
        with torch.cuda.stream(stream):
            ref = torch.zeros(B, dtype=torch.int64, device="cuda")
            out = torch.full((B,), -1, dtype=torch.int64, device="cuda")
        ms.maxsat_eval(ctx, x_d, ref)
        ms.maxsat_eval_noalloc(n, off_d, lits_d, None, x_d, out, stream)
        stream.synchronize()
        assert torch.equal(out.cpu(), ref.cpu())
    ms.maxsat_destroy(ctx)


def test_eval_noalloc_duplicate_and_out_of_range_literals(ms):
    """Duplicates and x OR NOT x count as in the oracle; literals outside
    [-n, n] \\ {0} (including INT32_MIN) are skipped, so the expected cost is
    the oracle's on the formula without them (a clause left empty is
    unsatisfied)."""
    import torch
    n = 40
    rng = np.random.default_rng(5)
    clauses, kept, weights = [], [], []
    bad = [0, n + 1, -(n + 1), 2 ** 31 - 1, -2 ** 31]
    for c in range(600):
        k = int(rng.integers(1, 6))
        cl = [int(v) * (1 if rng.random() < 0.5 else -1) for v in rng.integers(1, n + 1, k)]
        if c % 7 == 0:
            cl.append(cl[0])       # duplicate
        if c % 11 == 0:
            cl.append(-cl[0])      # tautology
        if c % 5 == 0:
            cl.insert(int(rng.integers(0, len(cl) + 1)), bad[c % len(bad)])
        if c % 97 == 0:
            cl = [bad[(c // 97) % len(bad)]]  # nothing valid left
        clauses.append(cl)
        kept.append([l for l in cl if l != 0 and -n <= l <= n])
        weights.append(int(rng.integers(1, 1000)))
    off = np.concatenate([[0], np.cumsum([len(c) for c in clauses])]).astype(np.int64)
    lits = np.array([l for c in clauses for l in c], np.int32)
    w = np.array(weights, np.int64)
    inst = oracle.Instance.from_clauses(n, kept, weights)
    stream = torch.cuda.Stream()
    off_d, lits_d, w_d = (_dev(torch, a, stream) for a in (off, lits, w))
    for B in (513, 64):
        X = rng.integers(0, 2, size=(B, n)).astype(np.uint8)
        X[X == 1] = rng.integers(1, 256, size=int((X == 1).sum()))  # any nonzero is True
        x_d = _dev(torch, X, stream)
        with torch.cuda.stream(stream):
            out = torch.full((B,), -1, dtype=torch.int64, device="cuda")
        ms.maxsat_eval_noalloc(n, off_d, lits_d, w_d, x_d, out, stream)
        stream.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.evaluate(inst, (X != 0).astype(np.uint8)))


def test_eval_noalloc_rejects_bad_requests(ms):
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
    # the binding refuses what the C entry point would trust blindly
    x1 = torch.zeros((4, 3), dtype=torch.uint8, device="cuda")
    c1 = torch.zeros(4, dtype=torch.int64, device="cuda")
    o1 = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    with pytest.raises(TypeError):
        ms.maxsat_eval_noalloc(3, o1.to(torch.int32), lits, None, x1, c1)
    with pytest.raises(ValueError):
        ms.maxsat_eval_noalloc(3, o1.cpu(), lits, None, x1, c1)
    with pytest.raises(ValueError):
        ms.maxsat_eval_noalloc(3, o1, lits, torch.ones(0, dtype=torch.int64, device="cuda"),
                               x1, c1)
    with pytest.raises(ValueError):
        ms.maxsat_eval_noalloc(3, o1, lits, None, x1, c1[:2])
