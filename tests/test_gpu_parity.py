"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs, the same clause-RBM parameters and the same seed.

Bar: costs, best costs, chain states and best assignments bit-exact; the free
energy within 1e-3 relative of the FP64 oracle; nu within the FP32 bound
derived from the update nu <- (1 - alpha) nu + alpha rho (1 - rho): each round
adds at most ~4 float32 rounding errors on a value <= 0.25 and shrinks older
errors by (1 - alpha), so |nu_gpu - nu_oracle| <= 4 * 2^-24 * 0.25 *
min(T, 1 / alpha) (plus the float32 rounding of alpha itself)."""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "or_rbm_params.txt")


def nu_tol(T, alpha):
    return 4 * 2.0 ** -24 * 0.25 * min(T, 1.0 / alpha) + 0.25 * abs(np.float32(alpha) - alpha) * T + 1e-9


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_02101_gb300 as m
    return m


@pytest.fixture(scope="module")
def stream(ms):
    import torch
    return torch.cuda.Stream()


@pytest.fixture(scope="module")
def small_table():
    """Lengths 1..4, one weight bucket, two temperatures (fitted by the oracle)."""
    return oracle.make_table([1, 2, 3, 4], [0.068, 0.528], n_buckets=1, iters=5000)


@pytest.fixture(scope="module")
def table3():
    """Length-3 sets fitted to convergence (20000 Adam iterations)."""
    return oracle.make_table([3], [0.068, 0.528], n_buckets=1, iters=20000)


@pytest.fixture(scope="module")
def golden_table():
    if not os.path.exists(GOLDEN):
        pytest.skip("golden parameter file missing")
    return oracle.RbmTable.load(GOLDEN)


def inst_of(gen):
    return oracle.Instance(*gen)


def make_ctx(ms, stream, inst, table, n_temps=2, n_buckets=1, alpha=0.01, spg=0, path=0,
             tune=0, up_device=1, vb=0, persist=0):
    params = ms.maxsat_default_params(sets=table.sets, n_temps=n_temps, n_buckets=n_buckets,
                                      alpha=alpha, steps_per_graph=spg, path=path,
                                      tune_blocks=tune, up_device=up_device, visible_batch=vb,
                                      persistent_round=persist)
    params.fstar = None
    return ms.maxsat_create(inst.n, inst.off, inst.lits, inst.w, params, stream)


def run_gpu(ms, stream, inst, table, B, T, seed, **kw):
    ctx = make_ctx(ms, stream, inst, table, **kw)
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, T)
    st = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    return st


def run_oracle(inst, table, B, T, seed, n_temps=2, n_buckets=1, alpha=0.01, chain_ids=None,
               B_total=None):
    st = oracle.init_chains(inst.n, B, seed, chain_ids=chain_ids, B_total=B_total)
    oracle.gibbs(inst, table, st, T, seed, n_temps=n_temps, n_buckets=n_buckets, alpha=alpha,
                 threads=os.cpu_count() or 4)
    return st


def assert_same(gpu, ora, T, alpha, rows=None):
    g = {k: (v if rows is None or np.ndim(v) == 0 else v[rows]) for k, v in gpu.items()}
    assert np.array_equal(g["x"], ora.x), "chain states"
    assert np.array_equal(g["best_cost"], ora.best_cost), "best costs"
    assert np.array_equal(g["best_x"], ora.best_x), "best assignments"
    assert np.array_equal(g["cost"], ora.cost), "costs"
    np.testing.assert_allclose(g["free_energy"], ora.free_energy, rtol=1e-3, atol=1e-6)
    assert np.max(np.abs(g["nu"] - ora.nu)) <= nu_tol(T, alpha)
    # the FP32 operation sequence of nu is reproduced exactly
    assert np.array_equal(g["nu"], ora.nu32), "nu (FP32 sequence)"


def edge_instance(seed=0, kmax=4, wmax=40):
    """Random clauses of lengths 1..kmax plus duplicates, a tautology, an empty
    clause, a variable in no clause, and weights spanning several buckets
    (kmax = 3: every clause has one-chunk tables and a 16-byte clause record)."""
    rng = np.random.default_rng(seed)
    n = 37
    lengths = rng.integers(1, kmax + 1, size=150)
    _, off, lits, _ = workloads.from_lengths(n - 1, lengths, rng)
    cl = [list(lits[off[c]:off[c + 1]]) for c in range(len(lengths))]
    cl += [[3, 3, -5], [7, -7], [], [12]] + ([[-2, -2, -2, 9]] if kmax >= 4 else [])
    w = list(rng.integers(1, wmax, size=len(cl)))
    return oracle.Instance.from_clauses(n, cl, w)


# --------------------------------------------------------------------------
# Exact cost evaluation (maxsat_eval)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("B", [1, 7, 300])
def test_eval_matches_oracle(ms, stream, small_table, B):
    import torch
    inst = edge_instance()
    ctx = make_ctx(ms, stream, inst, small_table)
    rng = np.random.default_rng(B)
    X = rng.integers(0, 2, size=(B, inst.n)).astype(np.uint8)
    X[0] *= 5  # any nonzero byte is True
    with torch.cuda.stream(stream):
        xd = torch.from_numpy(X).cuda()
        cd = torch.zeros(B, dtype=torch.int64, device="cuda")
    ms.maxsat_eval(ctx, xd, cd)
    stream.synchronize()
    expect = oracle.evaluate(inst, (X != 0).astype(np.uint8))
    assert np.array_equal(cd.cpu().numpy(), expect)
    ms.maxsat_destroy(ctx)


def test_eval_mixed_lengths_weighted(ms, stream, golden_table):
    import torch
    inst = inst_of(workloads.mixed_length(n=3000, m=15000, seed=3))
    ctx = make_ctx(ms, stream, inst, golden_table, n_buckets=4)
    B = 513
    X = np.random.default_rng(1).integers(0, 2, size=(B, inst.n)).astype(np.uint8)
    xd = torch.from_numpy(X).cuda()
    cd = torch.zeros(B, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    ms.maxsat_eval(ctx, xd, cd)
    stream.synchronize()
    assert np.array_equal(cd.cpu().numpy(), oracle.evaluate(inst, X))
    ms.maxsat_destroy(ctx)


@pytest.mark.parametrize("which", ["edge", "mixed12", "w3sat", "u3sat", "mixed-full"])
def test_dense_eval_matches_oracle(ms, stream, small_table, golden_table, which):
    """FP8 tensor-core gather (pattern-encoding matrix, tcgen05) against the
    literal-by-literal oracle: E4M3 operands up to length 9, E5M2 beyond."""
    import torch
    if which == "edge":
        inst, table, J, B = edge_instance(2), small_table, 1, 200
    elif which == "mixed12":
        inst, table, J, B = inst_of(workloads.mixed_length(n=1500, m=7000, seed=4)), golden_table, 4, 300
    elif which == "w3sat":
        inst, table, J, B = inst_of(workloads.weighted_3sat(1000, 6000, 1000, seed=0)), golden_table, 4, 4096
    elif which == "u3sat":  # unweighted: every 32-row group shares one weight
        inst, table, J, B = inst_of(workloads.random_ksat(300, 1290, 3, seed=8)), small_table, 1, 700
    else:  # mixed lengths 2..12 at full size: a 2 GB clause matrix, E5M2 operands
        inst, table, J, B = inst_of(workloads.mixed_length(seed=0)), golden_table, 4, 300
    ctx = make_ctx(ms, stream, inst, table, n_buckets=J, path=ms.MAXSAT_PATH_DENSE)
    assert ms.maxsat_get_path(ctx) == ms.MAXSAT_PATH_DENSE
    rng = np.random.default_rng(5)
    for rep in range(2):
        X = rng.integers(0, 2, size=(B, inst.n)).astype(np.uint8)
        with torch.cuda.stream(stream):
            xd = torch.from_numpy(X).cuda()
            cd = torch.full((B,), -1, dtype=torch.int64, device="cuda")
        ms.maxsat_eval(ctx, xd, cd)
        stream.synchronize()
        assert np.array_equal(cd.cpu().numpy(), oracle.evaluate(inst, X)), rep
    ms.maxsat_destroy(ctx)


@pytest.mark.parametrize("case", ["odd-n", "unaligned", "heavy", "batch-sizes"])
def test_dense_eval_layouts_and_batch_sizes(ms, stream, small_table, case):
    """The FP8 evaluation against the oracle: rows of n % 4 != 0 bytes, rows
    starting off a 4-byte boundary, 64-bit weight sums (total weight >=
    2^31), and one context evaluating several batch sizes in turn (a partial
    tile of one chain, growth of the scratch, smaller sizes after larger)."""
    import torch
    rng = np.random.default_rng(11)
    if case == "odd-n":
        inst, sizes = inst_of(workloads.random_ksat(333, 1500, 3, seed=2, wmax=90)), [257]
    elif case == "unaligned":
        inst, sizes = inst_of(workloads.random_ksat(400, 1700, 3, seed=3, wmax=90)), [300]
    elif case == "heavy":
        n_, off, lits, _ = workloads.random_ksat(500, 2000, 3, seed=4)
        w = rng.integers(1 << 38, 1 << 40, size=len(off) - 1).astype(np.int64)
        inst, sizes = oracle.Instance(n_, off, lits, w), [384]
    else:
        inst, sizes = inst_of(workloads.random_ksat(700, 3000, 3, seed=5, wmax=500)), \
            [1, 128, 129, 4096, 5, 1000]
    ctx = make_ctx(ms, stream, inst, small_table, path=ms.MAXSAT_PATH_DENSE)
    assert ms.maxsat_get_path(ctx) == ms.MAXSAT_PATH_DENSE
    for B in sizes:
        X = rng.integers(0, 2, size=(B, inst.n)).astype(np.uint8)
        with torch.cuda.stream(stream):
            if case == "unaligned":
                buf = torch.zeros(B * inst.n + 1, dtype=torch.uint8, device="cuda")
                xd = buf[1:].view(B, inst.n)
                xd.copy_(torch.from_numpy(X).cuda())
                assert xd.data_ptr() % 4 == 1
            else:
                xd = torch.from_numpy(X).cuda()
            cd = torch.full((B,), -1, dtype=torch.int64, device="cuda")
        ms.maxsat_eval(ctx, xd, cd)
        stream.synchronize()
        assert np.array_equal(cd.cpu().numpy(), oracle.evaluate(inst, X)), B
    ms.maxsat_destroy(ctx)


def test_dense_evals_back_to_back(ms, stream, small_table):
    """Consecutive dense evaluations overlap (the next conversion runs beside
    the previous product, into the other state buffer): five evaluations
    queued without a synchronisation, into separate cost arrays and, last,
    two into the same one, each against the oracle."""
    import torch
    inst = inst_of(workloads.random_ksat(400, 1700, 3, seed=7, wmax=60))
    ctx = make_ctx(ms, stream, inst, small_table, path=ms.MAXSAT_PATH_DENSE)
    assert ms.maxsat_get_path(ctx) == ms.MAXSAT_PATH_DENSE
    rng = np.random.default_rng(17)
    B = 520
    Xs = [rng.integers(0, 2, size=(B, inst.n)).astype(np.uint8) for _ in range(5)]
    with torch.cuda.stream(stream):
        xd = [torch.from_numpy(X).cuda() for X in Xs]
        cd = [torch.full((B,), -1, dtype=torch.int64, device="cuda") for _ in range(4)]
    stream.synchronize()
    for k in range(3):
        ms.maxsat_eval(ctx, xd[k], cd[k])
    ms.maxsat_eval(ctx, xd[3], cd[3])
    ms.maxsat_eval(ctx, xd[4], cd[3])  # the same cost array: the later evaluation wins
    stream.synchronize()
    for k in range(3):
        assert np.array_equal(cd[k].cpu().numpy(), oracle.evaluate(inst, Xs[k])), k
    assert np.array_equal(cd[3].cpu().numpy(), oracle.evaluate(inst, Xs[4]))
    ms.maxsat_destroy(ctx)


# --------------------------------------------------------------------------
# Gibbs trajectories
# --------------------------------------------------------------------------
@pytest.mark.parametrize("B", [256, 300])
def test_trajectory_3sat(ms, stream, small_table, B):
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    T, seed = 30, 11
    gpu = run_gpu(ms, stream, inst, small_table, B, T, seed)
    assert gpu["t"] == T
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed), T, 0.01)


@pytest.mark.parametrize("kmax", [3, 4])
def test_trajectory_edge_cases(ms, stream, small_table, kmax):
    inst = edge_instance(1, kmax)
    T, seed, B = 25, 3, 40
    gpu = run_gpu(ms, stream, inst, small_table, B, T, seed, alpha=0.05)
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed, alpha=0.05), T, 0.05)


def test_trajectory_edge_cases_heavy_weights(ms, stream, small_table):
    """Clauses of 1..3 literals and an empty one with weights up to 30000: a
    warp's clauses weigh more than 2^16, so the one-chunk gather keeps one
    32-bit cost per chain."""
    inst = edge_instance(2, 3, wmax=30000)
    T, seed, B = 25, 4, 64
    gpu = run_gpu(ms, stream, inst, small_table, B, T, seed)
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed), T, 0.01)


@pytest.mark.parametrize("w_hi", [32768, 32769])
def test_gather_cost_halves_at_the_16_bit_limit(ms, stream, small_table, w_hi):
    """16 clauses of 3 literals form one clause block whose warp k takes
    clauses k and k + 8, weighing 32767 and w_hi: warp sums of 65535 let two
    chains share a 32-bit cost register (a chain leaving both clauses
    unsatisfied fills its 16-bit half), 65536 does not."""
    rng = np.random.default_rng(21)
    n, off, lits, _ = workloads.from_lengths(12, np.full(16, 3), rng)
    w = np.array([32767] * 8 + [w_hi] * 8, dtype=np.int64)
    inst = oracle.Instance(n, off, lits, w)
    T, seed, B = 20, 7, 256
    gpu = run_gpu(ms, stream, inst, small_table, B, T, seed)
    ora = run_oracle(inst, small_table, B, T, seed)
    assert_same(gpu, ora, T, 0.01)
    # the first round's gather sees chains that leave both clauses of a warp
    # unsatisfied (initial states)
    x0 = oracle.init_chains(n, B, seed).x
    cl = inst.clauses()
    both = sum(int(np.sum(oracle.evaluate(oracle.Instance.from_clauses(n, [cl[k], cl[k + 8]]),
                                          x0) == 2)) for k in range(8))
    assert both > 0


def test_trajectory_mixed_weighted_buckets(ms, stream, golden_table):
    inst = inst_of(workloads.mixed_length(n=400, m=2000, seed=9))
    T, seed, B = 12, 5, 64
    gpu = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4)
    assert_same(gpu, run_oracle(inst, golden_table, B, T, seed, n_buckets=4), T, 0.01)


@pytest.fixture(scope="module")
def sat_table():
    """Lengths 3 (L = 3, one record chunk) and 5 (L = 6, two chunks) with unit
    0 forced on (b = 20: P = 65536 for every pattern) and the last unit
    forced off (b = -20: P = 0), so the saturated-threshold branch and the
    zero threshold both run."""
    base = oracle.make_table([3, 5], [0.068, 0.528], n_buckets=1, iters=3000)
    t = oracle.RbmTable()
    for s in base.sets:
        b = s["b"].copy()
        b[0], b[-1] = 20.0, -20.0
        t.add(s["len"], s["bucket"], s["temp"], s["W"], b, s["target"])
    return t


@pytest.mark.parametrize("path", [2, 1])
def test_saturated_hidden_units(ms, stream, sat_table, path):
    rng = np.random.default_rng(4)
    lengths = rng.choice([3, 5], size=400)
    n, off, lits, w = workloads.from_lengths(120, lengths, rng)
    inst = oracle.Instance(n, off, lits, w)
    # the tables really hold P = 65536 and P = 0
    for s in sat_table.sets:
        a_on = s["b"][0] + np.minimum(s["W"][:, 0], 0).sum()
        a_off = s["b"][-1] + np.maximum(s["W"][:, -1], 0).sum()
        assert np.rint(65536 / (1 + np.exp(-a_on))) == 65536
        assert np.rint(65536 / (1 + np.exp(-a_off))) == 0
    T, seed, B = 15, 9, 256
    gpu = run_gpu(ms, stream, inst, sat_table, B, T, seed, path=path)
    assert ms.MAXSAT_PATH_DENSE == 1 and ms.MAXSAT_PATH_SPARSE == 2
    assert_same(gpu, run_oracle(inst, sat_table, B, T, seed), T, 0.01)


def test_graph_replay_matches_plain_launches(ms, stream, small_table):
    inst = inst_of(workloads.random_ksat(60, 250, 3, seed=4, wmax=50))
    a = run_gpu(ms, stream, inst, small_table, 256, 23, 9, spg=0)
    b = run_gpu(ms, stream, inst, small_table, 256, 23, 9, spg=5)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_resume_is_bit_identical(ms, stream, small_table):
    inst = inst_of(workloads.random_ksat(60, 250, 3, seed=4, wmax=50))
    whole = run_gpu(ms, stream, inst, small_table, 256, 20, 13, spg=4)
    ctx = make_ctx(ms, stream, inst, small_table, spg=4)
    ms.maxsat_reset(ctx, 256, 13)
    ms.maxsat_step(ctx, 9)
    mid = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    ctx = make_ctx(ms, stream, inst, small_table, spg=4)
    ms.maxsat_set_state(ctx, 256, 13, mid["x"], mid["nu"], mid["best_cost"], mid["best_x"], mid["t"])
    ms.maxsat_step(ctx, 11)
    end = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    for k in ["x", "nu", "best_cost", "best_x", "cost", "free_energy"]:
        assert np.array_equal(whole[k], end[k]), k


def test_solve_matches_oracle(ms, stream, small_table):
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    ctx = make_ctx(ms, stream, inst, small_table, spg=16)
    cost, assign = ms.maxsat_solve(ctx, 256, 40, 21)
    st = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    ob, ox, ost = oracle.solve(inst, small_table, 256, 40, 21, n_temps=2,
                               threads=os.cpu_count() or 4)
    assert cost == ob and np.array_equal(assign, ox)
    assert np.array_equal(st["best_cost"], ost.best_cost)
    assert np.array_equal(st["best_x"], ost.best_x)
    assert oracle.evaluate(inst, assign[None])[0] == cost


def test_solve_timed_is_solve_of_the_rounds_it_ran(ms, stream, small_table):
    """The wall-clock budget only decides how many rounds run: with max_steps
    reached first the result is maxsat_solve's (and the oracle's) of those
    rounds; with a short budget it stops after whole chunks and equals
    maxsat_solve of the rounds it reports."""
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    ctx = make_ctx(ms, stream, inst, small_table, spg=16)
    cost, assign, done = ms.maxsat_solve_timed(ctx, 256, 60.0, 21, max_steps=40, chunk=16)
    assert done == 40
    ob, ox, _ = oracle.solve(inst, small_table, 256, 40, 21, n_temps=2,
                             threads=os.cpu_count() or 4)
    assert cost == ob and np.array_equal(assign, ox)
    cost2, assign2, done2 = ms.maxsat_solve_timed(ctx, 256, 0.02, 5, chunk=8)
    assert done2 >= 8 and done2 % 8 == 0
    ref, ref_assign = ms.maxsat_solve(ctx, 256, done2, 5)
    assert cost2 == ref and np.array_equal(assign2, ref_assign)
    c0, _, d0 = ms.maxsat_solve_timed(ctx, 256, 0.0, 5)
    assert d0 == 0 and c0 == ms.maxsat_solve(ctx, 256, 0, 5)[0]
    with pytest.raises(ms.MaxsatError):
        ms.maxsat_solve_timed(ctx, 256, -1.0, 5)
    ms.maxsat_destroy(ctx)


def test_brute_force_twin(ms, stream, table3):
    inst = inst_of(workloads.random_ksat(18, 77, 3, seed=0))
    ctx = make_ctx(ms, stream, inst, table3, spg=50)
    cost, assign = ms.maxsat_solve(ctx, 256, 200, 0)
    ms.maxsat_destroy(ctx)
    assert cost == oracle.brute_force_optimum(inst)
    assert oracle.evaluate(inst, assign[None])[0] == cost


def test_step_before_reset_is_an_error(ms, stream, small_table):
    inst = inst_of(workloads.random_ksat(10, 20, 3, seed=0))
    ctx = make_ctx(ms, stream, inst, small_table)
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_step(ctx, 1)
    assert e.value.code == ms.MAXSAT_ESTATE
    ms.maxsat_destroy(ctx)


# --------------------------------------------------------------------------
# Full sizes, in the launch configuration the benchmark times: sampled chains
# recomputed by the oracle one by one (chains are independent)
# --------------------------------------------------------------------------
def test_full_size_weighted_3sat_sampled(ms, stream, golden_table):
    inst = inst_of(workloads.weighted_3sat(1000, 6000, 1000, seed=0))
    B, T, seed = 4096, 6, 1
    gpu = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4, spg=3)
    rows = np.array([0, 1, 7, 8, 2047, 2048, 3000, 4095])
    ora = run_oracle(inst, golden_table, len(rows), T, seed, n_buckets=4, chain_ids=rows,
                     B_total=B)
    assert_same(gpu, ora, T, 0.01, rows=rows)


def test_full_size_mixed_sampled(ms, stream, golden_table):
    inst = inst_of(workloads.mixed_length(seed=0))
    B, T, seed = 1024, 3, 2
    gpu = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4, spg=0)
    rows = np.array([0, 255, 511, 512, 1023])
    ora = run_oracle(inst, golden_table, len(rows), T, seed, n_buckets=4, chain_ids=rows,
                     B_total=B)
    assert_same(gpu, ora, T, 0.01, rows=rows)


def test_full_size_mixed_dense_sampled(ms, stream, golden_table):
    """Mixed lengths at full size on the dense path (a 2 GB FP8 clause matrix,
    E5M2 above length 9, 16-bit hidden patterns): sampled chains against the
    oracle, as on the sparse path."""
    inst = inst_of(workloads.mixed_length(seed=0))
    B, T, seed = 1024, 3, 2
    gpu = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4, spg=0,
                  path=ms.MAXSAT_PATH_DENSE)
    rows = np.array([0, 255, 511, 512, 1023])
    ora = run_oracle(inst, golden_table, len(rows), T, seed, n_buckets=4, chain_ids=rows,
                     B_total=B)
    assert_same(gpu, ora, T, 0.01, rows=rows)


# --------------------------------------------------------------------------
# Dense tensor-core Gibbs round: the same contract, so the same trajectory
# --------------------------------------------------------------------------
@pytest.mark.parametrize("B", [256, 300])
def test_dense_trajectory_3sat(ms, stream, small_table, B):
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    T, seed = 20, 11
    gpu = run_gpu(ms, stream, inst, small_table, B, T, seed, path=ms.MAXSAT_PATH_DENSE)
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed), T, 0.01)


def test_dense_trajectory_mixed_weighted(ms, stream, golden_table):
    """Lengths up to 12: E5M2 gather operands, 13 hidden units (16-bit hidden
    patterns), four weight buckets."""
    inst = inst_of(workloads.mixed_length(n=400, m=2000, seed=9))
    T, seed, B = 8, 5, 64
    gpu = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4,
                  path=ms.MAXSAT_PATH_DENSE)
    assert_same(gpu, run_oracle(inst, golden_table, B, T, seed, n_buckets=4), T, 0.01)


def test_dense_equals_sparse_full_size(ms, stream, golden_table):
    inst = inst_of(workloads.weighted_3sat(1000, 6000, 1000, seed=0))
    B, T, seed = 4096, 6, 3
    d = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4, spg=3,
                path=ms.MAXSAT_PATH_DENSE)
    s = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4, spg=3,
                path=ms.MAXSAT_PATH_SPARSE)
    for k in ["x", "best_cost", "best_x", "cost"]:
        assert np.array_equal(d[k], s[k]), k
    np.testing.assert_allclose(d["free_energy"], s["free_energy"], rtol=1e-3)
    assert np.max(np.abs(d["nu"] - s["nu"])) <= nu_tol(T, 0.01)
    rows = np.array([0, 9, 2047, 2048, 4095])
    ora = run_oracle(inst, golden_table, len(rows), T, seed, n_buckets=4, chain_ids=rows, B_total=B)
    assert_same(d, ora, T, 0.01, rows=rows)


def test_dense_solve_and_resume(ms, stream, small_table):
    inst = inst_of(workloads.random_ksat(60, 250, 3, seed=4, wmax=50))
    ctx = make_ctx(ms, stream, inst, small_table, spg=8, path=ms.MAXSAT_PATH_DENSE)
    cost, assign = ms.maxsat_solve(ctx, 256, 30, 21)
    ms.maxsat_destroy(ctx)
    ob, ox, _ = oracle.solve(inst, small_table, 256, 30, 21, n_temps=2, threads=os.cpu_count() or 4)
    assert cost == ob and np.array_equal(assign, ox)
    whole = run_gpu(ms, stream, inst, small_table, 256, 20, 13, spg=4, path=ms.MAXSAT_PATH_DENSE)
    ctx = make_ctx(ms, stream, inst, small_table, spg=4, path=ms.MAXSAT_PATH_DENSE)
    ms.maxsat_reset(ctx, 256, 13)
    ms.maxsat_step(ctx, 9)
    mid = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    ctx = make_ctx(ms, stream, inst, small_table, spg=4, path=ms.MAXSAT_PATH_DENSE)
    ms.maxsat_set_state(ctx, 256, 13, mid["x"], mid["nu"], mid["best_cost"], mid["best_x"], mid["t"])
    ms.maxsat_step(ctx, 11)
    end = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    for k in ["x", "nu", "best_cost", "best_x", "cost", "free_energy"]:
        assert np.array_equal(whole[k], end[k]), k


def test_auto_path_choice_is_measured_and_consistent(ms, stream, golden_table):
    """MAXSAT_PATH_AUTO: the reset times both paths and keeps one; the chains
    it then runs follow the same contract (sampled chains vs the oracle)."""
    inst = inst_of(workloads.weighted_3sat(1000, 6000, 1000, seed=0))
    B, T, seed = 1024, 4, 8
    gpu = run_gpu(ms, stream, inst, golden_table, B, T, seed, n_buckets=4, spg=2,
                  path=ms.MAXSAT_PATH_AUTO)
    rows = np.array([0, 511, 512, 1023])
    ora = run_oracle(inst, golden_table, len(rows), T, seed, n_buckets=4, chain_ids=rows, B_total=B)
    assert_same(gpu, ora, T, 0.01, rows=rows)
    ctx = make_ctx(ms, stream, inst, golden_table, n_buckets=4, path=ms.MAXSAT_PATH_AUTO)
    ms.maxsat_reset(ctx, B, seed)
    assert ms.maxsat_get_path(ctx) in (ms.MAXSAT_PATH_DENSE, ms.MAXSAT_PATH_SPARSE)
    ms.maxsat_destroy(ctx)


@pytest.mark.parametrize("path", ["sparse", "dense"])
def test_chain_shards_reproduce_one_run(ms, stream, small_table, path):
    """Two shards of 256 chains (global chains 0..255 and 256..511 of 512) run
    exactly the chains of one 512-chain run: draws and temperature blocks
    follow the global chain index."""
    code = ms.MAXSAT_PATH_DENSE if path == "dense" else ms.MAXSAT_PATH_SPARSE
    inst = inst_of(workloads.random_ksat(80, 340, 3, seed=6, wmax=20))
    T, seed = 12, 77
    whole = run_gpu(ms, stream, inst, small_table, 512, T, seed, spg=4, path=code)
    for r in range(2):
        ctx = make_ctx(ms, stream, inst, small_table, spg=4, path=code)
        ms.maxsat_reset_shard(ctx, 256, seed, 256 * r, 512)
        ms.maxsat_step(ctx, T)
        part = ms.maxsat_get_state(ctx)
        ms.maxsat_destroy(ctx)
        sl = slice(256 * r, 256 * r + 256)
        for k in ["x", "best_cost", "best_x", "cost", "nu", "free_energy"]:
            assert np.array_equal(part[k], whole[k][sl]), (k, r)


# --------------------------------------------------------------------------
# Batches of formulas (maxsat_create_batch): every formula against the oracle
# run alone with its batch index
# --------------------------------------------------------------------------
def small_batch(seed=3):
    rng = np.random.default_rng(seed)
    insts = workloads.ragged_batch(count=9, n_lo=12, n_hi=160, seed=seed)
    # a formula without clauses and one with an empty clause and a tautology
    insts.insert(4, (7, np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64)))
    cl = [[1, -2, 3], [], [4, -4], [2, 5, -6]] + [list(rng.choice([-1, 1], 3) * (rng.permutation(6)[:3] + 1))
                                                 for _ in range(30)]
    e = oracle.Instance.from_clauses(6, cl, list(rng.integers(1, 50, size=len(cl))))
    insts.insert(7, (e.n, e.off, e.lits, e.w))
    return insts


def batch_ctx(ms, stream, insts, table, n_buckets=4, alpha=0.01, up_device=1, persist=0,
              spg=100):
    params = ms.maxsat_default_params(sets=table.sets, n_temps=2, n_buckets=n_buckets,
                                      alpha=alpha, up_device=up_device,
                                      persistent_round=persist, steps_per_graph=spg)
    params.fstar = None
    return ms.maxsat_create_batch(insts, params, stream)


@pytest.mark.parametrize("B", [256, 300])
def test_batch_trajectories_match_oracle(ms, stream, golden_table, B):
    insts = small_batch()
    T, seed = 9, 17
    ctx = batch_ctx(ms, stream, insts, golden_table)
    assert ms.maxsat_get_n_instances(ctx) == len(insts)
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, T)
    g = ms.maxsat_get_state(ctx)
    vb = ctx.var_base
    for k, (n, off, lits, w) in enumerate(insts):
        inst = oracle.Instance(n, off, lits, w)
        st = oracle.init_chains(n, B, seed, instance=k)
        oracle.gibbs(inst, golden_table, st, T, seed, n_temps=2, n_buckets=4,
                     threads=os.cpu_count() or 4)
        sl = slice(int(vb[k]), int(vb[k + 1]))
        assert np.array_equal(g["x"][:, sl], st.x), k
        assert np.array_equal(g["best_x"][:, sl], st.best_x), k
        assert np.array_equal(g["best_cost"][k], st.best_cost), k
        assert np.array_equal(g["cost"][k], st.cost), k
        np.testing.assert_allclose(g["free_energy"][k], st.free_energy, rtol=1e-3, atol=1e-6)
        assert np.max(np.abs(g["nu"][:, sl] - st.nu)) <= nu_tol(T, 0.01)
        assert np.array_equal(g["nu"][:, sl], st.nu32), k
    ms.maxsat_destroy(ctx)


def test_batch_eval_and_solve_match_oracle(ms, stream, golden_table):
    import torch
    insts = small_batch(5)
    ctx = batch_ctx(ms, stream, insts, golden_table)
    rng = np.random.default_rng(2)
    B = 37
    a = rng.integers(0, 2, size=(B, ctx.n)).astype(np.uint8)
    cost = torch.zeros(len(insts) * B, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(stream):
        ms.maxsat_eval(ctx, torch.tensor(a, device="cuda"), cost)
    stream.synchronize()
    cost = cost.cpu().numpy().reshape(len(insts), B)
    vb = ctx.var_base
    for k, (n, off, lits, w) in enumerate(insts):
        ref = oracle.evaluate(oracle.Instance(n, off, lits, w), a[:, vb[k]:vb[k + 1]])
        assert np.array_equal(cost[k], ref), k
    T, seed, Bs = 12, 8, 64
    best, assign = ms.maxsat_solve(ctx, Bs, T, seed)
    for k, (n, off, lits, w) in enumerate(insts):
        inst = oracle.Instance(n, off, lits, w)
        c, x, _ = oracle.solve(inst, golden_table, Bs, T, seed, n_temps=2, n_buckets=4,
                               threads=os.cpu_count() or 4, instance=k)
        assert best[k] == c, k
        assert np.array_equal(assign[vb[k]:vb[k + 1]], x), k
        assert oracle.evaluate(inst, assign[None, vb[k]:vb[k + 1]])[0] == c
    ms.maxsat_destroy(ctx)


def test_batch_full_size_sampled(ms, stream, golden_table):
    """512 formulas, n log-uniform in [100, 5000], m / n in [4, 8], B = 256:
    the first, middle and last formulas, the smallest and the largest, and
    the ones with the lowest and highest clause ratio recomputed by the
    oracle."""
    insts = workloads.ragged_batch(seed=0)
    B, T, seed = 256, 4, 23
    ctx = batch_ctx(ms, stream, insts, golden_table)
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, T)
    g = ms.maxsat_get_state(ctx)
    vb = ctx.var_base
    ns = np.array([i[0] for i in insts])
    ratio = np.array([(len(i[1]) - 1) / i[0] for i in insts])
    picks = sorted({0, 255, 511, int(np.argmin(ns)), int(np.argmax(ns)), int(np.argmin(ratio)),
                    int(np.argmax(ratio))})
    for k in picks:
        n, off, lits, w = insts[k]
        inst = oracle.Instance(n, off, lits, w)
        st = oracle.init_chains(n, B, seed, instance=k)
        oracle.gibbs(inst, golden_table, st, T, seed, n_temps=2, n_buckets=4,
                     threads=os.cpu_count() or 4)
        sl = slice(int(vb[k]), int(vb[k + 1]))
        assert np.array_equal(g["x"][:, sl], st.x), k
        assert np.array_equal(g["best_cost"][k], st.best_cost), k
        assert np.array_equal(g["cost"][k], st.cost), k
    ms.maxsat_destroy(ctx)


@pytest.mark.parametrize("vb,kmax", [(2, 3), (8, 3), (2, 4), (8, 4)])
def test_visible_batches_keep_parity(ms, stream, small_table, vb, kmax):
    """Every load batch of the visible update (2 and 8 beside the default 4
    of the other tests) gives the oracle's trajectory, on one-chunk (kmax 3)
    and multi-chunk tables."""
    inst = edge_instance(5, kmax)
    T, seed, B = 20, 6, 300
    ctx = make_ctx(ms, stream, inst, small_table, vb=vb)
    assert ms.maxsat_get_visible_batch(ctx) == vb
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, T)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed), T, 0.01)


def test_visible_batch_is_checked(ms, stream, small_table):
    inst = edge_instance(5, 3)
    with pytest.raises(ms.MaxsatError):
        make_ctx(ms, stream, inst, small_table, vb=3)


def test_measured_clause_blocks_keep_parity(ms, stream, golden_table):
    """With tune_blocks the gather's clause-block size and then the visible
    update's load batch are measured at the first reset; the trajectory is
    the oracle's whatever shape wins."""
    inst = inst_of(workloads.mixed_length(n=400, m=2000, seed=9))
    T, seed, B = 10, 5, 512
    ctx = make_ctx(ms, stream, inst, golden_table, n_buckets=4, path=ms.MAXSAT_PATH_SPARSE,
                   tune=1, spg=4)
    ms.maxsat_reset(ctx, B, seed)
    cb = ms.maxsat_get_clause_block(ctx)
    assert cb >= 16
    assert ms.maxsat_get_visible_batch(ctx) in (2, 4, 8)
    ms.maxsat_step(ctx, T)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    assert_same(gpu, run_oracle(inst, golden_table, B, T, seed, n_buckets=4), T, 0.01)


# --------------------------------------------------------------------------
# Unit-propagation heuristic (maxsat_up_begin / maxsat_up_end, Sec. 4.4)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("path,up_device", [("sparse", 1), ("sparse", 0), ("dense", 1)])
def test_unit_propagation_round_matches_oracle(ms, stream, golden_table, path, up_device):
    """reset, T1 rounds, send for propagation, upw rounds while it works,
    fetch + B-of-2B merge, T2 rounds: the oracle's same sequence (its FP32
    nu ranks the variables) gives the same chains bit for bit. Propagation
    and merge on the GPU (sparse path, up_device 1) or on host threads
    (up_device 0, and the dense path)."""
    inst = inst_of(workloads.weighted_3sat(300, 1500, 1000, seed=4))
    B, T1, upw, T2, seed = 256, 6, 3, 5, 13
    path = {"sparse": ms.MAXSAT_PATH_SPARSE, "dense": ms.MAXSAT_PATH_DENSE}[path]
    ctx = make_ctx(ms, stream, inst, golden_table, n_buckets=4, path=path, spg=2,
                   up_device=up_device)
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, T1)
    ms.maxsat_up_begin(ctx)
    ms.maxsat_step(ctx, upw)
    ms.maxsat_up_end(ctx)
    ms.maxsat_step(ctx, T2)
    gpu = ms.maxsat_get_state(ctx)
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_up_end(ctx)
    assert e.value.code == ms.MAXSAT_ESTATE
    ms.maxsat_destroy(ctx)

    st = oracle.init_chains(inst.n, B, seed)
    kw = dict(n_temps=2, n_buckets=4, threads=os.cpu_count() or 4)
    oracle.gibbs(inst, golden_table, st, T1, seed, **kw)
    up_x = oracle.unit_prop(inst, st.x, st.nu32)
    oracle.gibbs(inst, golden_table, st, upw, seed, **kw)
    before = evaluate_min(inst, st.x)
    oracle.up_merge(inst, st, up_x)
    assert evaluate_min(inst, st.x) <= before
    oracle.gibbs(inst, golden_table, st, T2, seed, **kw)
    assert_same(gpu, st, T1 + upw + T2, 0.01)


def evaluate_min(inst, x):
    return int(oracle.evaluate(inst, x).min())


@pytest.mark.parametrize("up_device", [1, 0])
def test_unit_propagation_edge_cases_two_rounds(ms, stream, small_table, up_device):
    """Duplicate literals, a tautology, an empty clause, a variable in no
    clause, B not a multiple of 256, and two propagation rounds in a row
    (the second as maxsat_up): the same chains as the oracle."""
    inst = edge_instance(1, 4)
    B, seed, alpha = 300, 5, 0.05
    ctx = make_ctx(ms, stream, inst, small_table, alpha=alpha, path=ms.MAXSAT_PATH_SPARSE, spg=2,
                   up_device=up_device)
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, 4)
    ms.maxsat_up_begin(ctx)
    ms.maxsat_step(ctx, 2)
    ms.maxsat_up_end(ctx)
    ms.maxsat_step(ctx, 3)
    ms.maxsat_up(ctx)
    ms.maxsat_step(ctx, 2)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)

    st = oracle.init_chains(inst.n, B, seed)
    kw = dict(n_temps=2, n_buckets=1, alpha=alpha, threads=os.cpu_count() or 4)
    oracle.gibbs(inst, small_table, st, 4, seed, **kw)
    up_x = oracle.unit_prop(inst, st.x, st.nu32)
    oracle.gibbs(inst, small_table, st, 2, seed, **kw)
    oracle.up_merge(inst, st, up_x)
    oracle.gibbs(inst, small_table, st, 3, seed, **kw)
    oracle.up_merge(inst, st, oracle.unit_prop(inst, st.x, st.nu32))
    oracle.gibbs(inst, small_table, st, 2, seed, **kw)
    assert_same(gpu, st, 11, alpha)


def test_unit_propagation_large_formula_takes_the_host_form(ms, stream, golden_table):
    """n = 17000 (a chain's ranking state would need 279 KB of shared
    memory): the round runs on host threads and still equals the oracle."""
    inst = inst_of(workloads.weighted_3sat(17000, 68000, 1000, seed=8))
    B, seed = 64, 17
    ctx = make_ctx(ms, stream, inst, golden_table, n_buckets=4, path=ms.MAXSAT_PATH_SPARSE, spg=2,
                   up_device=1)
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, 3)
    ms.maxsat_up(ctx)
    ms.maxsat_step(ctx, 2)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    st = oracle.init_chains(inst.n, B, seed)
    kw = dict(n_temps=2, n_buckets=4, threads=os.cpu_count() or 4)
    oracle.gibbs(inst, golden_table, st, 3, seed, **kw)
    oracle.up_merge(inst, st, oracle.unit_prop(inst, st.x, st.nu32))
    oracle.gibbs(inst, golden_table, st, 2, seed, **kw)
    assert_same(gpu, st, 5, 0.01)


def test_unit_propagation_of_a_batch_needs_the_gpu_form(ms, stream, golden_table):
    insts = small_batch()
    ctx = batch_ctx(ms, stream, insts, golden_table, up_device=0)
    ms.maxsat_reset(ctx, 64, 1)
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_up(ctx)
    assert e.value.code == ms.MAXSAT_EINVAL
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_up_end(ctx)
    assert e.value.code == ms.MAXSAT_ESTATE
    ms.maxsat_destroy(ctx)


@pytest.mark.parametrize("B", [256, 300])
def test_batch_unit_propagation_and_flips_match_oracle(ms, stream, golden_table, B):
    """A batch of 11 formulas (one without clauses, one with an empty clause
    and a tautology): rounds, a unit-propagation round sent and merged 2
    rounds later, rounds, a flip-proposal merge, rounds; every formula equals
    the oracle run alone with its batch index."""
    insts = small_batch()
    seed = 23
    ctx = batch_ctx(ms, stream, insts, golden_table)
    n_all = int(ctx.var_base[-1])
    prob = np.random.default_rng(5).random(n_all).astype(np.float32)
    tau = 0.2
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, 4)
    ms.maxsat_up_begin(ctx)
    ms.maxsat_step(ctx, 2)
    ms.maxsat_up_end(ctx)
    ms.maxsat_step(ctx, 3)
    ms.maxsat_propose_flips(ctx, prob, tau)
    ms.maxsat_step(ctx, 2)
    g = ms.maxsat_get_state(ctx)
    vb = ctx.var_base
    ms.maxsat_destroy(ctx)
    kw = dict(n_temps=2, n_buckets=4, threads=os.cpu_count() or 4)
    for k, (n, off, lits, w) in enumerate(insts):
        inst = oracle.Instance(n, off, lits, w)
        sl = slice(int(vb[k]), int(vb[k + 1]))
        st = oracle.init_chains(n, B, seed, instance=k)
        oracle.gibbs(inst, golden_table, st, 4, seed, **kw)
        up_x = oracle.unit_prop(inst, st.x, st.nu32)
        oracle.gibbs(inst, golden_table, st, 2, seed, **kw)
        oracle.up_merge(inst, st, up_x)
        oracle.gibbs(inst, golden_table, st, 3, seed, **kw)
        oracle.up_merge(inst, st, oracle.flip_proposals(st.x, prob[sl], tau))
        oracle.gibbs(inst, golden_table, st, 2, seed, **kw)
        assert np.array_equal(g["x"][:, sl], st.x), k
        assert np.array_equal(g["best_cost"][k], st.best_cost), k
        assert np.array_equal(g["nu"][:, sl], st.nu32), k


# --------------------------------------------------------------------------
# Parallel tempering (maxsat_pt_swap) with a 4-temperature ensemble
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def table4():
    """Length 3, two weight buckets, four temperatures."""
    return oracle.make_table([3], [0.05, 0.15, 0.4, 0.9], n_buckets=2, iters=3000)


def test_parallel_tempering_matches_oracle(ms, stream, table4):
    inst = inst_of(workloads.weighted_3sat(200, 900, 8, seed=6))
    B, seed = 256, 21
    ctx = make_ctx(ms, stream, inst, table4, n_temps=4, n_buckets=2,
                   path=ms.MAXSAT_PATH_SPARSE, spg=3)
    ms.maxsat_reset(ctx, B, seed)
    st = oracle.init_chains(inst.n, B, seed)
    kw = dict(n_temps=4, n_buckets=2, threads=os.cpu_count() or 4)
    swaps = []
    for steps, parity in ((4, 0), (3, 1), (5, 0), (2, 1)):
        ms.maxsat_step(ctx, steps)
        oracle.gibbs(inst, table4, st, steps, seed, **kw)
        got = ms.maxsat_pt_swap(ctx, parity)
        want = oracle.pt_swap(inst, table4, st, seed, parity, n_temps=4, n_buckets=2)
        assert got == want
        swaps.append(got)
    ms.maxsat_step(ctx, 3)
    oracle.gibbs(inst, table4, st, 3, seed, **kw)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    assert sum(swaps) > 0
    assert_same(gpu, st, 17, 0.01)


def test_parallel_tempering_rejects_bad_ensembles(ms, stream, table4):
    inst = inst_of(workloads.weighted_3sat(100, 400, 8, seed=6))
    ctx = make_ctx(ms, stream, inst, table4, n_temps=4, n_buckets=2, path=ms.MAXSAT_PATH_SPARSE)
    ms.maxsat_reset(ctx, 100, 1)  # 100 = 4 x 25, 25 not a multiple of 8
    with pytest.raises(ms.MaxsatError) as e:
        ms.maxsat_pt_swap(ctx, 0)
    assert e.value.code == ms.MAXSAT_EINVAL
    ms.maxsat_destroy(ctx)


# --------------------------------------------------------------------------
# Persistent round (params.persistent_round): one cooperative launch of
# several rounds, grid barriers between the gather and the visible update
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["3sat", "edge", "heavy"])
def test_persistent_round_matches_oracle(ms, stream, small_table, case):
    """3-literal formulas, clauses of 0..3 literals with duplicates and a
    tautology, and heavy weights (one 32-bit cost per chain) each take the
    persistent round; 30 rounds in launches of 7 (a ragged last launch)
    follow the oracle's trajectory."""
    inst = {"3sat": lambda: inst_of(workloads.random_ksat(50, 215, 3, seed=0)),
            "edge": lambda: edge_instance(1, 3),
            "heavy": lambda: edge_instance(2, 3, wmax=30000)}[case]()
    T, seed, B = 30, 11, 256
    ctx = make_ctx(ms, stream, inst, small_table, alpha=0.05, spg=7, persist=1)
    ms.maxsat_reset(ctx, B, seed)
    assert ms.maxsat_get_persistent_round(ctx) == 1
    ms.maxsat_step(ctx, 12)
    ms.maxsat_step(ctx, T - 12)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    assert gpu["t"] == T
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed, alpha=0.05), T, 0.05)


def test_persistent_round_falls_back_where_it_does_not_apply(ms, stream, small_table):
    """4-literal clauses (multi-chunk tables) and octets that straddle a
    temperature block (B = 300) keep the two-launch round, with the same
    results."""
    inst = edge_instance(1, 4)
    ctx = make_ctx(ms, stream, inst, small_table, persist=1)
    ms.maxsat_reset(ctx, 256, 3)
    assert ms.maxsat_get_persistent_round(ctx) == 0
    ms.maxsat_destroy(ctx)
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    T, seed, B = 10, 4, 300
    ctx = make_ctx(ms, stream, inst, small_table, spg=4, persist=1)
    ms.maxsat_reset(ctx, B, seed)
    assert ms.maxsat_get_persistent_round(ctx) == 0
    ms.maxsat_step(ctx, T)
    gpu = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    assert_same(gpu, run_oracle(inst, small_table, B, T, seed), T, 0.01)


def test_persistent_batch_matches_oracle(ms, stream, golden_table):
    """The 11-formula batch (one formula without clauses, one with an empty
    clause and a tautology) at B = 256: every formula follows the oracle
    run alone with its batch index."""
    insts = small_batch()
    T, seed, B = 9, 17, 256
    ctx = batch_ctx(ms, stream, insts, golden_table, persist=1, spg=4)
    ms.maxsat_reset(ctx, B, seed)
    assert ms.maxsat_get_persistent_round(ctx) == 1
    ms.maxsat_step(ctx, T)
    g = ms.maxsat_get_state(ctx)
    vb = ctx.var_base
    for k, (n, off, lits, w) in enumerate(insts):
        inst = oracle.Instance(n, off, lits, w)
        st = oracle.init_chains(n, B, seed, instance=k)
        oracle.gibbs(inst, golden_table, st, T, seed, n_temps=2, n_buckets=4,
                     threads=os.cpu_count() or 4)
        sl = slice(int(vb[k]), int(vb[k + 1]))
        assert np.array_equal(g["x"][:, sl], st.x), k
        assert np.array_equal(g["best_x"][:, sl], st.best_x), k
        assert np.array_equal(g["best_cost"][k], st.best_cost), k
        assert np.array_equal(g["cost"][k], st.cost), k
        np.testing.assert_allclose(g["free_energy"][k], st.free_energy, rtol=1e-3, atol=1e-6)
        assert np.array_equal(g["nu"][:, sl], st.nu32), k
    ms.maxsat_destroy(ctx)


def _state_of_rounds(ms, stream, make, B, T, seed, chunks):
    ctx = make()
    ms.maxsat_reset(ctx, B, seed)
    persistent = ms.maxsat_get_persistent_round(ctx)
    for c in chunks:
        ms.maxsat_step(ctx, c)
    g = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    return persistent, g


@pytest.mark.parametrize("workload", ["w3sat-n1000-m6000", "ragged-512"])
def test_persistent_equals_two_launch_full_size(ms, stream, golden_table, workload):
    """At full size, in the launch configurations the bench times (weighted
    3-SAT n = 1000, m = 6000, 4096 chains; 512 formulas of 256 chains each),
    the persistent round and the graph-replayed two-launch round give the
    same states, costs, best-so-far, nu and free energies, bit for bit."""
    spec = workloads.WORKLOADS[workload]
    B, T, seed = spec["B"], 7, 5
    if spec.get("batch"):
        insts = spec["gen"](0)
        make = lambda p: batch_ctx(ms, stream, insts, golden_table, persist=p, spg=3)
    else:
        inst = inst_of(spec["gen"](0))
        make = lambda p: make_ctx(ms, stream, inst, golden_table, n_buckets=4, spg=3, persist=p)
    p0, two = _state_of_rounds(ms, stream, lambda: make(0), B, T, seed, (T,))
    p1, per = _state_of_rounds(ms, stream, lambda: make(1), B, T, seed, (2, T - 2))
    assert (p0, p1) == (0, 1)
    for k in ["x", "best_cost", "best_x", "cost", "free_energy", "nu"]:
        assert np.array_equal(two[k], per[k]), k
