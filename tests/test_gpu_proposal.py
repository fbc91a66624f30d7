"""GPU parity of the learned proposal: the library's hand-written forward and
backward kernels against the FP64 oracle (oracle/proposal.py) with the same
BF16-rounded weights, training progress, and the biased chain start.

Bar: loss within 1e-5 relative, probabilities within 1e-5 absolute, gradient
within 1e-3 relative per element of the largest gradient magnitude (FP32
activations and sums against FP64, the same BF16 weights)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import proposal as mpo

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


@pytest.fixture(scope="module")
def stream(ms):
    import torch
    return torch.cuda.Stream()


def formula(seed=2, n=300, m=1300):
    n0, off, lits, w = workloads.weighted_3sat(n, m, 1000, seed=seed)
    lits = np.asarray(lits).copy()
    lits[1] = lits[0]  # a repeated literal
    return n0 + 1, off, lits, w  # and a variable in no clause


def ctx_for(ms, stream, n, off, lits, w):
    return ms.maxsat_create(n, off, lits, w, ms.maxsat_default_params(fit_iters=2000), stream)


@pytest.mark.parametrize("layers", [1, 3])
def test_gradient_matches_oracle(ms, stream, layers):
    import torch
    n, off, lits, w = formula()
    ctx = ctx_for(ms, stream, n, off, lits, w)
    model = ms.maxsat_mp_create(layers, seed=5)
    rng = np.random.default_rng(0)
    theta = (mpo.init_params(seed=1, L=layers) + rng.normal(0, 0.02, mpo.n_params(layers))
             ).astype(np.float32)
    ms.maxsat_mp_set_params(model, theta)
    y = rng.integers(0, 2, n).astype(np.uint8)
    with torch.cuda.stream(stream):
        yd = torch.tensor(y, device="cuda")
        pd = torch.zeros(n, dtype=torch.float32, device="cuda")
    loss = ms.maxsat_mp_gradient(model, ctx, yd)
    _, g = ms.maxsat_mp_get_params(model)
    ms.maxsat_mp_forward(model, ctx, pd)
    stream.synchronize()
    G = mpo.graph(n, off, lits, w)
    z, _ = mpo.forward(G, theta.astype(np.float64), L=layers, bf16=True)
    loss_o, g_o = mpo.backward(G, theta.astype(np.float64), y, L=layers, bf16=True)
    assert abs(loss - loss_o) <= 1e-5 * abs(loss_o)
    assert np.max(np.abs(pd.cpu().numpy() - 1 / (1 + np.exp(-z)))) <= 1e-5
    assert np.max(np.abs(g - g_o)) <= 1e-3 * np.max(np.abs(g_o))
    ms.maxsat_mp_destroy(model)
    ms.maxsat_destroy(ctx)


def test_training_reduces_the_loss(ms, stream):
    import torch
    n, off, lits, w = formula(seed=3)
    ctx = ctx_for(ms, stream, n, off, lits, w)
    _, best = ms.maxsat_solve(ctx, 256, 100, 1)
    model = ms.maxsat_mp_create(3, seed=1)
    with torch.cuda.stream(stream):
        yd = torch.tensor(best, device="cuda")
    losses = []
    for _ in range(60):
        losses.append(ms.maxsat_mp_gradient(model, ctx, yd))
        ms.maxsat_mp_adam(model, ctx, 3e-3)
    assert losses[-1] < 0.9 * losses[0]
    ms.maxsat_mp_destroy(model)
    ms.maxsat_destroy(ctx)


def test_reset_from_probabilities(ms, stream):
    n, off, lits, w = formula(seed=4, n=120, m=500)
    ctx = ctx_for(ms, stream, n, off, lits, w)
    B, seed = 64, 9
    ms.maxsat_reset(ctx, B, seed)
    plain = ms.maxsat_get_state(ctx)["x"]
    ms.maxsat_reset_probs(ctx, B, seed, np.full(n, 0.5, np.float32))
    assert np.array_equal(ms.maxsat_get_state(ctx)["x"], plain)
    p = np.where(np.arange(n) % 2 == 0, 0.0, 1.0).astype(np.float32)
    ms.maxsat_reset_probs(ctx, B, seed, p)
    x = ms.maxsat_get_state(ctx)["x"]
    assert np.all(x == (np.arange(n) % 2 == 1)[None, :])
    # the draw decision: x = [u < rint(65536 p)] with the initial draw u
    q = np.random.default_rng(1).random(n).astype(np.float32)
    ms.maxsat_reset_probs(ctx, B, seed, q)
    x = ms.maxsat_get_state(ctx)["x"]
    P = np.rint(q.astype(np.float64) * 65536)
    for b in (0, 7, 63):
        for i in (0, 5, n - 1):
            assert x[b, i] == (oracle.draw16(seed, 1, 0, i, 0, b) < P[i])
    ms.maxsat_destroy(ctx)


def test_learned_start_reaches_lower_costs(ms, stream):
    """Trained on solver-labelled formulas, the network's start distribution
    gives lower best costs than uniform starts on held-out formulas after the
    same number of rounds (same seed, same chains, deterministic training)."""
    from paper_2311_02101_gb300 import proposal as P
    import os
    table = oracle.RbmTable.load(os.path.join(os.path.dirname(__file__), "golden",
                                              "or_rbm_params.txt"))
    params = ms.maxsat_default_params(sets=[s for s in table.sets if s["len"] == 3],
                                      n_temps=2, n_buckets=4)
    params.fstar = None
    rng = np.random.default_rng(5)

    def gen(k, n_lo, n_hi):
        out = []
        for _ in range(k):
            n = int(rng.integers(n_lo, n_hi + 1))
            out.append(workloads.random_ksat(n, 6 * n, 3, int(rng.integers(1 << 30)), 1000))
        return out

    train = gen(512, 300, 800)
    labels = P.label_with_solver(train, params, restarts=256, steps=500, seed=3, stream=stream)
    model = ms.maxsat_mp_create(3, seed=0)
    losses = P.train(model, train, labels, params, epochs=12, batch=32, lr=2e-3, stream=stream)
    assert np.mean(losses[-16:]) < losses[0]
    plain, learned = [], []
    for f in gen(8, 800, 800):
        ctx = ms.maxsat_create(*f, params, stream)
        p = P.propose(model, ctx)
        for out, reset in ((plain, lambda: ms.maxsat_reset(ctx, 256, 11)),
                           (learned, lambda: ms.maxsat_reset_probs(ctx, 256, 11, p))):
            reset()
            ms.maxsat_step(ctx, 400)
            ms.maxsat_score(ctx)
            out.append(int(ms.maxsat_get_state(ctx)["best_cost"].min()))
        ms.maxsat_destroy(ctx)
    assert np.mean(learned) < np.mean(plain)
    ms.maxsat_mp_destroy(model)


@pytest.mark.parametrize("path", ["sparse", "dense"])
def test_flip_proposals_match_oracle(ms, stream, path):
    """Gibbs rounds, a flip-proposal merge with given probabilities, more
    rounds: the oracle's same sequence gives the same chains (merge on the
    device on the sparse path, on the host on the dense path)."""
    import os
    n, off, lits, w = formula(seed=7, n=200, m=900)
    table = oracle.RbmTable.load(os.path.join(os.path.dirname(__file__), "golden",
                                              "or_rbm_params.txt"))
    sets = [s for s in table.sets if s["len"] == 3]
    path = {"sparse": ms.MAXSAT_PATH_SPARSE, "dense": ms.MAXSAT_PATH_DENSE}[path]
    params = ms.maxsat_default_params(sets=sets, n_temps=2, n_buckets=4, path=path)
    params.fstar = None
    ctx = ms.maxsat_create(n, off, lits, w, params, stream)
    rng = np.random.default_rng(3)
    prob = rng.random(n).astype(np.float32)
    B, seed = 128, 4
    ms.maxsat_reset(ctx, B, seed)
    ms.maxsat_step(ctx, 6)
    ms.maxsat_propose_flips(ctx, prob, 0.15)
    ms.maxsat_step(ctx, 4)
    g = ms.maxsat_get_state(ctx)
    ms.maxsat_destroy(ctx)
    inst = oracle.Instance(n, off, lits, w)
    t = oracle.RbmTable()
    for s_ in sets:
        t.add(s_["len"], s_["bucket"], s_["temp"], s_["W"], s_["b"])
    st = oracle.init_chains(n, B, seed)
    kw = dict(n_temps=2, n_buckets=4, threads=os.cpu_count() or 4)
    oracle.gibbs(inst, t, st, 6, seed, **kw)
    oracle.up_merge(inst, st, oracle.flip_proposals(st.x, prob, 0.15))
    oracle.gibbs(inst, t, st, 4, seed, **kw)
    assert np.array_equal(g["x"], st.x)
    assert np.array_equal(g["best_cost"], st.best_cost)
    assert np.array_equal(g["nu"], st.nu32)
