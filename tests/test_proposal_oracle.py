"""Pins of the learned-proposal oracle (numpy, FP64): its analytic gradient
against central finite differences, its aggregation against a per-clause loop,
the BF16 rounding against exact cases, and the flip-proposal rule against a
hand-written case."""
import numpy as np

import workloads
from oracle import proposal as mp


def small_graph(seed=0):
    n, off, lits, w = workloads.weighted_3sat(40, 150, 100, seed=seed)
    lits = np.asarray(lits).copy()
    lits[1] = lits[0]  # clause 0 repeats a literal
    # and variable n + 1 is in no clause
    return mp.graph(n + 1, off, lits, w)


def test_gradient_matches_finite_differences():
    G = small_graph(1)
    rng = np.random.default_rng(0)
    theta = mp.init_params(3) + rng.normal(0, 0.05, mp.n_params())
    y = rng.integers(0, 2, G["n"])
    L0, g = mp.backward(G, theta, y, bf16=False)
    eps = 1e-6
    idx = rng.choice(mp.n_params(), 40, replace=False)
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (mp.loss(mp.forward(G, tp, bf16=False)[0], y) -
              mp.loss(mp.forward(G, tm, bf16=False)[0], y)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(fd), (k, fd, g[k])


def test_clause_aggregation_is_the_signed_mean():
    n, off, lits, w = workloads.weighted_3sat(30, 80, 10, seed=3)
    G = mp.graph(n, off, lits, w)
    rng = np.random.default_rng(1)
    h = rng.normal(size=(n, 5))
    got = G["inv_len"][:, None] * (G["S"] @ h)
    for c in range(len(off) - 1):
        ls = lits[off[c]:off[c + 1]]
        want = np.mean([np.sign(l) * h[abs(l) - 1] for l in ls], axis=0)
        assert np.allclose(got[c], want)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0],
                    np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to the even mantissa (1.0)
    want = [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0]
    assert np.array_equal(mp.bf16_round(vals), np.array(want))


def test_flip_proposals_hand_written():
    """Flip proposals (the network's confident values written into every
    chain): with tau = 1/4, p >= 3/4 sets the variable to 1, p <= 1/4 to 0,
    anything between keeps the chain's value; both bounds are inclusive."""
    import oracle
    x = np.array([[0, 1, 0, 1, 0, 1],
                  [1, 0, 1, 0, 1, 0]], np.uint8)
    p = np.array([0.75, 0.25, 0.7499999, 0.2500001, 0.99, 0.0], np.float32)
    want = np.array([[1, 0, 0, 1, 1, 0],
                     [1, 0, 1, 0, 1, 0]], np.uint8)
    assert np.array_equal(oracle.flip_proposals(x, p, 0.25), want)
    # tau = 0 sets only certain variables
    assert np.array_equal(oracle.flip_proposals(x, np.array([1, 0, .5, .5, .5, .5], np.float32), 0.0),
                          np.array([[1, 0, 0, 1, 0, 1], [1, 0, 1, 0, 1, 0]], np.uint8))
