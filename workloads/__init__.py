"""Seeded synthetic MaxSAT workloads.

The paper evaluates on MaxSAT Evaluation 2018-2021 instances (Sec. 5), which
are not available here; these seeded generators stand in for them with random
(weighted) k-SAT of the same kind: CNF clauses over distinct variables with
uniformly random polarities. This module holds no part of the solver's
arithmetic. Both the CUDA library's tests/benchmark and the CPU oracle draw
their inputs from it.

Every generator returns (n, off, lits, w): the number of variables, clause
offsets (int64, m + 1), DIMACS literals (int32, signed, 1-based) and integer
weights (int64, >= 1).
"""
from __future__ import annotations

import numpy as np

__all__ = ["random_ksat", "weighted_3sat", "mixed_length", "ragged_batch", "from_lengths",
           "WORKLOADS", "workload"]


def _distinct_rows(rng, n, lengths, kmax):
    """For each clause, `lengths[c]` distinct variables uniform in [0, n)."""
    m = len(lengths)
    V = rng.integers(0, n, size=(m, kmax))
    mask = np.arange(kmax)[None, :] < lengths[:, None]
    # redraw clauses whose used prefix has a repeated variable
    while True:
        s = np.sort(np.where(mask, V, -1 - np.arange(kmax)[None, :]), axis=1)
        dup = (s[:, 1:] == s[:, :-1]).any(axis=1)
        if not dup.any():
            return V
        idx = np.nonzero(dup)[0]
        V[idx] = rng.integers(0, n, size=(len(idx), kmax))


def from_lengths(n, lengths, rng, weights=None):
    lengths = np.asarray(lengths, np.int64)
    kmax = int(lengths.max()) if len(lengths) else 1
    if kmax > n:
        raise ValueError("clause longer than the number of variables")
    V = _distinct_rows(rng, n, lengths, max(kmax, 1))
    S = rng.integers(0, 2, size=V.shape) * 2 - 1  # polarity +-1 with p = 0.5
    mask = np.arange(V.shape[1])[None, :] < lengths[:, None]
    lits = ((V + 1) * S)[mask].astype(np.int32)
    off = np.zeros(len(lengths) + 1, np.int64)
    off[1:] = np.cumsum(lengths)
    w = np.ones(len(lengths), np.int64) if weights is None else np.asarray(weights, np.int64)
    return n, off, lits, w


def random_ksat(n, m, k=3, seed=0, wmax=None):
    """Uniform random k-SAT: each clause has k distinct variables chosen
    uniformly, each negated with probability 1/2; weights uniform in
    [1, wmax] when wmax is given, else all 1."""
    rng = np.random.default_rng(seed)
    lengths = np.full(m, k, np.int64)
    n_, off, lits, _ = from_lengths(n, lengths, rng)
    w = np.ones(m, np.int64) if wmax is None else rng.integers(1, wmax + 1, size=m).astype(np.int64)
    return n_, off, lits, w


def weighted_3sat(n=1000, m=6000, wmax=1000, seed=0):
    return random_ksat(n, m, 3, seed, wmax)


def mixed_length(n=20000, m=100000, p=0.4, cap=12, hard_frac=0.1, soft_max=100, seed=0):
    """Clause length 2 + Geometric(p) (failures before the first success, so
    >= 0), capped at `cap`; a uniformly chosen round(hard_frac * m) clauses are
    hard with weight 1 + (sum of the soft weights); soft weights uniform in
    [1, soft_max]."""
    rng = np.random.default_rng(seed)
    lengths = np.minimum(2 + (rng.geometric(p, size=m) - 1), cap).astype(np.int64)
    n_, off, lits, _ = from_lengths(n, lengths, rng)
    w = rng.integers(1, soft_max + 1, size=m).astype(np.int64)
    hard = rng.choice(m, size=int(round(hard_frac * m)), replace=False)
    soft = np.ones(m, bool)
    soft[hard] = False
    w[hard] = 1 + int(w[soft].sum())
    return n_, off, lits, w


def ragged_batch(count=512, n_lo=100, n_hi=5000, ratio_lo=4.0, ratio_hi=8.0, wmax=1000, seed=0):
    """`count` weighted 3-SAT instances with n log-uniform in [n_lo, n_hi] and
    m / n uniform in [ratio_lo, ratio_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        m = int(round(rng.uniform(ratio_lo, ratio_hi) * n))
        out.append(random_ksat(n, m, 3, int(rng.integers(0, 2 ** 31)), wmax))
    return out


# The workloads named by the benchmark configurations.
WORKLOADS = {
    # random unweighted 3-SAT at clause/variable ratio 4.3, 256 restarts
    "3sat-n50-m215": dict(gen=lambda seed=0: random_ksat(50, 215, 3, seed), B=256, steps=200),
    # its brute-force twin: n = 18, m = round(4.3 * 18)
    "3sat-n18-m77": dict(gen=lambda seed=0: random_ksat(18, 77, 3, seed), B=256, steps=200),
    # weighted Max-3-SAT, weights uniform in [1, 1000], 4096 restarts
    "w3sat-n1000-m6000": dict(gen=lambda seed=0: weighted_3sat(1000, 6000, 1000, seed), B=4096),
    # mixed clause lengths 2 + Geom(0.4) capped at 12, 10 % hard, 1024 restarts
    "mixed-n20000-m100000": dict(gen=lambda seed=0: mixed_length(seed=seed), B=1024),
    # batch of 512 weighted 3-SAT instances, n log-uniform in [100, 5000], m / n uniform in
    # [4, 8], 256 restarts each (gen returns a list of instances)
    "ragged-512": dict(gen=lambda seed=0: ragged_batch(seed=seed), B=256, batch=True),
}


def workload(name, seed=0):
    return WORKLOADS[name]["gen"](seed)
