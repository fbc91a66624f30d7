"""The GPU form of the unit-propagation heuristic (Sec. 4.4) differs from the
host form in two ways that must not change any result:
  * a clause's state is read from the variable values (satisfied: a true
    literal; unit: no true literal and exactly one unassigned literal
    occurrence) instead of incrementally kept counters;
  * a variable enters the queue at most once (the first entry of a variable
    is the one that assigns it; a later entry would find it assigned).
This file restates that procedure in plain Python and checks it against the
oracle's unit propagation (counters, every entry queued) on formulas with
duplicate literals, tautologies, empty clauses, ties in nu and -0.0.
"""
import numpy as np

import oracle
import workloads


def up_queue_once(n, off, lits, x, nu):
    order = sorted(range(n), key=lambda v: (-float(nu[v]), v))
    occ = [[] for _ in range(n)]
    for c in range(len(off) - 1):
        for j in range(off[c], off[c + 1]):
            occ[abs(int(lits[j])) - 1].append(c)
    val = [2] * n  # 0 / 1 assigned, 2 unassigned, 3 unassigned and queued
    half = n // 2
    for r in range(half):
        val[order[r]] = int(x[order[r]])

    def unit(c):
        nun, first = 0, None
        for j in range(off[c], off[c + 1]):
            lit = int(lits[j])
            s = val[abs(lit) - 1]
            if s >= 2:
                if nun == 0:
                    first = lit
                nun += 1
            elif (s == 1) == (lit > 0):
                return None
        return first if nun == 1 else None

    queue = []

    def push(lit):
        v = abs(lit) - 1
        if val[v] == 2:
            val[v] = 3
            queue.append(lit)

    def set_check(v, value):
        val[v] = value
        for c in occ[v]:
            lit = unit(c)
            if lit is not None:
                push(lit)

    head = 0

    def drain():
        nonlocal head
        while head < len(queue):
            lit = queue[head]
            head += 1
            if val[abs(lit) - 1] >= 2:
                set_check(abs(lit) - 1, 1 if lit > 0 else 0)

    for c in range(len(off) - 1):
        lit = unit(c)
        if lit is not None:
            push(lit)
    drain()
    for r in range(half, n):
        v = order[r]
        if val[v] >= 2:
            set_check(v, int(x[v]))
            drain()
    assert len(queue) <= n
    return np.array(val, np.uint8)


def edge_formula(seed):
    rng = np.random.default_rng(seed)
    n = 30
    lengths = rng.integers(1, 5, size=110)
    _, off, lits, _ = workloads.from_lengths(n - 1, lengths, rng)
    cl = [list(lits[off[c]:off[c + 1]]) for c in range(len(lengths))]
    cl += [[3, 3, -5], [7, -7], [], [-2, -2, -2, 9], [12], [12, 12]]
    rng.shuffle(cl)
    return oracle.Instance.from_clauses(n, cl, list(rng.integers(1, 9, size=len(cl))))


def test_queue_once_matches_the_oracle():
    for seed in range(6):
        inst = edge_formula(seed)
        rng = np.random.default_rng(100 + seed)
        B = 24
        x = rng.integers(0, 2, size=(B, inst.n)).astype(np.uint8)
        # coarse values (many ties), some -0.0
        nu = (rng.integers(0, 6, size=(B, inst.n)) * 0.05).astype(np.float32)
        nu[rng.random((B, inst.n)) < 0.1] = np.float32(-0.0)
        ref = oracle.unit_prop(inst, x, nu)
        for b in range(B):
            got = up_queue_once(inst.n, inst.off, inst.lits, x[b], nu[b])
            assert np.array_equal(got, ref[b]), (seed, b)


def test_queue_once_on_random_3sat():
    inst_t = workloads.random_ksat(60, 258, 3, seed=2)
    inst = oracle.Instance(inst_t[0], inst_t[1], inst_t[2], inst_t[3])
    rng = np.random.default_rng(7)
    x = rng.integers(0, 2, size=(16, inst.n)).astype(np.uint8)
    nu = rng.random((16, inst.n)).astype(np.float32) * 0.25
    ref = oracle.unit_prop(inst, x, nu)
    for b in range(16):
        assert np.array_equal(up_queue_once(inst.n, inst.off, inst.lits, x[b], nu[b]), ref[b])
