"""Pins for the CPU oracle: each test ties it to something other than itself
(values printed in the paper, published known answers, definitions evaluated
another way, exact enumeration, brute force, invariants, statistics)."""
import itertools
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def inst_of(gen):
    n, off, lits, w = gen
    return oracle.Instance(n, off, lits, w)


# --------------------------------------------------------------------------
# Randomness: Philox4x32-10 known-answer values (Salmon et al., SC'11; the
# Random123 distribution's published known-answer vectors).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key,expect", [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
])
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_draw16_lanes_and_uniformity():
    seed = 0x123456789ABCDEF0
    out = oracle.philox4x32_10([7, (16 >> 3) | (2 << 24), 5, 2], [seed & 0xFFFFFFFF, seed >> 32])
    lanes = [(int(out[l >> 1]) >> (16 * (l & 1))) & 0xFFFF for l in range(8)]
    assert [oracle.draw16(seed, 2, 5, 7, 2, 16 + l) for l in range(8)] == lanes
    u = np.array([oracle.draw16(1, 3, t, i, 0, b) for t in range(4) for i in range(64)
                  for b in range(32)])
    assert abs(u.mean() / 65536 - 0.5) < 0.02
    assert u.min() >= 0 and u.max() < 65536


# --------------------------------------------------------------------------
# Cost: worked examples of the paper's text (Sec. 4.3, Sec. 4.4), hand-scored
# --------------------------------------------------------------------------
def _paper_examples():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "paper_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#") or line.startswith("up "):
                continue
            if line.startswith("formula"):
                head, body = line.split("|")
                n = int(head.split()[1])
                clauses = [[int(t) for t in c.split()] for c in body.split(";")]
                cur = (n, clauses, [])
                cases.append(cur)
            else:
                _, bits, _, cost = line.split()
                cur[2].append(([int(ch) for ch in bits], int(cost)))
    return cases


def test_eval_paper_examples():
    cases = _paper_examples()
    assert len(cases) == 2
    for n, clauses, rows in cases:
        inst = oracle.Instance.from_clauses(n, clauses)
        X = np.array([r[0] for r in rows], np.uint8)
        assert list(oracle.evaluate(inst, X)) == [r[1] for r in rows]


def test_eval_matches_matrix_form():
    """count_c = (C s + len_c) / 2 with s = 2x - 1 and C the signed
    clause-literal matrix; satisfied iff count > 0; weighted cost."""
    rng = np.random.default_rng(3)
    n, off, lits, w = workloads.mixed_length(n=40, m=300, cap=12, seed=5)
    inst = oracle.Instance(n, off, lits, w)
    # duplicates, tautologies and an empty clause on top of the random ones
    extra = [[1, 1, 2], [3, -3], [], [-4, -4], [5]]
    cl = inst.clauses() + extra
    ws = list(w) + [7, 9, 11, 13, 17]
    inst = oracle.Instance.from_clauses(n, cl, ws)
    C = np.zeros((inst.m, n))
    for c, lc in enumerate(cl):
        for l in lc:
            C[c, abs(l) - 1] += np.sign(l)
    ln = np.diff(inst.off)
    X = rng.integers(0, 2, size=(200, n)).astype(np.uint8)
    S = 2.0 * X - 1.0
    count = (S @ C.T + ln[None, :]) / 2
    assert np.all(count == np.round(count)) and count.min() >= 0
    # brute count of true literal occurrences agrees
    for b in range(5):
        for c, lc in enumerate(cl):
            assert count[b, c] == sum((l > 0) == bool(X[b, abs(l) - 1]) for l in lc)
    cost = ((count == 0) * inst.w[None, :]).sum(axis=1)
    assert np.array_equal(oracle.evaluate(inst, X), cost)


def test_padding_by_repetition_keeps_the_satisfying_set():
    """Sec. 4.3: a clause padded to length K by repeating one of its
    variables with the same polarity has the same satisfying assignments, so
    every assignment keeps its cost (the build groups clauses by length
    instead of padding them, R14; the cost must not depend on it)."""
    rng = np.random.default_rng(11)
    n = 12
    lengths = rng.integers(1, 5, size=60)
    _, off, lits, w = workloads.from_lengths(n, lengths, rng)
    plain = oracle.Instance(n, off, lits, w)
    K = 4
    padded = [c + [c[int(rng.integers(0, len(c)))]] * (K - len(c)) for c in plain.clauses()]
    inst = oracle.Instance.from_clauses(n, padded, list(w))
    assert set(np.diff(inst.off)) == {K}
    X = np.array(list(itertools.product([0, 1], repeat=n)), np.uint8)
    assert np.array_equal(oracle.evaluate(inst, X), oracle.evaluate(plain, X))


def test_printed_count_form_misses_negated_literals():
    """The count printed in the appendix listing tests only positive
    polarities, so a clause made only of negated literals is never counted as
    satisfied. The text (Sec. 4.3) compares signs with the Boolean values; the
    oracle follows the text."""
    inst = oracle.Instance.from_clauses(2, [[-1, -2]])
    x = np.array([[0, 0]], np.uint8)
    assert oracle.evaluate(inst, x)[0] == 0  # NOT x1 is true
    gathered = x[0][[0, 1]]  # values of the clause's variables
    polarity = np.array([-1, -1])
    printed_any = bool(((polarity > 0) * gathered).any())
    assert printed_any is False  # the printed form would call it unsatisfied


def test_brute_force_small_independent():
    """Brute-force optimum via the oracle equals a pure-Python enumeration."""
    inst = inst_of(workloads.random_ksat(10, 43, 3, seed=2, wmax=9))
    cl = inst.clauses()
    best = min(sum(int(inst.w[c]) for c, lc in enumerate(cl)
                   if not any((l > 0) == bool(v[abs(l) - 1]) for l in lc))
               for v in itertools.product([0, 1], repeat=inst.n))
    assert oracle.brute_force_optimum(inst) == best


# --------------------------------------------------------------------------
# RBM pins
# --------------------------------------------------------------------------
def _tiny_table(lengths, fstars, iters=4000):
    return oracle.make_table(lengths, fstars, n_buckets=1, iters=iters)


def test_fit_reaches_or_targets():
    """Sec. 4.1: F(0) ~ 0 and F(v) ~ F_s = -F* for v != 0."""
    for K, fs in [(2, 0.528), (3, 0.528), (3, 0.068)]:
        W, b = oracle.fit_or_rbm(K, fs)
        V = np.array(list(itertools.product([0.0, 1.0], repeat=K)))
        F = oracle.or_free_energy(W, b, V)
        assert abs(F[0]) < 0.05
        assert np.max(np.abs(F[1:] + fs)) < 0.05
        Wq, bq = oracle.quantise(K, fs, W, b)
        assert np.all(Wq * 16 == np.round(Wq * 16))
        assert np.all(bq * 2 ** 24 == np.round(bq * 2 ** 24))
        assert oracle.fit_loss(K, fs, Wq, bq) < 4 * oracle.fit_loss(K, fs, W, b) + 1e-3


def test_hidden_unit_counts_follow_the_printed_rule():
    """Appendix "Pretraining": 3 hidden units for clause size 3 and K + 1
    for K in 4..7 (written out here from that sentence); the fitted W has
    that many columns."""
    printed = {3: 3, 4: 5, 5: 6, 6: 7, 7: 8}
    for K, L in printed.items():
        assert oracle.hidden_units_for(K) == L
    W, b = oracle.fit_or_rbm(4, 0.528, iters=10)
    assert W.shape == (4, 5) and b.shape == (5,)


def test_tied_weights_cannot_fit_or():
    """Reading check: with one weight shared by all inputs of a hidden unit,
    -F(s) = sum_h softplus(b_h + w_h s) is convex in the count s, while the OR
    target (0, F*, F*, ...) is not, so the general per-position W of the paper
    is required. A tied fit stays far from the target; the general fit does
    not."""
    K, fs = 3, 0.528
    s = np.arange(K + 1, dtype=float)
    # best tied fit by brute-force search over a grid of 2 hidden units
    best = np.inf
    grid = np.linspace(-6, 6, 49)
    for w1, b1, w2, b2 in itertools.product(grid[::4], grid[::4], grid[::4], grid[::4]):
        F = -(np.logaddexp(0, b1 + w1 * s) + np.logaddexp(0, b2 + w2 * s))
        F = F - F[0]  # free energies matter up to a constant
        err = np.array([3, 3, 1]) @ (F[1:] + fs) ** 2
        best = min(best, err)
    assert best > 0.05
    W, b = oracle.fit_or_rbm(K, fs)
    assert oracle.fit_loss(K, fs, W, b) < 0.01


def test_free_energy_matches_hidden_enumeration():
    """Eq. 1 (softplus form) equals -log sum_h exp(-E(v, h)) with
    E = -v^T W_f h - b_f^T h, enumerated over every hidden configuration of
    the formula RBM (product of clause RBMs, Sec. 4.1)."""
    table = _tiny_table([2, 3], [0.528])
    inst = oracle.Instance.from_clauses(4, [[1, -2, 3], [-1, 4], [-3, -4, 2]])
    Wf, bf = oracle.formula_rbm(inst, table, temp=0)
    H = np.array(list(itertools.product([0.0, 1.0], repeat=Wf.shape[1])))
    X = oracle.all_assignments(4)
    Fo = oracle.free_energy(inst, table, X, temp=0)
    for r, v in enumerate(X.astype(float)):
        negE = H @ (Wf.T @ v) + H @ bf
        F_enum = -np.log(np.exp(negE).sum())
        assert abs(F_enum - Fo[r]) < 1e-9


def test_negation_transform_eq4():
    """Eq. 4: the transformed clause RBM on v equals the canonical one on the
    input with negated literals flipped."""
    table = _tiny_table([3], [0.528])
    s = table.get(3, 0, 0)
    W, b = s["W"], s["b"]
    clause = [2, -1, -3]
    inst = oracle.Instance.from_clauses(3, [clause])
    X = oracle.all_assignments(3)
    F_t = oracle.free_energy(inst, table, X, temp=0)
    for r, x in enumerate(X):
        u = np.array([x[abs(l) - 1] if l > 0 else 1 - x[abs(l) - 1] for l in clause], float)
        F_c = -np.logaddexp(0, u @ W + b).sum()
        assert abs(F_c - F_t[r]) < 1e-12


def test_formula_free_energy_orders_by_satisfied_clauses():
    """Sec. 4.1: each satisfied clause contributes ~F_s < 0, an unsatisfied
    one ~0, so F tracks the number of satisfied clauses."""
    table = _tiny_table([3], [0.528], iters=20000)
    inst = inst_of(workloads.random_ksat(8, 30, 3, seed=1))
    X = oracle.all_assignments(8)
    F = oracle.free_energy(inst, table, X, temp=0)
    sat = inst.m - oracle.evaluate(inst, X)
    slope = np.polyfit(sat, F, 1)[0]
    assert abs(slope + 0.528) < 0.05


def _exact_one_step(inst, table, x0):
    """Exact distribution of x' after one Gibbs round from x0 with the 16-bit
    probabilities P/65536 of the sampling contract: sum over hidden states of
    p(h|x0) p(x'|h), from the dense formula RBM (Eqs. 2, 3)."""
    Wf, bf = oracle.formula_rbm(inst, table, temp=0)
    q = lambda a: np.rint(65536.0 / (1.0 + np.exp(-a))) / 65536.0
    ph = q(bf + Wf.T @ x0.astype(float))
    H = np.array(list(itertools.product([0.0, 1.0], repeat=len(bf))))
    X = oracle.all_assignments(inst.n).astype(float)
    dist = np.zeros(len(X))
    for h in H:
        p_h = np.prod(np.where(h > 0, ph, 1 - ph))
        pv = q(Wf @ h)
        dist += p_h * np.prod(np.where(X > 0, pv, 1 - pv), axis=1)
    return dist


def test_one_step_transition_matches_enumeration():
    """One round of the oracle from a fixed state, over many chains, matches
    the exact transition kernel (catches a dropped term, a wrong sign or a
    wrong index in the hidden or visible conditionals)."""
    table = _tiny_table([2, 3], [0.528])
    inst = oracle.Instance.from_clauses(3, [[1, -2, 3], [-1, -3], [2, 3, -1]])
    x0 = np.array([1, 0, 1], np.uint8)
    B = 1 << 16
    st = oracle.init_chains(3, B, seed=11)
    st.x[:] = x0
    oracle.gibbs(inst, table, st, 1, seed=11, n_temps=1)
    idx = (st.x.astype(np.int64) << np.arange(3)).sum(axis=1)
    emp = np.bincount(idx, minlength=8) / B
    exact = _exact_one_step(inst, table, x0)
    chi2 = (B * (emp - exact) ** 2 / np.maximum(exact, 1e-12)).sum()
    assert chi2 < 30.0, (emp, exact)  # 7 dof: p ~ 1e-4


def test_stationary_distribution():
    """Block Gibbs leaves p(v) ~ exp(-F(v)) invariant (Sec. 3.1): the empirical
    state frequencies over many chains and steps match it."""
    table = _tiny_table([2, 3], [0.528])
    inst = oracle.Instance.from_clauses(4, [[1, -2, 3], [-1, 4], [-3, -4, 2], [2, 4]])
    X = oracle.all_assignments(4)
    F = oracle.free_energy(inst, table, X, temp=0)
    p = np.exp(-(F - F.min()))
    p /= p.sum()
    B = 4096
    st = oracle.init_chains(4, B, seed=5)
    oracle.gibbs(inst, table, st, 10, seed=5, n_temps=1)
    counts = np.zeros(16)
    for _ in range(40):
        oracle.gibbs(inst, table, st, 1, seed=5, n_temps=1)
        counts += np.bincount((st.x.astype(np.int64) << np.arange(4)).sum(axis=1), minlength=16)
    emp = counts / counts.sum()
    assert 0.5 * np.abs(emp - p).sum() < 0.01


def test_swap_threshold_is_the_metropolis_rule():
    """A swap with log-ratio D (units 2^-20) is accepted for exactly the
    16-bit draws u < 65536 exp(D 2^-20): ceil(65536 exp(D 2^-20)) of the
    65536 values when exp(D 2^-20) < 1, all of them when D >= 0."""
    T = oracle.swap_thresholds()
    for ratio in (0.3, 0.01, 0.5, 0.9999):
        D = int(np.floor(np.ldexp(np.log(ratio), 20)))
        want = int(np.ceil(65536 * np.exp(np.ldexp(D, -20))))
        assert int(np.sum(D >= T)) == want
    assert np.all(0 >= T) and np.all(5 >= T)
    assert int(np.sum(-(40 << 20) >= T)) == 1  # only u = 0


def test_parallel_tempering_keeps_each_temperature_stationary():
    """Block Gibbs interleaved with swap rounds leaves every temperature's
    target exp(-F_e) invariant (swaps are Metropolis moves on the product of
    the targets): the empirical state frequencies of each temperature block
    match it, and swaps do happen."""
    table = _tiny_table([2, 3], [0.2, 1.0])
    inst = oracle.Instance.from_clauses(4, [[1, -2, 3], [-1, 4], [-3, -4, 2], [2, 4]])
    X = oracle.all_assignments(4)
    targets = []
    for e in range(2):
        F = oracle.free_energy(inst, table, X, temp=e)
        p = np.exp(-(F - F.min()))
        targets.append(p / p.sum())
    B, S = 8192, 4096
    st = oracle.init_chains(4, B, seed=5)
    oracle.gibbs(inst, table, st, 10, seed=5, n_temps=2)
    counts = np.zeros((2, 16))
    swaps = 0
    for r in range(40):
        swaps += oracle.pt_swap(inst, table, st, seed=5, parity=0, n_temps=2)
        oracle.gibbs(inst, table, st, 1, seed=5, n_temps=2)
        code = (st.x.astype(np.int64) << np.arange(4)).sum(axis=1)
        for e in range(2):
            counts[e] += np.bincount(code[e * S:(e + 1) * S], minlength=16)
    assert swaps > 1000
    for e in range(2):
        emp = counts[e] / counts[e].sum()
        assert 0.5 * np.abs(emp - targets[e]).sum() < 0.01, e


# --------------------------------------------------------------------------
# Search: determinism, resume, best-keep, quality
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg1_table():
    return _tiny_table([3], [0.068, 0.528], iters=20000)


def test_init_contract():
    st = oracle.init_chains(50, 64, seed=9)
    assert abs(st.x.mean() - 0.5) < 0.03
    assert np.all(st.nu == 0.25)
    assert np.all(st.best_cost == np.iinfo(np.int64).max)
    assert st.x[3, 17] == (oracle.draw16(9, 1, 0, 17, 0, 3) < 32768)


def test_instance_index_enters_only_the_phase_word(cfg1_table):
    """A formula solved as instance 5 of a batch draws from phase words
    phase | 5 << 8: its initial state is those draws, and one round of Gibbs
    from a common state differs from instance 0 only through its draws (the
    scores of the common state agree)."""
    st = oracle.init_chains(50, 16, seed=9, instance=5)
    assert st.x[3, 17] == (oracle.draw16(9, 1 | (5 << 8), 0, 17, 0, 3) < 32768)
    assert not np.array_equal(st.x, oracle.init_chains(50, 16, seed=9).x)
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    a = oracle.init_chains(50, 16, seed=9)
    b = a.copy()
    b.instance = 5
    oracle.gibbs(inst, cfg1_table, a, 1, seed=9, n_temps=2)
    oracle.gibbs(inst, cfg1_table, b, 1, seed=9, n_temps=2)
    assert np.array_equal(a.cost, b.cost) and np.array_equal(a.best_cost, b.best_cost)
    assert not np.array_equal(a.x, b.x)


def test_fp32_nu_sequence_tracks_fp64_nu(cfg1_table):
    """The oracle's FP32 nu (the solver's operation sequence, used where nu
    decides a ranking) stays within the FP32 rounding bound of the FP64 EMA
    of Sec. 4.4: each round adds at most ~4 roundings of a value <= 0.25 and
    shrinks older errors by (1 - alpha)."""
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    T, alpha = 60, 0.05
    st = oracle.init_chains(50, 64, seed=3)
    oracle.gibbs(inst, cfg1_table, st, T, seed=3, n_temps=2, alpha=alpha)
    bound = 4 * 2.0 ** -24 * 0.25 * min(T, 1 / alpha) + 0.25 * abs(np.float32(alpha) - alpha) * T
    assert np.max(np.abs(st.nu32.astype(np.float64) - st.nu)) <= bound
    assert st.nu32.dtype == np.float32 and np.all(st.nu32 <= 0.25) and np.all(st.nu32 >= 0)


def _paper_up_cases():
    out = []
    with open(os.path.join(GOLDEN, "paper_examples.txt")) as f:
        for line in f:
            if line.startswith("up "):
                left, right = line[3:].split("->")
                xs, nus = left.split(" nu ")
                out.append((np.array([int(c) for c in xs.strip()], np.uint8),
                            np.array([float(v) for v in nus.split()], np.float32),
                            np.array([int(c) for c in right.strip()], np.uint8)))
    return out


def test_unit_prop_paper_example():
    """Sec. 4.4: with a = b = False held fixed, (a OR b OR c) AND (NOT c OR
    NOT d) implies c = True, then d = False."""
    inst = oracle.Instance.from_clauses(4, [[1, 2, 3], [-3, -4]])
    cases = _paper_up_cases()
    assert len(cases) == 3
    for x, nu, want in cases:
        assert np.array_equal(oracle.unit_prop(inst, x, nu)[0], want)


def test_unit_prop_keeps_a_satisfying_assignment():
    """If x satisfies every clause, every clause that becomes unit is satisfied
    by x's value of its open literal, so propagation reproduces x."""
    rng = np.random.default_rng(8)
    n, m = 60, 240
    sol = rng.integers(0, 2, n).astype(np.uint8)
    cl = []
    while len(cl) < m:
        v = rng.choice(n, 3, replace=False)
        s = rng.choice([-1, 1], 3)
        lits = [int(s[k] * (v[k] + 1)) for k in range(3)]
        if any((l > 0) == bool(sol[abs(l) - 1]) for l in lits):
            cl.append(lits)
    inst = oracle.Instance.from_clauses(n, cl)
    assert oracle.evaluate(inst, sol[None])[0] == 0
    nu = rng.random((16, n)).astype(np.float32)
    out = oracle.unit_prop(inst, np.repeat(sol[None], 16, 0), nu)
    assert np.all(out == sol[None])


def test_unit_prop_follows_an_implication_chain():
    """(v1) AND (NOT v1 OR v2) AND ... AND (NOT v9 OR v10), with v1..v10
    ranked below the fixed half: the unit clause forces v1 and the chain
    forces every later variable True, whatever x says."""
    n = 20
    cl = [[1]] + [[-k, k + 1] for k in range(1, 10)]
    inst = oracle.Instance.from_clauses(n, cl)
    nu = np.concatenate([np.zeros(10), np.ones(10)]).astype(np.float32)
    x = np.zeros(n, np.uint8)
    x[10:] = 1
    out = oracle.unit_prop(inst, x, nu)[0]
    assert np.all(out[:10] == 1) and np.all(out[10:] == 1)
    # a conflicting fixed value stays fixed: v2 fixed False breaks the chain there
    nu2 = nu.copy()
    nu2[1] = 2.0
    x2 = x.copy()
    x2[1] = 0
    out2 = oracle.unit_prop(inst, x2, nu2)[0]
    assert out2[0] == 1 and out2[1] == 0


def test_up_merge_keeps_the_lowest_costs():
    """The B-of-2B merge keeps the B lowest-cost candidates, ordered as a
    stable ascending sort of satisfied weight (ties: later candidates later)."""
    inst = oracle.Instance.from_clauses(3, [[1], [2], [3]])
    st = oracle.init_chains(3, 3, seed=1)
    st.x = np.array([[1, 1, 0], [0, 0, 0], [1, 1, 1]], np.uint8)  # costs 1, 3, 0
    up = np.array([[1, 0, 0], [0, 1, 1], [1, 1, 1]], np.uint8)     # costs 2, 1, 0
    st.nu32 = np.arange(9, dtype=np.float32).reshape(3, 3)
    st.nu = st.nu32.astype(np.float64)
    oracle.up_merge(inst, st, up)
    # stacked costs [1, 3, 0, 2, 1, 0]; ascending satisfied weight, stable:
    # 3(1) 2(3) 1(0) 1(4) 0(2) 0(5) -> last three: candidates 4, 2, 5
    assert np.array_equal(st.x, np.array([[0, 1, 1], [1, 1, 1], [1, 1, 1]], np.uint8))
    assert np.array_equal(st.nu32, np.array([[3, 4, 5], [6, 7, 8], [6, 7, 8]], np.float32))


def test_determinism_and_resume(cfg1_table):
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    a = oracle.init_chains(50, 32, seed=4)
    b = a.copy()
    oracle.gibbs(inst, cfg1_table, a, 30, seed=4, n_temps=2)
    oracle.gibbs(inst, cfg1_table, b, 12, seed=4, n_temps=2)
    oracle.gibbs(inst, cfg1_table, b, 18, seed=4, n_temps=2)
    for f in ["x", "nu", "best_cost", "best_x", "cost", "free_energy"]:
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_best_keep_invariants(cfg1_table):
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    st = oracle.init_chains(50, 16, seed=1)
    seen = np.full(16, np.iinfo(np.int64).max)
    for _ in range(20):
        oracle.gibbs(inst, cfg1_table, st, 1, seed=1, n_temps=2)
        seen = np.minimum(seen, st.cost)
    oracle.score_and_keep(inst, st)
    seen = np.minimum(seen, st.cost)
    assert np.array_equal(st.best_cost, seen)
    assert np.array_equal(oracle.evaluate(inst, st.best_x), st.best_cost)


def test_nu_update_range(cfg1_table):
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    st = oracle.init_chains(50, 8, seed=2)
    oracle.gibbs(inst, cfg1_table, st, 50, seed=2, n_temps=2, alpha=0.05)
    assert st.nu.min() >= 0 and st.nu.max() <= 0.25


def test_brute_force_twin_reaches_optimum(cfg1_table):
    """n = 18, m = 77 (ratio 4.3): the best cost found is never below the
    exact optimum, and 256 chains x 200 steps reach it."""
    inst = inst_of(workloads.random_ksat(18, 77, 3, seed=0))
    opt = oracle.brute_force_optimum(inst)
    best, bx, st = oracle.solve(inst, cfg1_table, 256, 200, seed=0, n_temps=2, threads=4)
    assert best >= opt
    assert oracle.evaluate(inst, bx[None])[0] == best
    assert best == opt


def test_gibbs_beats_uniform_random(cfg1_table):
    """Ablation idea of Table 2 (-Gibbs): at an equal number of evaluated
    assignments, Gibbs sampling finds lower costs than uniform random ones."""
    inst = inst_of(workloads.random_ksat(50, 215, 3, seed=0))
    best, _, _ = oracle.solve(inst, cfg1_table, 64, 100, seed=3, n_temps=2, threads=4)
    rng = np.random.default_rng(0)
    X = rng.integers(0, 2, size=(64 * 101, 50)).astype(np.uint8)
    assert best < oracle.evaluate(inst, X).min()


def test_draw_decision_is_strict_below_threshold():
    """The sampling contract's decision x = [u < P]: with no clauses every
    visible logit is 0, so P = 65536 * sigma(0) = 32768 and x' must equal
    [u < 32768] for every chain and variable (2^18 draws hit u == 32768)."""
    inst = oracle.Instance.from_clauses(4, [])
    B = 1 << 16
    st = oracle.init_chains(4, B, seed=21)
    oracle.gibbs(inst, oracle.RbmTable(), st, 1, seed=21, n_temps=1)
    draws = np.array([[oracle.draw16(21, 3, 0, i, 0, b) for i in range(4)] for b in range(B)])
    assert (draws == 32768).any()
    assert np.array_equal(st.x, (draws < 32768).astype(np.uint8))
    assert np.allclose(st.nu, 0.99 * 0.25 + 0.01 * 0.25)


# --------------------------------------------------------------------------
# Weight buckets (reading of the unweighted paper, Sec. 5 "Datasets": clause c
# uses the set of bucket j, the largest j < J with w_min 2^j <= w_c). The
# expected buckets below are written out by hand for weights on both sides of
# every boundary; the oracle's choice is read through the free energy of a
# probe formula whose bucket sets differ only in their bias.
# --------------------------------------------------------------------------
def _bucket_probe_table(J):
    """Length-1 sets, one hidden unit, W = 0 and bias j + 1 for bucket j: the
    clause free energy is -softplus(j + 1) whatever the assignment."""
    t = oracle.RbmTable()
    for j in range(J):
        t.add(1, j, 0, np.zeros((1, 1)), np.array([float(j + 1)]))
    return t


def _bucket_chosen(w_min, w, J):
    inst = oracle.Instance.from_clauses(2, [[1], [-2]], [w_min, w])
    F = oracle.free_energy(inst, _bucket_probe_table(J), np.zeros((1, 2), np.uint8), temp=0,
                           n_buckets=J)[0]
    # clause 0 (the lightest) is in bucket 0: -softplus(1); the rest is clause 1
    rest = F + np.log1p(np.exp(1.0))
    cand = [-np.log1p(np.exp(float(j + 1))) for j in range(J)]
    j = int(np.argmin([abs(rest - c) for c in cand]))
    assert abs(rest - cand[j]) < 1e-12
    return j


@pytest.mark.parametrize("w_min,cases", [
    (1, [(1, 0), (2, 1), (3, 1), (4, 2), (5, 2), (7, 2), (8, 3), (9, 3), (1000, 3)]),
    (3, [(3, 0), (5, 0), (6, 1), (7, 1), (11, 1), (12, 2), (13, 2), (23, 2), (24, 3),
         (25, 3), (10 ** 6, 3)]),
    (7, [(7, 0), (8, 0), (13, 0), (14, 1), (15, 1), (27, 1), (28, 2), (29, 2), (55, 2),
         (56, 3), (57, 3)]),
])
def test_weight_bucket_boundaries(w_min, cases):
    for w, want in cases:
        assert _bucket_chosen(w_min, w, 4) == want, (w_min, w)


def test_weight_bucket_hard_clause_and_limits():
    """A hard clause (weight 1 + the sum of the soft weights, as in the mixed-
    length workload) lands in the top bucket; J = 1 puts everything in bucket
    0; J = 2 stops at bucket 1; weights near 2^63 do not overflow the rule
    (2^61 and 2^63 - 1: 2^62 <= w < 2^63, so bucket 1)."""
    soft = [1, 100, 37]
    hard = 1 + sum(soft)
    assert _bucket_chosen(1, hard, 4) == 3
    assert _bucket_chosen(1, hard, 1) == 0
    assert _bucket_chosen(1, hard, 2) == 1
    assert _bucket_chosen(2 ** 61, 2 ** 63 - 1, 4) == 1
    assert _bucket_chosen(2 ** 61, 2 ** 62 - 1, 4) == 0


# --------------------------------------------------------------------------
# Sampled chains: a row of a run started with chain_ids is that chain of the
# full ensemble (the full-size GPU parity tests compare such samples).
# --------------------------------------------------------------------------
def test_sampled_chains_equal_rows_of_the_full_run(cfg1_table):
    inst = inst_of(workloads.random_ksat(20, 86, 3, seed=4))
    ids = np.array([0, 7, 8, 300, 511], np.int32)
    full = oracle.init_chains(20, 512, seed=11)
    oracle.gibbs(inst, cfg1_table, full, 12, seed=11, n_temps=2, threads=4)
    part = oracle.init_chains(20, 0, seed=11, chain_ids=ids, B_total=512)
    oracle.gibbs(inst, cfg1_table, part, 12, seed=11, n_temps=2)
    for f in ["x", "nu", "nu32", "best_cost", "best_x", "cost", "free_energy"]:
        assert np.array_equal(getattr(part, f), getattr(full, f)[ids]), f


def test_temperature_blocks_follow_the_global_chain_index(cfg1_table):
    """With E = 2 over 512 chains, chains 0..255 run the temperature-0 sets
    and chains 256..511 the temperature-1 sets: each block equals a run with
    E = 1 whose only sets are that temperature's (relabelled as 0)."""
    inst = inst_of(workloads.random_ksat(20, 86, 3, seed=4))
    ids = np.array([0, 7, 255, 256, 300, 511], np.int32)
    full = oracle.init_chains(20, 0, seed=11, chain_ids=ids, B_total=512)
    oracle.gibbs(inst, cfg1_table, full, 8, seed=11, n_temps=2)
    for e, rows in [(0, [0, 1, 2]), (1, [3, 4, 5])]:
        single = oracle.init_chains(20, 0, seed=11, chain_ids=ids[rows], B_total=512)
        oracle.gibbs(inst, cfg1_table.select(temps=[e]), single, 8, seed=11, n_temps=1)
        assert np.array_equal(single.x, full.x[rows]), e
        assert np.array_equal(single.best_cost, full.best_cost[rows]), e


# --------------------------------------------------------------------------
# Swap thresholds T[u] = ceil(2^20 ln(u / 65536)) against 60-digit arithmetic
# --------------------------------------------------------------------------
def test_swap_thresholds_match_high_precision_logs():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    T = oracle.swap_thresholds()
    assert T[0] == -np.inf
    scale = mpmath.mpf(2) ** 20
    for u in range(1, 65536):
        exact = scale * mpmath.log(mpmath.mpf(u) / 65536)
        assert T[u] == int(mpmath.ceil(exact)), u
