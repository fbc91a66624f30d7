"""RbmSAT oracle (Python side): test infrastructure, not product code.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this module. It shares no code with the CUDA library
``paper_2311_02101_gb300`` and never imports it.

Contents
--------
* ``fit_or_rbm`` -- fits a canonical OR-gate clause RBM by regressing its free
  energy on all 2^K inputs (Sec. 4.1 "Learning OR gate RBM parameters"; Adam at
  learning rate 1e-3, 3 hidden units for K = 3 and K + 1 for larger K, appendix
  "Pretraining"). General per-position weights W in R^{K x L}, as in the
  paper's ``W_c`` (Fig. code).
* ``quantise`` -- puts W on the 2^-Q grid and b on the 2^-24 grid (a reading:
  it makes every logit an exact double and every visible logit an exact
  multiple of 2^-Q, so two implementations can agree bit for bit).
* thin ctypes wrappers around ``rbmsat_oracle.c`` (literal-by-literal cost,
  initialisation, block Gibbs sampling, free energy);
* ``brute_force_optimum`` -- exact MaxSAT optimum by enumerating 2^n
  assignments (n <= 20);
* ``formula_rbm`` -- the dense formula-RBM matrices (W_f, b_f) of Sec. 4.1 for
  tiny instances, used by the pins that enumerate hidden states exactly.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from dataclasses import dataclass, field
from math import comb

import numpy as np

MAX_LEN = 12
MAX_H = 16
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rbmsat_oracle.c")


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o",
             tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u32, u64, f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        _lib.oracle_philox4x32_10.argtypes = [P, P, P]
        _lib.oracle_draw16.argtypes = [u64, u32, u32, u32, u32, u32]
        _lib.oracle_draw16.restype = u32
        _lib.oracle_eval.argtypes = [i32, i64, P, P, P, P, i32, P]
        _lib.oracle_init.argtypes = [i32, i32, u64, P, P, P, P, P, u32]
        _lib.oracle_gibbs.argtypes = [i32, i64, P, P, P, i32, P, P, P, P, P, P, i32, i32,
                                      f64, u64, i32, P, i32, u32, i32, P, P, P, P, P, P, P,
                                      i32, u32]
        _lib.oracle_unit_prop.argtypes = [i32, i64, P, P, P, P, P]
        _lib.oracle_free_energy.argtypes = [i32, i64, P, P, P, i32, P, P, P, P, P, P, i32,
                                            i32, P, i32, P]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Instances
# --------------------------------------------------------------------------
@dataclass
class Instance:
    """CNF in CSR form: clause c holds DIMACS literals lits[off[c]:off[c+1]]
    (signed, 1-based: the table T of Sec. 4.3); w[c] >= 1 is its weight."""

    n: int
    off: np.ndarray  # int64, m + 1
    lits: np.ndarray  # int32
    w: np.ndarray  # int64, m

    @property
    def m(self) -> int:
        return len(self.off) - 1

    @staticmethod
    def from_clauses(n, clauses, weights=None):
        off = np.zeros(len(clauses) + 1, np.int64)
        off[1:] = np.cumsum([len(c) for c in clauses])
        lits = np.array([l for c in clauses for l in c], np.int32)
        w = np.ones(len(clauses), np.int64) if weights is None else np.asarray(weights, np.int64)
        return Instance(n, off, lits, w)

    def clauses(self):
        return [list(self.lits[self.off[c]:self.off[c + 1]]) for c in range(self.m)]


# --------------------------------------------------------------------------
# OR-gate RBM fitting (Sec. 4.1; appendix "Pretraining")
# --------------------------------------------------------------------------
def hidden_units_for(length: int) -> int:
    """3 hidden units up to length 3, K + 1 above (appendix "Pretraining";
    lengths 1, 2 and 8..12 extend the rule)."""
    return 3 if length <= 3 else length + 1


def _softplus(a):
    return np.logaddexp(0.0, a)


def _sigmoid(a):
    return 1.0 / (1.0 + np.exp(-a))


def or_free_energy(W, b, V):
    """Clause free energy F(v) = -sum_h softplus(b_h + sum_k W_kh v_k), Eq. 1
    with no visible bias; V is (patterns x K)."""
    return -_softplus(V @ W + b).sum(axis=1)


def _adam(V, target, W, b, iters, lr, fit_w=True):
    params = [W.copy(), b.copy()]
    m1 = [np.zeros_like(p) for p in params]
    m2 = [np.zeros_like(p) for p in params]
    beta1, beta2, eps = 0.9, 0.999, 1e-8
    for it in range(1, iters + 1):
        a = V @ params[0] + params[1]
        r = -_softplus(a).sum(axis=1) - target  # F(v) - target
        g_a = (2.0 * r)[:, None] * (-_sigmoid(a))  # d loss / d a
        grads = [V.T @ g_a, g_a.sum(axis=0)]
        for j in range(2):
            if j == 0 and not fit_w:
                continue
            m1[j] = beta1 * m1[j] + (1 - beta1) * grads[j]
            m2[j] = beta2 * m2[j] + (1 - beta2) * grads[j] ** 2
            mh = m1[j] / (1 - beta1 ** it)
            vh = m2[j] / (1 - beta2 ** it)
            params[j] = params[j] - lr * mh / (np.sqrt(vh) + eps)
    return params


def fit_or_rbm(length: int, fstar: float, iters: int = 20000, lr: float = 1e-3,
               seed: int = 0, n_hidden: int | None = None):
    """Regress the clause free energy onto the OR-gate target: F(0) = 0 and
    F(v) = F_s = -fstar for every v != 0 (Sec. 4.1; F_s < 0 while the printed
    targets F* are positive, so F_s = -F*). Loss
    ||F(0)||^2 + sum_{v != 0} ||F(v) - F_s||^2 over all 2^K inputs, Adam at
    learning rate 1e-3. Returns (W (K x L), b (L)) in float64."""
    L = hidden_units_for(length) if n_hidden is None else n_hidden
    V = np.array(list(itertools.product([0.0, 1.0], repeat=length)), np.float64)
    target = np.where(V.sum(axis=1) == 0, 0.0, -fstar)
    rng = np.random.default_rng(seed)
    W0 = rng.normal(0.0, 0.1, (length, L))
    b0 = np.zeros(L)
    W, b = _adam(V, target, W0, b0, iters, lr)
    return W, b


def quantise(length: int, fstar: float, W, b, Q: int = 4, refit_iters: int = 2000,
             lr: float = 1e-3):
    """W -> round-half-even onto the 2^-Q grid; b refitted by Adam with W held
    fixed; b -> the 2^-24 grid."""
    Wq = np.rint(W * 2.0 ** Q) / 2.0 ** Q
    V = np.array(list(itertools.product([0.0, 1.0], repeat=length)), np.float64)
    target = np.where(V.sum(axis=1) == 0, 0.0, -fstar)
    _, b2 = _adam(V, target, Wq, b, refit_iters, lr, fit_w=False)
    bq = np.rint(b2 * 2.0 ** 24) / 2.0 ** 24
    return Wq, bq


def fit_loss(length, fstar, W, b):
    V = np.array(list(itertools.product([0.0, 1.0], repeat=length)), np.float64)
    target = np.where(V.sum(axis=1) == 0, 0.0, -fstar)
    r = or_free_energy(W, b, V) - target
    return float((r * r).sum())


@dataclass
class RbmTable:
    """Parameter sets keyed by (clause length, weight bucket, temperature)."""

    sets: list = field(default_factory=list)  # dicts: len, bucket, temp, W, b, target

    def add(self, length, bucket, temp, W, b, target=None):
        self.sets.append(dict(len=int(length), bucket=int(bucket), temp=int(temp),
                              W=np.asarray(W, np.float64), b=np.asarray(b, np.float64),
                              target=target))

    def get(self, length, bucket, temp):
        for s in self.sets:
            if (s["len"], s["bucket"], s["temp"]) == (length, bucket, temp):
                return s
        raise KeyError((length, bucket, temp))

    def arrays(self):
        S = len(self.sets)
        ln = np.array([s["len"] for s in self.sets], np.int32)
        bk = np.array([s["bucket"] for s in self.sets], np.int32)
        tp = np.array([s["temp"] for s in self.sets], np.int32)
        nh = np.array([s["W"].shape[1] for s in self.sets], np.int32)
        W = np.zeros((S, MAX_LEN, MAX_H), np.float64)
        b = np.zeros((S, MAX_H), np.float64)
        for i, s in enumerate(self.sets):
            K, L = s["W"].shape
            W[i, :K, :L] = s["W"]
            b[i, :L] = s["b"]
        return ln, bk, tp, nh, W, b

    # text format: one header line per set, then K lines of W, then one of b
    def save(self, path, header=""):
        with open(path, "w") as f:
            for line in header.strip().splitlines():
                f.write("# " + line + "\n")
            for s in self.sets:
                K, L = s["W"].shape
                f.write(f"set {s['len']} {s['bucket']} {s['temp']} {L} {s['target']!r}\n")
                for k in range(K):
                    f.write("W " + " ".join(repr(float(v)) for v in s["W"][k]) + "\n")
                f.write("b " + " ".join(repr(float(v)) for v in s["b"]) + "\n")

    @staticmethod
    def load(path):
        t = RbmTable()
        cur = None
        with open(path) as f:
            for line in f:
                line = line.strip()
                if not line or line.startswith("#"):
                    continue
                tok = line.split()
                if tok[0] == "set":
                    cur = dict(len=int(tok[1]), bucket=int(tok[2]), temp=int(tok[3]),
                               L=int(tok[4]), target=float(tok[5]), W=[], b=None)
                    t.sets.append(cur)
                elif tok[0] == "W":
                    cur["W"].append([float(v) for v in tok[1:]])
                elif tok[0] == "b":
                    cur["b"] = np.array([float(v) for v in tok[1:]], np.float64)
                    cur["W"] = np.array(cur["W"], np.float64).reshape(cur["len"], cur["L"])
        for s in t.sets:
            s.pop("L", None)
        return t

    def select(self, temps=None, buckets=None, lengths=None):
        """Sub-table; `temps` maps new temperature index -> stored index."""
        out = RbmTable()
        for s in self.sets:
            if lengths is not None and s["len"] not in lengths:
                continue
            if buckets is not None and s["bucket"] >= buckets:
                continue
            if temps is not None:
                if s["temp"] not in temps:
                    continue
                for new, old in enumerate(temps):
                    if old == s["temp"]:
                        out.add(s["len"], s["bucket"], new, s["W"], s["b"], s["target"])
            else:
                out.add(s["len"], s["bucket"], s["temp"], s["W"], s["b"], s["target"])
        return out


def bucket_target(fstar: float, bucket: int, gamma: float) -> float:
    """Target F* of weight bucket j: F*_e (1 + j gamma) (reading; the paper is
    unweighted)."""
    return fstar * (1.0 + bucket * gamma)


def make_table(lengths, fstars, n_buckets=1, gamma=0.5, Q=4, iters=20000, seed=0):
    t = RbmTable()
    for e, fs in enumerate(fstars):
        for j in range(n_buckets):
            tgt = bucket_target(fs, j, gamma)
            for K in lengths:
                W, b = fit_or_rbm(K, tgt, iters=iters, seed=seed)
                Wq, bq = quantise(K, tgt, W, b, Q=Q)
                t.add(K, j, e, Wq, bq, tgt)
    return t


# --------------------------------------------------------------------------
# ctypes wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def draw16(seed, phase, t, a, h, b):
    return int(lib().oracle_draw16(seed, phase, t, a, h, b))


def evaluate(inst: Instance, x: np.ndarray) -> np.ndarray:
    """Weighted unsatisfied cost of each row of x (B x n, {0,1})."""
    x = np.ascontiguousarray(x, np.uint8)
    B = x.shape[0]
    cost = np.zeros(B, np.int64)
    lib().oracle_eval(inst.n, inst.m, _ptr(inst.off), _ptr(inst.lits), _ptr(inst.w),
                      _ptr(x), B, _ptr(cost))
    return cost


@dataclass
class ChainState:
    x: np.ndarray  # B x n uint8
    nu: np.ndarray  # B x n float64
    best_cost: np.ndarray  # B int64
    best_x: np.ndarray  # B x n uint8
    cost: np.ndarray  # B int64 (last scored state)
    free_energy: np.ndarray  # B float64 (last scored state)
    t: int = 0
    chain_ids: np.ndarray | None = None  # global chain index of each row
    B_total: int = 0  # ensemble size the temperatures are spread over
    instance: int = 0  # index of the formula in a batch (draws carry it)
    nu32: np.ndarray | None = None  # B x n float32: nu in the solver's FP32 sequence

    def copy(self):
        return ChainState(self.x.copy(), self.nu.copy(), self.best_cost.copy(),
                          self.best_x.copy(), self.cost.copy(), self.free_energy.copy(), self.t,
                          None if self.chain_ids is None else self.chain_ids.copy(), self.B_total,
                          self.instance, None if self.nu32 is None else self.nu32.copy())


def init_chains(n: int, B: int, seed: int, chain_ids=None, B_total=None,
                instance: int = 0) -> ChainState:
    """B chains; with `chain_ids`, row r is chain chain_ids[r] of an ensemble
    of B_total chains (so a sample of a large run can be reproduced).
    `instance` is the formula's index in a batch: its draws carry it in the
    high 24 bits of the phase word."""
    if chain_ids is not None:
        chain_ids = np.ascontiguousarray(chain_ids, np.int32)
        B = len(chain_ids)
    x = np.zeros((B, n), np.uint8)
    nu = np.zeros((B, n), np.float64)
    nu32 = np.zeros((B, n), np.float32)
    best = np.zeros(B, np.int64)
    lib().oracle_init(n, B, seed, _ptr(chain_ids), _ptr(x), _ptr(nu), _ptr(nu32), _ptr(best),
                      instance)
    return ChainState(x, nu, best, x.copy(), np.zeros(B, np.int64), np.zeros(B), 0,
                      chain_ids, int(B_total if B_total is not None else B), int(instance), nu32)


def gibbs(inst: Instance, table: RbmTable, st: ChainState, steps: int, seed: int,
          n_temps: int, n_buckets: int = 1, alpha: float = 0.01,
          threads: int = 1) -> ChainState:
    """`steps` rounds of block Gibbs sampling, in place on `st`."""
    ln, bk, tp, nh, W, b = table.arrays()
    B = st.x.shape[0]
    rc = lib().oracle_gibbs(inst.n, inst.m, _ptr(inst.off), _ptr(inst.lits), _ptr(inst.w),
                            len(ln), _ptr(ln), _ptr(bk), _ptr(tp), _ptr(nh), _ptr(W), _ptr(b),
                            n_temps, n_buckets, alpha, seed, B, _ptr(st.chain_ids),
                            st.B_total or B, st.t, steps,
                            _ptr(st.x), _ptr(st.nu), _ptr(st.nu32), _ptr(st.best_cost),
                            _ptr(st.best_x),
                            _ptr(st.cost), _ptr(st.free_energy), threads, st.instance)
    if rc != 0:
        raise ValueError("a clause has no RBM parameter set")
    st.t += steps
    return st


def score_and_keep(inst: Instance, st: ChainState) -> ChainState:
    """Score the current states once more and update the best-so-far
    (the final evaluation after the last step)."""
    cost = evaluate(inst, st.x)
    st.cost = cost
    better = cost < st.best_cost
    st.best_cost = np.where(better, cost, st.best_cost)
    st.best_x[better] = st.x[better]
    return st


def solve(inst, table, B, steps, seed, n_temps, n_buckets=1, alpha=0.01, threads=1,
          instance=0):
    """reset + `steps` rounds + final score; returns (best cost, best
    assignment, chain state). Ties go to the lowest chain index."""
    st = init_chains(inst.n, B, seed, instance=instance)
    gibbs(inst, table, st, steps, seed, n_temps, n_buckets, alpha, threads)
    score_and_keep(inst, st)
    b = int(np.argmin(st.best_cost))
    return int(st.best_cost[b]), st.best_x[b].copy(), st


def unit_prop(inst: Instance, x, nu32):
    """Prioritized unit propagation (Sec. 4.4) of each row of x (B x n, or
    one assignment) ranked by the FP32 nu of the same shape; see
    oracle_unit_prop for the steps."""
    x = np.ascontiguousarray(np.atleast_2d(x), np.uint8)
    nu32 = np.ascontiguousarray(np.atleast_2d(nu32), np.float32)
    out = np.zeros_like(x)
    for b in range(x.shape[0]):
        lib().oracle_unit_prop(inst.n, inst.m, _ptr(inst.off), _ptr(inst.lits), _ptr(x[b]),
                               _ptr(nu32[b]), _ptr(out[b]))
    return out


def up_merge(inst: Instance, st: ChainState, up_x) -> ChainState:
    """The B-of-2B merge of the appendix code: the B current states and the B
    unit-propagation results are stacked (current first), scored, sorted by
    satisfied weight ascending with a stable sort, and the last B rows become
    the new chains in that order; nu rows follow their states (the results
    inherit the nu of the chain they came from). In place on st."""
    B = st.x.shape[0]
    cand = np.vstack([st.x, np.asarray(up_x, np.uint8)])
    cost = evaluate(inst, cand)
    ranks = np.argsort(-cost, kind="stable")  # satisfied weight ascending
    sel = ranks[-B:]
    st.x = np.ascontiguousarray(cand[sel])
    st.nu = np.ascontiguousarray(np.vstack([st.nu, st.nu])[sel])
    st.nu32 = np.ascontiguousarray(np.vstack([st.nu32, st.nu32])[sel])
    return st


def flip_proposals(x, prob, tau):
    """Each row of x with every confident variable set to the network's
    value: 1 where prob >= 1 - tau, 0 where prob <= tau (prob compared in
    FP32, as given)."""
    prob = np.asarray(prob, np.float32)
    out = np.array(x, np.uint8, copy=True)
    out[:, prob >= np.float32(1.0) - np.float32(tau)] = 1
    out[:, prob <= np.float32(tau)] = 0
    return out


def free_energy(inst, table, x, temp, n_buckets=1, fixed=False):
    """Formula free energy (Eq. 1) of each row of x at temperature `temp`;
    with fixed=True also its fixed-point form sum_c rint(2^20 F_c) (int64)."""
    ln, bk, tp, nh, W, b = table.arrays()
    x = np.ascontiguousarray(x, np.uint8)
    B = x.shape[0]
    F = np.zeros(B, np.float64)
    Fq = np.zeros(B, np.int64)
    rc = lib().oracle_free_energy(inst.n, inst.m, _ptr(inst.off), _ptr(inst.lits),
                                  _ptr(inst.w), len(ln), _ptr(ln), _ptr(bk), _ptr(tp),
                                  _ptr(nh), _ptr(W), _ptr(b), n_buckets, temp, _ptr(x), B,
                                  _ptr(F), _ptr(Fq))
    if rc != 0:
        raise ValueError("a clause has no RBM parameter set")
    return (F, Fq) if fixed else F


PH_SWAP = 4  # draw phase of parallel-tempering swaps


def swap_thresholds():
    """T[u] = ceil(2^20 ln(u / 65536)) for the 16-bit draw u (T[0] = -inf):
    a swap with fixed-point log-ratio D (units 2^-20) is accepted iff D >= T[u],
    i.e. iff u < 65536 exp(D 2^-20)."""
    import math
    T = np.empty(65536, np.float64)
    T[0] = -np.inf
    T[1:] = [math.ceil(math.ldexp(math.log(u / 65536.0), 20)) for u in range(1, 65536)]
    return T


def pt_swap(inst, table, st, seed, parity, n_temps, n_buckets=1):
    """One parallel-tempering swap round on the ensemble st (B chains in E
    contiguous temperature blocks of S = B / E; S a multiple of 8). For every
    block e = parity, parity + 2, ... with e + 1 < E, chain a = e S + k and
    chain b = a + S exchange their states (x, nu) iff
        D = F_e(x_a) + F_{e+1}(x_b) - F_e(x_b) - F_{e+1}(x_a) >= T[u],
    F in the fixed-point form, u the 16-bit draw of chain a in phase 4 at the
    current round (Metropolis acceptance min(1, exp(D)) of exchanging two
    states between the targets exp(-F_e) and exp(-F_{e+1})). The best-so-far
    stays with the chain index. In place; returns the number of swaps."""
    B = st.x.shape[0]
    E = n_temps
    S = B // E
    assert B % E == 0 and S % 8 == 0 and st.chain_ids is None
    T = swap_thresholds()
    done = 0
    for e in range(parity, E - 1, 2):
        a = np.arange(e * S, (e + 1) * S)
        b = a + S
        _, Fa0 = free_energy(inst, table, st.x[a], e, n_buckets, fixed=True)
        _, Fa1 = free_energy(inst, table, st.x[a], e + 1, n_buckets, fixed=True)
        _, Fb0 = free_energy(inst, table, st.x[b], e, n_buckets, fixed=True)
        _, Fb1 = free_energy(inst, table, st.x[b], e + 1, n_buckets, fixed=True)
        D = Fa0 + Fb1 - Fb0 - Fa1
        u = np.array([draw16(seed, PH_SWAP, st.t, 0, 0, int(k)) for k in a])
        ok = D >= T[u]
        for arr in (st.x, st.nu, st.nu32):
            if arr is None:
                continue
            tmp = arr[a[ok]].copy()
            arr[a[ok]] = arr[b[ok]]
            arr[b[ok]] = tmp
        done += int(ok.sum())
    return done


# --------------------------------------------------------------------------
# Exact references for small cases
# --------------------------------------------------------------------------
def all_assignments(n: int) -> np.ndarray:
    """All 2^n assignments, row r = binary digits of r (variable 0 = LSB)."""
    r = np.arange(2 ** n, dtype=np.int64)
    return ((r[:, None] >> np.arange(n)) & 1).astype(np.uint8)


def brute_force_optimum(inst: Instance, chunk: int = 1 << 16):
    """Exact minimum weighted cost over all 2^n assignments (n <= 20)."""
    assert inst.n <= 20
    best = None
    for start in range(0, 2 ** inst.n, chunk):
        r = np.arange(start, min(start + chunk, 2 ** inst.n), dtype=np.int64)
        X = ((r[:, None] >> np.arange(inst.n)) & 1).astype(np.uint8)
        c = evaluate(inst, X).min()
        best = c if best is None else min(best, c)
    return int(best)


def formula_rbm(inst: Instance, table: RbmTable, temp: int, n_buckets: int = 1):
    """Dense formula-RBM parameters (W_f: n x sum_c L_c, b_f) built clause by
    clause from Eq. 4 and concatenated as in Sec. 4.1 (visible bias d = 0).
    For tiny instances only."""
    wmin = int(inst.w.min())
    cols_W, cols_b = [], []
    for c in range(inst.m):
        lits = inst.lits[inst.off[c]:inst.off[c + 1]]
        K = len(lits)
        if K == 0:
            continue
        j = 0
        while j + 1 < n_buckets and wmin * 2 ** (j + 1) <= int(inst.w[c]):
            j += 1
        s = table.get(K, j, temp)
        W, b = s["W"], s["b"]
        L = W.shape[1]
        lam = np.where(lits > 0, 1.0, -1.0)
        Wp = lam[:, None] * W
        bp = b + 0.5 * ((1.0 - lam)[:, None] * W).sum(axis=0)
        Wc = np.zeros((inst.n, L))
        for k, l in enumerate(lits):
            Wc[abs(int(l)) - 1] += Wp[k]
        cols_W.append(Wc)
        cols_b.append(bp)
    if not cols_W:
        return np.zeros((inst.n, 0)), np.zeros(0)
    return np.concatenate(cols_W, axis=1), np.concatenate(cols_b)
