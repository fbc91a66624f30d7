"""Thin ctypes binding of libmaxsat.so (include/maxsat.h): argument marshalling
only. Every step of a Gibbs round runs in the library's CUDA kernels; PyTorch
provides device buffers and streams. There is no CPU fallback: importing
works without a GPU, but the library must have been built (``build()``), and
calls that need the device fail with MaxsatError(MAXSAT_ENODEV) without one.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAXSAT_OK = 0
MAXSAT_EINVAL = -1
MAXSAT_ENOMEM = -2
MAXSAT_ECUDA = -3
MAXSAT_ENODEV = -4
MAXSAT_ESTATE = -5
MAXSAT_MAX_LEN = 12
MAXSAT_MAX_HIDDEN = 16
MAXSAT_PATH_AUTO = 0
MAXSAT_PATH_DENSE = 1
MAXSAT_PATH_SPARSE = 2

LIB_PATH = _build.LIB


class MaxsatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class maxsat_rbm_set(ctypes.Structure):
    _fields_ = [("len", ctypes.c_int32), ("bucket", ctypes.c_int32), ("temp", ctypes.c_int32),
                ("n_hidden", ctypes.c_int32), ("W", ctypes.c_void_p), ("b", ctypes.c_void_p)]


class maxsat_params(ctypes.Structure):
    _fields_ = [("n_temps", ctypes.c_int32), ("fstar", ctypes.c_void_p),
                ("n_buckets", ctypes.c_int32), ("bucket_gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("quant_bits", ctypes.c_int32),
                ("path", ctypes.c_int32), ("fit_iters", ctypes.c_int32),
                ("n_sets", ctypes.c_int32), ("sets", ctypes.POINTER(maxsat_rbm_set)),
                ("steps_per_graph", ctypes.c_int32), ("tune_blocks", ctypes.c_int32),
                ("up_device", ctypes.c_int32), ("visible_batch", ctypes.c_int32),
                ("persistent_round", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmaxsat.so is not built ({LIB_PATH}); run "
                               "__graft_entry__.build() or paper_2311_02101_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u32, u64, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
        L.maxsat_default_params.argtypes = [ctypes.POINTER(maxsat_params)]
        L.maxsat_default_params.restype = None
        L.maxsat_create.argtypes = [ctypes.POINTER(P), i32, i64, P, P, P,
                                    ctypes.POINTER(maxsat_params), P]
        L.maxsat_create_batch.argtypes = [ctypes.POINTER(P), i32, P, P, P, P, P,
                                          ctypes.POINTER(maxsat_params), P]
        L.maxsat_get_n_instances.argtypes = [P]
        L.maxsat_get_clause_block.argtypes = [P]
        L.maxsat_get_visible_batch.argtypes = [P]
        L.maxsat_get_persistent_round.argtypes = [P]
        L.maxsat_mp_create.argtypes = [ctypes.POINTER(P), i32, u64]
        L.maxsat_mp_n_params.argtypes = [P]
        L.maxsat_mp_set_params.argtypes = [P, P]
        L.maxsat_mp_get_params.argtypes = [P, P, P]
        L.maxsat_mp_forward.argtypes = [P, P, P]
        L.maxsat_mp_gradient.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_double)]
        L.maxsat_mp_adam.argtypes = [P, P, ctypes.c_float]
        L.maxsat_mp_last_error.argtypes = [P]
        L.maxsat_mp_last_error.restype = ctypes.c_char_p
        L.maxsat_mp_destroy.argtypes = [P]
        L.maxsat_mp_destroy.restype = None
        L.maxsat_reset_probs.argtypes = [P, i32, u64, P]
        L.maxsat_propose_flips.argtypes = [P, P, ctypes.c_float]
        L.maxsat_pt_swap.argtypes = [P, i32, ctypes.POINTER(i32)]
        L.maxsat_up_begin.argtypes = [P]
        L.maxsat_up_end.argtypes = [P]
        L.maxsat_up.argtypes = [P]
        L.maxsat_reset.argtypes = [P, i32, u64]
        L.maxsat_reset_shard.argtypes = [P, i32, u64, i32, i32]
        L.maxsat_step.argtypes = [P, i64]
        L.maxsat_score.argtypes = [P]
        L.maxsat_eval.argtypes = [P, P, i32, P]
        L.maxsat_solve.argtypes = [P, i32, i64, u64, P, P]
        L.maxsat_solve_timed.argtypes = [P, i32, f64, i64, i64, u64, P, P, P]
        L.maxsat_get_state.argtypes = [P, P, P, P, P, P, P, P]
        L.maxsat_set_state.argtypes = [P, i32, u64, P, P, P, P, u32]
        L.maxsat_get_path.argtypes = [P]
        L.maxsat_destroy.argtypes = [P]
        L.maxsat_destroy.restype = None
        L.maxsat_last_error.argtypes = [P]
        L.maxsat_last_error.restype = ctypes.c_char_p
        L.maxsat_fit_or_rbm.argtypes = [i32, i32, f64, i32, i32, P, P]
        L.maxsat_eval_noalloc.argtypes = [i32, i64, i64, P, P, P, P, i32, P, P]
        L.maxsat_set_profiling.argtypes = [P, i32]
        L.maxsat_kernel_times.argtypes = [P, i32, P, P, P]
        for name in ["maxsat_create", "maxsat_create_batch", "maxsat_get_n_instances",
                     "maxsat_get_clause_block", "maxsat_get_visible_batch",
                     "maxsat_get_persistent_round", "maxsat_up_begin",
                     "maxsat_up_end", "maxsat_up",
                     "maxsat_mp_create", "maxsat_mp_n_params", "maxsat_mp_set_params",
                     "maxsat_mp_get_params", "maxsat_mp_forward", "maxsat_mp_gradient",
                     "maxsat_mp_adam", "maxsat_reset_probs", "maxsat_pt_swap",
                     "maxsat_propose_flips",
                     "maxsat_reset", "maxsat_reset_shard", "maxsat_step",
                     "maxsat_score",
                     "maxsat_eval", "maxsat_solve", "maxsat_solve_timed", "maxsat_get_state",
                     "maxsat_set_state",
                     "maxsat_get_path", "maxsat_fit_or_rbm", "maxsat_set_profiling",
                     "maxsat_kernel_times", "maxsat_eval_noalloc"]:
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, ctx=None):
    if rc != MAXSAT_OK:
        raise MaxsatError(rc, maxsat_last_error(ctx))
    return rc


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Context:
    """Opaque solver handle (the C maxsat_ctx*) plus the few facts the binding
    needs for marshalling."""

    def __init__(self, handle, n, m, n_inst=1, var_base=None):
        self.handle = handle
        self.n = n          # variables (of all formulas of a batch)
        self.m = m
        self.n_inst = n_inst
        self.var_base = var_base if var_base is not None else np.array([0, n], np.int64)
        self.B = 0

    def __del__(self):
        try:
            maxsat_destroy(self)
        except Exception:
            pass


def maxsat_default_params(**overrides):
    """A maxsat_params with the library defaults, fields overridden by keyword;
    `fstar` (list of floats) and `sets` (list of dicts with len, bucket, temp,
    W, b) are converted; the returned object keeps their buffers alive."""
    p = maxsat_params()
    lib().maxsat_default_params(ctypes.byref(p))
    keep = []
    for k, v in overrides.items():
        if k == "fstar":
            arr = np.ascontiguousarray(v, np.float64)
            keep.append(arr)
            p.fstar = arr.ctypes.data
            p.n_temps = len(arr)
        elif k == "sets":
            sets = list(v)
            S = (maxsat_rbm_set * max(1, len(sets)))()
            for i, s in enumerate(sets):
                W = np.ascontiguousarray(s["W"], np.float64)
                b = np.ascontiguousarray(s["b"], np.float64)
                keep += [W, b]
                S[i] = maxsat_rbm_set(int(s["len"]), int(s["bucket"]), int(s["temp"]),
                                      int(W.shape[1]), W.ctypes.data, b.ctypes.data)
            keep.append(S)
            p.sets = ctypes.cast(S, ctypes.POINTER(maxsat_rbm_set))
            p.n_sets = len(sets)
        else:
            setattr(p, k, v)
    p._keep = keep
    return p


def maxsat_create(n, off, lits, weights=None, params=None, stream=None) -> Context:
    off = np.ascontiguousarray(off, np.int64)
    lits = np.ascontiguousarray(lits, np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, np.int64)
    h = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    rc = lib().maxsat_create(ctypes.byref(h), int(n), len(off) - 1, _np_ptr(off), _np_ptr(lits),
                             _np_ptr(w), pp, _stream_handle(stream))
    _check(rc, None)
    return Context(h.value, int(n), len(off) - 1)


def maxsat_create_batch(instances, params=None, stream=None) -> Context:
    """instances: sequence of (n, off, lits, weights-or-None), literals local
    to each formula. One context runs all of them (maxsat_create_batch)."""
    nv = np.array([int(i[0]) for i in instances], np.int32)
    offs = [np.ascontiguousarray(i[1], np.int64) for i in instances]
    nc = np.array([len(o) - 1 for o in offs], np.int64)
    base = np.concatenate([[0], np.cumsum([o[-1] for o in offs])]).astype(np.int64)
    off = np.concatenate([[0]] + [o[1:] + base[k] for k, o in enumerate(offs)]).astype(np.int64)
    lits = np.ascontiguousarray(np.concatenate([np.asarray(i[2], np.int32) for i in instances]),
                                np.int32)
    if all(i[3] is None for i in instances):
        w = None
    else:
        w = np.ascontiguousarray(np.concatenate(
            [np.ones(len(o) - 1, np.int64) if i[3] is None else np.asarray(i[3], np.int64)
             for i, o in zip(instances, offs)]), np.int64)
    h = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    rc = lib().maxsat_create_batch(ctypes.byref(h), len(instances), _np_ptr(nv), _np_ptr(nc),
                                   _np_ptr(off), _np_ptr(lits), _np_ptr(w), pp,
                                   _stream_handle(stream))
    _check(rc, None)
    var_base = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
    return Context(h.value, int(var_base[-1]), int(nc.sum()), len(instances), var_base)


def maxsat_get_n_instances(ctx: Context) -> int:
    return int(lib().maxsat_get_n_instances(ctx.handle))


def maxsat_get_clause_block(ctx: Context) -> int:
    return int(lib().maxsat_get_clause_block(ctx.handle))


def maxsat_get_visible_batch(ctx: Context) -> int:
    return int(lib().maxsat_get_visible_batch(ctx.handle))


def maxsat_get_persistent_round(ctx: Context) -> int:
    return int(lib().maxsat_get_persistent_round(ctx.handle))


def maxsat_reset(ctx: Context, restarts: int, seed: int):
    _check(lib().maxsat_reset(ctx.handle, int(restarts), int(seed) & (2 ** 64 - 1)), ctx)
    ctx.B = int(restarts)


def maxsat_reset_shard(ctx: Context, restarts: int, seed: int, chain_offset: int,
                       total_chains: int):
    _check(lib().maxsat_reset_shard(ctx.handle, int(restarts), int(seed) & (2 ** 64 - 1),
                                    int(chain_offset), int(total_chains)), ctx)
    ctx.B = int(restarts)


def maxsat_step(ctx: Context, steps: int):
    _check(lib().maxsat_step(ctx.handle, int(steps)), ctx)


def maxsat_score(ctx: Context):
    _check(lib().maxsat_score(ctx.handle), ctx)


def maxsat_eval(ctx: Context, assign_dev, cost_dev):
    """assign_dev: torch uint8 CUDA tensor (B x n, contiguous); cost_dev: torch
    int64 CUDA tensor (B; n_inst x B for a batch)."""
    B = int(assign_dev.shape[0])
    assert assign_dev.is_cuda and cost_dev.is_cuda and assign_dev.is_contiguous()
    assert tuple(assign_dev.shape) == (B, ctx.n) and cost_dev.numel() >= B * ctx.n_inst
    _check(lib().maxsat_eval(ctx.handle, assign_dev.data_ptr(), B, cost_dev.data_ptr()), ctx)


def maxsat_eval_noalloc(n, off_dev, lits_dev, weights_dev, assign_dev, cost_dev, stream=None):
    """Allocation-free evaluation (no context): all arguments are contiguous
    torch tensors on the current CUDA device (int64 offsets, int32 DIMACS
    literals, int64 weights or None, uint8 B x n assignments, int64 B costs).
    stream=None runs on torch's current stream. Every tensor is checked here,
    because the C entry point trusts the pointers and sizes it is given."""
    import torch
    dev = torch.cuda.current_device()
    named = [("off_dev", off_dev, torch.int64), ("lits_dev", lits_dev, torch.int32),
             ("assign_dev", assign_dev, torch.uint8), ("cost_dev", cost_dev, torch.int64)]
    if weights_dev is not None:
        named.append(("weights_dev", weights_dev, torch.int64))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be on the current CUDA device (cuda:{dev})")
        if t.dtype != dt:
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if off_dev.dim() != 1 or off_dev.numel() < 1:
        raise ValueError("off_dev must hold n_clauses + 1 offsets")
    if assign_dev.dim() != 2 or int(assign_dev.shape[1]) != int(n):
        raise ValueError(f"assign_dev must be B x {int(n)}")
    m = int(off_dev.numel()) - 1
    B = int(assign_dev.shape[0])
    if weights_dev is not None and weights_dev.numel() < m:
        raise ValueError(f"weights_dev holds {weights_dev.numel()} weights for {m} clauses")
    if cost_dev.numel() < B:
        raise ValueError(f"cost_dev holds {cost_dev.numel()} entries for {B} assignments")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().maxsat_eval_noalloc(int(n), m, int(lits_dev.numel()), off_dev.data_ptr(),
                                     lits_dev.data_ptr(),
                                     None if weights_dev is None else weights_dev.data_ptr(),
                                     assign_dev.data_ptr(), B, cost_dev.data_ptr(),
                                     _stream_handle(stream)))


def maxsat_solve(ctx: Context, restarts: int, steps: int, seed: int):
    """Returns (best cost, best assignment as n uint8); for a batch, (n_inst
    best costs, every formula's best assignment over all variables)."""
    best = np.zeros(ctx.n, np.uint8)
    cost = np.zeros(ctx.n_inst, np.int64)
    _check(lib().maxsat_solve(ctx.handle, int(restarts), int(steps), int(seed) & (2 ** 64 - 1),
                              _np_ptr(best), _np_ptr(cost)), ctx)
    ctx.B = int(restarts)
    if ctx.n_inst == 1:
        return int(cost[0]), best
    return cost, best


def maxsat_solve_timed(ctx: Context, restarts: int, seconds: float, seed: int,
                       max_steps: int = 2 ** 62, chunk: int = 0):
    """maxsat_solve under a wall-clock budget; returns (best cost(s), best
    assignment, rounds run)."""
    best = np.zeros(ctx.n, np.uint8)
    cost = np.zeros(ctx.n_inst, np.int64)
    done = ctypes.c_int64(0)
    _check(lib().maxsat_solve_timed(ctx.handle, int(restarts), float(seconds), int(max_steps),
                                    int(chunk), int(seed) & (2 ** 64 - 1), _np_ptr(best),
                                    _np_ptr(cost), ctypes.byref(done)), ctx)
    ctx.B = int(restarts)
    if ctx.n_inst == 1:
        return int(cost[0]), best, int(done.value)
    return cost, best, int(done.value)


def maxsat_get_state(ctx: Context):
    """Chain state; best_cost, cost and free_energy are (B,) for one formula
    and (n_inst, B) for a batch."""
    B, n, K = ctx.B, ctx.n, ctx.n_inst
    shp = (B,) if K == 1 else (K, B)
    out = dict(x=np.zeros((B, n), np.uint8), nu=np.zeros((B, n), np.float32),
               best_cost=np.zeros(shp, np.int64), best_x=np.zeros((B, n), np.uint8),
               cost=np.zeros(shp, np.int64), free_energy=np.zeros(shp, np.float32))
    t = ctypes.c_uint32()
    _check(lib().maxsat_get_state(ctx.handle, _np_ptr(out["x"]), _np_ptr(out["nu"]),
                                  _np_ptr(out["best_cost"]), _np_ptr(out["best_x"]),
                                  _np_ptr(out["cost"]), _np_ptr(out["free_energy"]),
                                  ctypes.byref(t)), ctx)
    out["t"] = int(t.value)
    return out


def maxsat_set_state(ctx: Context, restarts, seed, x, nu, best_cost, best_x, t):
    x = np.ascontiguousarray(x, np.uint8)
    nu = np.ascontiguousarray(nu, np.float32)
    best_cost = np.ascontiguousarray(best_cost, np.int64)
    best_x = np.ascontiguousarray(best_x, np.uint8)
    _check(lib().maxsat_set_state(ctx.handle, int(restarts), int(seed) & (2 ** 64 - 1),
                                  _np_ptr(x), _np_ptr(nu), _np_ptr(best_cost), _np_ptr(best_x),
                                  int(t)), ctx)
    ctx.B = int(restarts)


def maxsat_set_profiling(ctx: Context, on: bool):
    _check(lib().maxsat_set_profiling(ctx.handle, 1 if on else 0), ctx)


def maxsat_kernel_times(ctx: Context, max_kernels: int = 32):
    """{kernel name: (launches, total device ms)} since profiling was enabled."""
    names = ctypes.create_string_buffer(32 * max_kernels)
    cnt = np.zeros(max_kernels, np.int64)
    ms = np.zeros(max_kernels, np.float64)
    k = lib().maxsat_kernel_times(ctx.handle, max_kernels, names, _np_ptr(cnt), _np_ptr(ms))
    if k < 0:
        _check(k, ctx)
    raw = names.raw
    return {raw[32 * i:32 * i + 32].split(b"\0")[0].decode(): (int(cnt[i]), float(ms[i]))
            for i in range(k)}


def maxsat_pt_swap(ctx: Context, parity: int) -> int:
    """One parallel-tempering swap round; returns the number of swaps."""
    acc = ctypes.c_int32()
    _check(lib().maxsat_pt_swap(ctx.handle, int(parity), ctypes.byref(acc)), ctx)
    return int(acc.value)


def maxsat_up_begin(ctx: Context):
    _check(lib().maxsat_up_begin(ctx.handle), ctx)


def maxsat_up_end(ctx: Context):
    _check(lib().maxsat_up_end(ctx.handle), ctx)


def maxsat_up(ctx: Context):
    _check(lib().maxsat_up(ctx.handle), ctx)


class Model:
    """Handle of a learned-proposal network (the C maxsat_mp*)."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        try:
            maxsat_mp_destroy(self)
        except Exception:
            pass


def _check_mp(rc, mp=None):
    if rc != MAXSAT_OK:
        h = None if mp is None else mp.handle
        raise MaxsatError(rc, lib().maxsat_mp_last_error(h).decode())
    return rc


def maxsat_mp_create(n_layers: int = 3, seed: int = 0) -> Model:
    h = ctypes.c_void_p()
    _check_mp(lib().maxsat_mp_create(ctypes.byref(h), int(n_layers), int(seed) & (2 ** 64 - 1)))
    return Model(h.value)


def maxsat_mp_n_params(mp: Model) -> int:
    return int(lib().maxsat_mp_n_params(mp.handle))


def maxsat_mp_set_params(mp: Model, theta):
    theta = np.ascontiguousarray(theta, np.float32)
    assert theta.size == maxsat_mp_n_params(mp)
    _check_mp(lib().maxsat_mp_set_params(mp.handle, _np_ptr(theta)), mp)


def maxsat_mp_get_params(mp: Model):
    """(parameters, last gradient) as FP32 host vectors."""
    k = maxsat_mp_n_params(mp)
    theta, grad = np.zeros(k, np.float32), np.zeros(k, np.float32)
    _check_mp(lib().maxsat_mp_get_params(mp.handle, _np_ptr(theta), _np_ptr(grad)), mp)
    return theta, grad


def maxsat_mp_forward(mp: Model, ctx: Context, prob_dev):
    """prob_dev: torch float32 CUDA tensor of ctx.n elements."""
    assert prob_dev.is_cuda and prob_dev.numel() >= ctx.n
    _check_mp(lib().maxsat_mp_forward(mp.handle, ctx.handle, prob_dev.data_ptr()), mp)


def maxsat_mp_gradient(mp: Model, ctx: Context, labels_dev) -> float:
    """labels_dev: torch uint8 CUDA tensor (0 / 1) of ctx.n elements."""
    assert labels_dev.is_cuda and labels_dev.numel() >= ctx.n
    loss = ctypes.c_double()
    _check_mp(lib().maxsat_mp_gradient(mp.handle, ctx.handle, labels_dev.data_ptr(),
                                       ctypes.byref(loss)), mp)
    return float(loss.value)


def maxsat_mp_adam(mp: Model, ctx: Context, lr: float):
    _check_mp(lib().maxsat_mp_adam(mp.handle, ctx.handle, float(lr)), mp)


def maxsat_mp_destroy(mp: Model):
    if mp is not None and mp.handle:
        lib().maxsat_mp_destroy(mp.handle)
        mp.handle = None


def maxsat_reset_probs(ctx: Context, restarts: int, seed: int, prob):
    prob = np.ascontiguousarray(prob, np.float32)
    assert prob.size == ctx.n
    _check(lib().maxsat_reset_probs(ctx.handle, int(restarts), int(seed) & (2 ** 64 - 1),
                                    _np_ptr(prob)), ctx)
    ctx.B = int(restarts)


def maxsat_propose_flips(ctx: Context, prob, tau: float = 0.1):
    prob = np.ascontiguousarray(prob, np.float32)
    assert prob.size == ctx.n
    _check(lib().maxsat_propose_flips(ctx.handle, _np_ptr(prob), float(tau)), ctx)


def maxsat_get_path(ctx: Context) -> int:
    return int(lib().maxsat_get_path(ctx.handle))


def maxsat_destroy(ctx: Context):
    if ctx is not None and ctx.handle:
        lib().maxsat_destroy(ctx.handle)
        ctx.handle = None


def maxsat_last_error(ctx: Context | None = None) -> str:
    h = None if ctx is None else ctx.handle
    return lib().maxsat_last_error(h).decode()


def maxsat_fit_or_rbm(length, n_hidden, fstar, quant_bits=4, iters=20000):
    W = np.zeros((length, n_hidden), np.float64)
    b = np.zeros(n_hidden, np.float64)
    _check(lib().maxsat_fit_or_rbm(int(length), int(n_hidden), float(fstar), int(quant_bits),
                                   int(iters), _np_ptr(W), _np_ptr(b)))
    return W, b
