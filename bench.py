#!/usr/bin/env python
"""Throughput benchmark of RbmSAT block Gibbs sampling on GB300.

A step is one full Gibbs round over all chains: score (weighted unsatisfied
cost + free energy), best-keep, hidden draws, scatter-sum of visible logits,
visible draws and the nu update. Metric: clause-assignment evaluations per
second = m * B * steps / seconds, summed over ranks (weak scaling: every rank
runs its own B chains; no data-path collective).

Default workload: weighted Max-3-SAT, n = 1000 variables, m = 6000 clauses,
weights uniform in [1, 1000], B = 4096 chains, seeded synthetic instance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on the
host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "clause·assignment evals/s"
UNIT = "evals/s"
BAD_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="w3sat-n1000-m6000")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--path", default="auto", choices=["auto", "sparse", "dense"])
    ap.add_argument("--no-fp32", action="store_true", help="skip the plain FP32 comparator")
    ap.add_argument("--no-proposal", action="store_true",
                    help="skip the learned-proposal probe (training + held-out comparison)")
    ap.add_argument("--proposal-epochs", type=int, default=4,
                    help="training epochs of the learned proposal")
    ap.add_argument("--proposal-held-out", type=int, default=32,
                    help="held-out formulas of the learned proposal")
    ap.add_argument("--proposal-train", type=int, default=10000,
                    help="solver-labelled training formulas for the proposal probe")
    ap.add_argument("--no-pt", action="store_true", help="skip the parallel-tempering probe")
    ap.add_argument("--no-dense", action="store_true",
                    help="skip the dense-path probes (path comparison, FP8 eval product)")
    ap.add_argument("--no-up", action="store_true",
                    help="skip the unit-propagation ablation probe")
    ap.add_argument("--no-ragged", action="store_true",
                    help="skip the batched ragged-instance probe (512 formulas)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the config 1 and config 3 probes")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the config 3 probe (mixed lengths, n = 20000, m = 100000)")
    ap.add_argument("--fixed-seconds", type=float, default=3.0,
                    help="wall time of the equal-time best-cost comparison")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name, seed):
    spec = workloads.WORKLOADS[name]
    n, off, lits, w = spec["gen"](seed)
    return n, off, lits, w, spec["B"]


# --------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------
def oracle_rate(n, off, lits, w, B, seconds, seed, table=None, n_buckets=4, threads=None):
    """Times the oracle's Gibbs rounds on a sample of chains with every host
    core (or `threads` of them); returns (evals/s, threads, sample
    description, seconds)."""
    import oracle
    inst = oracle.Instance(n, off, lits, w)
    if table is None:
        table = oracle.make_table(sorted(set(np.diff(off)) - {0}), [0.068, 0.528],
                                  n_buckets=n_buckets, iters=2000)
    if threads is None:
        threads = (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                   else os.cpu_count())
    m = len(off) - 1
    # calibrate on one round of `threads` chains, then size the sample
    ids = np.linspace(0, B - 1, threads).astype(np.int32)
    st = oracle.init_chains(n, 0, seed, chain_ids=ids, B_total=B)
    t0 = time.perf_counter()
    oracle.gibbs(inst, table, st, 1, seed, n_temps=2, n_buckets=n_buckets, threads=threads)
    per_round = time.perf_counter() - t0
    rounds = max(1, int(seconds / max(per_round, 1e-6)))
    chains = threads * min(8, max(1, rounds // 4))
    steps = max(1, int(rounds * threads / chains))
    ids = np.linspace(0, B - 1, chains).astype(np.int32)
    st = oracle.init_chains(n, 0, seed, chain_ids=ids, B_total=B)
    t0 = time.perf_counter()
    oracle.gibbs(inst, table, st, steps, seed, n_temps=2, n_buckets=n_buckets, threads=threads)
    dt = time.perf_counter() - t0
    sample = (f"{chains} of {B} chains x {steps} Gibbs rounds of the full formula "
              f"(m = {m}), {dt:.1f} s on {threads} threads")
    return m * chains * steps / dt, threads, sample, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n, off, lits, w, B = workload(args.workload, args.seed)
    m = len(off) - 1
    import oracle
    table = oracle.make_table(sorted(set(np.diff(off)) - {0}), [0.068, 0.528], n_buckets=4,
                              iters=2000)
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    inst = oracle.Instance(n, off, lits, w)
    chains = threads
    ids = np.linspace(0, B - 1, chains).astype(np.int32)
    st = oracle.init_chains(n, 0, args.seed, chain_ids=ids, B_total=B)
    oracle.gibbs(inst, table, st, max(args.warmup, 0), args.seed, n_temps=2, n_buckets=4,
                 threads=threads)
    t0 = time.perf_counter()
    oracle.gibbs(inst, table, st, args.steps, args.seed, n_temps=2, n_buckets=4, threads=threads)
    dt = time.perf_counter() - t0
    value = m * chains * args.steps / dt
    sample = f"{chains} of {B} chains per step (full formula, m = {m})"
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=ws,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * dt / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", config=dict(workload=args.workload, n=n, m=m, B=B),
                cpu_baseline=dict(value=value, unit=UNIT, cores=threads, kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def wait_first(self, timeout=5.0):
        """Blocks until nvidia-smi has written its first sample (or timeout)."""
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < timeout:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                return True
            time.sleep(0.02)
        return False

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].strip() == "Active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0), "fallback"


_FP8_PEAK = None


def fp8_peak(torch, peaks):
    """Dense FP8 (e4m3) tensor peak measured in this run with cuBLAS through
    torch._scaled_mm on 8192^3 (burst: 20 products, sustained: 200), once;
    falls back to 2 x the measured BF16 peaks (the nominal FP8 / BF16 ratio)."""
    global _FP8_PEAK
    if _FP8_PEAK is not None:
        return _FP8_PEAK
    try:
        N = 8192
        a = torch.randn(N, N, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(N, N, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.tensor(1.0, device="cuda")
        run = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(10):
            run()
        out = []
        for reps in (20, 200):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                run()
            e1.record()
            torch.cuda.synchronize()
            out.append(2.0 * N ** 3 / (e0.elapsed_time(e1) / reps / 1e3) / 1e12)
        _FP8_PEAK = (out[0], out[1], "cuBLAS FP8 e4m3 8192^3 measured in this run (burst / sustained)")
    except Exception as e:  # no FP8 GEMM available: nominal ratio
        _FP8_PEAK = (2.0 * peaks["bf16_tflops"], 2.0 * peaks["bf16_tflops_sustained"],
                     f"2 x measured BF16 (FP8 GEMM unavailable: {type(e).__name__})")
    return _FP8_PEAK


def dense_block_work(n, off, lits):
    """Executed dense work of the scatter-add per chain: each 128-variable tile
    spans its own incidence range (incidences sorted by variable), padded to
    64."""
    var = np.abs(lits.astype(np.int64)) - 1
    deg = np.bincount(var, minlength=n)
    vo = np.concatenate([[0], np.cumsum(deg)])
    n_pad = (n + 127) // 128 * 128
    tot = 0
    for tv in range(n_pad // 128):
        k0, k1 = vo[min(tv * 128, n)], vo[min((tv + 1) * 128, n)]
        tot += 128 * max(1, -(-(k1 - k0) // 64)) * 64
    return tot


def alu_peak(clock_mhz, sms):
    """Instruction-issue peak: SMs x 4 sub-partitions x 32 lanes, one
    instruction per sub-partition per clock, at the SM clock seen."""
    return sms * 4 * 32 * clock_mhz * 1e6 / 1e12


def sampling_ops(off):
    """Algorithmic integer operations of the hidden sampling per chain: per
    clause with L hidden units, L/8 Philox4x32-10 calls (10 rounds x (2
    multiplies + 2 three-way XORs) = 40 operations for 8 draws, i.e. 5 per
    draw), one threshold compare per unit, one truth test per literal."""
    lens = np.diff(off)
    L = np.where(lens <= 3, 3, lens + 1)
    L = np.where(lens == 0, 0, L)
    return float((6 * L + lens).sum())


def kernel_roofline(kernel, n, m, nnz, B, off, lits, peaks, clock_mhz, sms, fp8=None):
    """(bound, algorithmic amount per launch, unit, peak) of one kernel.
    Sparse gather: integer operations of the hidden sampling against the
    instruction-issue peak. Sparse visible update: compulsory bytes against
    the copy bandwidth. Dense kernels: tensor-core FLOPs (the dense gather
    product C x states, 2 m n B; the block-diagonal scatter-add, 2 B sum over
    variable tiles of 128 x its incidence range) against the FP8 / BF16 dense
    peak."""
    if kernel in ("gemm1_step", "gemm1_score", "gemm1_eval"):
        return "tensor", 2.0 * m * n * B, "TFLOP/s", (fp8[1] if fp8 else
                                                        2.0 * peaks["bf16_tflops_sustained"])
    if kernel == "gemm2":
        return "tensor", 2.0 * B * dense_block_work(n, off, lits), "TFLOP/s", peaks["bf16_tflops_sustained"]
    if kernel == "gather_hidden":
        return "alu", B * sampling_ops(off), "Tops/s", alu_peak(clock_mhz, sms)
    return "hbm", algorithmic_bytes(kernel, n, m, nnz, B), "GB/s", peaks["hbm_gbs"]


def algorithmic_bytes(kernel, n, m, nnz, B):
    """Compulsory bytes one launch moves (sparse path): the state it must read
    and write once, nothing re-read. Per clause and chain the hidden state is
    one byte (up to 8 hidden units); per variable and chain the state is one
    byte and nu four bytes."""
    formula = 4 * (m + 1) + 4 * nnz + 4 * m + 8 * m
    if kernel == "gather_hidden":
        return n * B + m * B + formula
    if kernel == "visible":
        return m * B + 2 * n * B + 8 * n * B + 8 * nnz
    if kernel == "best_keep":
        return 12 * B
    return None


def run_mine(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_02101_gb300 as ms

    n, off, lits, w, B = workload(args.workload, args.seed)
    m, nnz = len(off) - 1, int(off[-1])
    stream = torch.cuda.Stream()
    path_code = {"auto": ms.MAXSAT_PATH_AUTO, "sparse": ms.MAXSAT_PATH_SPARSE,
                 "dense": ms.MAXSAT_PATH_DENSE}[args.path]
    # launch shapes measured at the first reset (tune_blocks: the gather's
    # clause block, then the visible update's load batch)
    params = ms.maxsat_default_params(path=path_code, tune_blocks=1)
    ctx = ms.maxsat_create(n, off, lits, w, params, stream)
    # every rank runs its own shard of one ensemble of ws * B chains (weak
    # scaling): global chains rank * B .. rank * B + B - 1
    seed = args.seed * 1000003
    offset, total = rank * B, ws * B
    ms.maxsat_reset_shard(ctx, B, seed, offset, total)
    ms.maxsat_step(ctx, args.warmup)
    stream.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # The chains' state (about 50 MB: hidden patterns, nu, x) fits in the L2,
    # so every timed round starts from a flushed L2: a buffer of twice the L2
    # is written on the library's stream before the round, outside the
    # round's CUDA-event interval, and the K intervals are summed.
    l2 = int(getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 0) or (126 << 20))
    flush = torch.empty(2 * l2, dtype=torch.uint8, device="cuda")

    def flushed_rounds(k, events=None):
        with torch.cuda.stream(stream):
            for r in range(k):
                flush.fill_(r & 0xFF)
                if events is not None:
                    events[r][0].record(stream)
                ms.maxsat_step(ctx, 1)
                if events is not None:
                    events[r][1].record(stream)

    flushed_rounds(3)  # warm-up of this launch pattern
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    # SM clocks are sampled every 100 ms over a load window that contains the
    # timed region (which alone is a few ms): a second context of the same
    # formula runs Gibbs rounds for 0.5 s before and 0.3 s after it
    clocks = Clocks(local)
    clocks.wait_first()
    load_ctx = ms.maxsat_create(n, off, lits, w, params, stream)
    ms.maxsat_reset_shard(load_ctx, B, seed + 1, offset, total)

    def load(seconds):
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            ms.maxsat_step(load_ctx, 100)
            stream.synchronize()

    load(0.5)
    barrier()
    torch.cuda.synchronize()
    flushed_rounds(args.steps, evs)
    torch.cuda.synchronize()
    barrier()
    load(0.3)
    ck = clocks.stop()
    if ck is not None:
        ck["window"] = "load window of about 0.8 s containing the timed region"
    ms.maxsat_destroy(load_ctx)
    ms_total = sum(a.elapsed_time(b) for a, b in evs)
    if ws > 1:
        t = torch.tensor([ms_total], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    value = m * B * args.steps * ws / (ms_total / 1e3)

    # the same rounds in steady state: replayed from CUDA graphs, the state
    # carried in L2 from round to round, one interval over all K rounds
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    start.record(stream)
    ms.maxsat_step(ctx, args.steps)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_warm = start.elapsed_time(stop)
    if ws > 1:
        t = torch.tensor([ms_warm], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_warm = float(t.item())
    steady = dict(value=m * B * args.steps * ws / (ms_warm / 1e3), unit=UNIT,
                  ms_per_step=ms_warm / args.steps,
                  note=f"L2 not flushed: state carried round to round, CUDA graphs of "
                       f"{params.steps_per_graph} rounds")

    # per-kernel device times over a third region of the same length, flushed
    # as the timed one (plain launches, CUDA events around every launch on the
    # library's stream)
    ms.maxsat_set_profiling(ctx, True)
    flushed_rounds(args.steps)
    kt = ms.maxsat_kernel_times(ctx)
    ms.maxsat_set_profiling(ctx, False)
    top = max(kt, key=lambda k: kt[k][1])
    launches, tot = kt[top]
    avg_s = tot / launches / 1e3
    peaks, peak_src = measured_peaks()
    clock = (ck or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp8 = fp8_peak(torch, peaks) if "gemm1" in top else None
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    bound, alg, unit, peak = kernel_roofline(top, n, m, nnz, B, off, lits, peaks, clock, sms, fp8)
    scale = 1e9 if unit == "GB/s" else 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f).get(args.workload, {}).get(top)
        if tr and tr.get("source_hash") == kernel_source_hash(top):
            traffic = tr.get("bytes_per_launch")
    roofline = dict(kernel=top, bound=bound, achieved=alg / avg_s / scale, peak=peak, unit=unit,
                    frac=alg / avg_s / scale / peak, traffic=traffic,
                    algorithmic=alg, avg_launch_us=avg_s * 1e6,
                    peak_source=(f"{peak_src} copy bandwidth" if unit == "GB/s" else
                                 f"issue peak {sms} SM x 4 x 32 lanes at {clock:.0f} MHz (SM clock "
                                 "seen in the timed region)" if unit == "Tops/s" else
                                 (fp8[2] + ", sustained") if fp8 else f"{peak_src} BF16 sustained"),
                    kernels={k: dict(launches=v[0], avg_us=1e3 * v[1] / v[0])
                             for k, v in kt.items()})

    # end to end through the public API with host buffers: create from host
    # arrays (pre-fitted parameters, so no fitting), solve, best assignment and
    # cost back to the host
    sets = []
    for s in (ms_fitted_sets(ms, off, params)):
        sets.append(s)
    e2e_steps = args.steps

    def e2e_run(path):
        p2 = ms.maxsat_default_params(sets=sets, path=path)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2 = ms.maxsat_create(n, off, lits, w, p2, stream)
        t1 = time.perf_counter()
        cost, _ = ms.maxsat_solve(ctx2, B, e2e_steps, seed)
        t2 = time.perf_counter()
        ms.maxsat_destroy(ctx2)
        t3 = time.perf_counter()
        return cost, t3 - t0, dict(create_ms=1e3 * (t1 - t0), solve_ms=1e3 * (t2 - t1),
                                    destroy_ms=1e3 * (t3 - t2))

    # the headline: the path the main context's measurement chose (MAXSAT_PATH_AUTO
    # measures once per context and chain count; a caller solving many formulas
    # of one kind passes the choice in), median of 3 solves
    chosen = ms.maxsat_get_path(ctx)
    runs = sorted((e2e_run(chosen) for _ in range(3)), key=lambda r: r[1])
    cost, e2e_s, split = runs[1]
    e2e = dict(value=m * B * e2e_steps * ws / e2e_s, unit=UNIT,
               h2d_bytes_per_step=(off.nbytes + lits.nbytes + w.nbytes) / e2e_steps,
               d2h_bytes_per_step=(n + 8 * B) / e2e_steps, best_cost=int(cost),
               path={1: "dense", 2: "sparse"}[chosen], **split)
    if path_code == ms.MAXSAT_PATH_AUTO:
        # the same solve with the path measured inside it (create builds the
        # dense operands, the first reset times both paths)
        _, e2e_a, split_a = e2e_run(path_code)
        e2e["auto_path"] = dict(split_a, value=m * B * e2e_steps * ws / e2e_a)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:  # one GPU only: the host is shared
        v, threads, sample, _ = oracle_rate(n, off, lits, w, B, args.cpu_seconds, seed)
        cpu = dict(value=v, unit=UNIT, cores=threads, kind="oracle", sample=sample)
        # the same oracle on one host core (a shorter sample)
        v1, _, sample1, _ = oracle_rate(n, off, lits, w, B, max(1.0, args.cpu_seconds / 4), seed,
                                        threads=1)
        cpu["single_thread"] = dict(value=v1, unit=UNIT, cores=1, sample=sample1)

    # the one exchange of the multi-rank path: best cost and assignment
    ms.maxsat_score(ctx)
    stt = ms.maxsat_get_state(ctx)
    lb = int(np.argmin(stt["best_cost"]))
    gbest = (int(stt["best_cost"][lb]), offset + lb)
    if ws > 1:
        from paper_2311_02101_gb300 import distributed as dd
        c_, ch_, _ = dd.reduce_best(gbest[0], gbest[1], stt["best_x"][lb])
        gbest = (c_, ch_)

    dense_eval = (dense_eval_probe(ms, torch, n, off, lits, w, B, stream, sets, args)
                  if not args.no_dense else None)
    paths = (compare_paths(ms, torch, n, off, lits, w, B, stream, sets, seed, args)
             if not args.no_dense else None)
    fp32 = fp32_form_probe(ms, torch, n, off, lits, w, B, stream, sets, seed, args,
                           ms_total / args.steps) if not args.no_fp32 else None
    ragged = ragged_probe(ms, torch, stream, sets, args) if not args.no_ragged else None
    persistent = persistent_probe(
        ms, torch, stream,
        lambda p: ms.maxsat_create(n, off, lits, w, ms.maxsat_default_params(
            sets=sets, path=ms.MAXSAT_PATH_SPARSE, tune_blocks=1, persistent_round=p), stream),
        B, m, args)
    up = up_probe(ms, torch, n, off, lits, w, B, stream, sets, args) if not args.no_up else None
    prop = proposal_probe(ms, torch, stream, sets, args) if not args.no_proposal else None
    pt = pt_probe(ms, torch, n, off, lits, w, B, stream, args) if not args.no_pt else None
    configs = config_probe(ms, torch, stream, args) if not args.no_configs else None

    # the chains' state per round: hidden patterns (2 bytes when some clause
    # has 8 literals or more), x and best x, nu, per-block partials
    Bp = (B + 255) // 256 * 256
    hbytes = 2 if int(np.max(np.diff(off), initial=0)) >= 8 else 1
    state_mb = (m * Bp * hbytes + n * Bp * 6 + 12 * Bp * (m // 100 + 1)) / 2**20
    S = params.steps_per_graph
    per_round = len([k for k in kt if k not in ("gather_score", "keep_copy", "gemm1_score")])
    launches_timed = per_round * args.steps  # one plain-launch round per interval
    path = {1: "dense", 2: "sparse"}[ms.maxsat_get_path(ctx)]
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_total / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="fp8" if path == "dense" else "int32",
                data="synthetic",
                config=dict(workload=args.workload, n=n, m=m, B=B, path=path, path_requested=args.path,
                            steps_per_graph=S, clause_block=ms.maxsat_get_clause_block(ctx),
                            visible_batch=ms.maxsat_get_visible_batch(ctx),
                            parallelism=f"chain-shards{ws}",
                            l2=f"flushed before every timed round ({2 * l2 >> 20} MB buffer written "
                               f"outside the round's event interval; the chains' state, about "
                               f"{state_mb:.0f} MB, {'fits in' if state_mb * 2**20 < l2 else 'exceeds'} "
                               f"the {l2 >> 20} MB L2); steady_state: the same rounds without "
                               "flushes"),
                roofline=roofline, cpu_baseline=cpu, e2e=e2e, clocks=ck, steady_state=steady,
                gpu_launches=launches_timed, dense_eval=dense_eval, paths=paths,
                best=dict(cost=gbest[0], chain=gbest[1], rounds=args.warmup + 3 + 3 * args.steps,
                          chains=ws * B),
                fp32_form=fp32, ragged=ragged, persistent_round=persistent, unit_prop=up,
                proposal=prop, tempering=pt,
                configs=configs)
    line["summary"] = summary_of(line)
    ms.maxsat_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


class Fp32Form:
    """The plain FP32 form of one Gibbs round (the comparator): the same
    clause RBMs and tables, the gather and the scatter-add as FP32 matrix
    products in PyTorch (TF32 off), lookups and Bernoulli draws as tensor
    ops with torch's generator. Uniform clause length only (k-SAT)."""

    def __init__(self, torch, n, off, lits, w, B, sets, fstar=(0.068, 0.528), J=4, Q=4):
        torch.backends.cuda.matmul.allow_tf32 = False
        lens = np.diff(off)
        K = int(lens[0])
        assert (lens == K).all()
        m = len(off) - 1
        E = len(fstar)
        self.t, self.n, self.m, self.B, self.K, self.E = torch, n, m, B, K, E
        dev = "cuda"
        lit = lits.reshape(m, K).astype(np.int64)
        var, lam = np.abs(lit) - 1, np.sign(lit)
        A = np.zeros((m, n), np.float32)
        for k in range(K):
            np.add.at(A, (np.arange(m), var[:, k]), lam[:, k] * float(2 ** k))
        self.A = torch.tensor(A, device=dev)
        Pm = np.zeros((m * K, n), np.float32)  # literal x variable, +-1
        Pm[np.arange(m * K), var.reshape(-1)] = lam.reshape(-1)
        self.P = torch.tensor(Pm, device=dev)
        wmin = int(w.min())
        bucket = np.zeros(m, np.int64)
        for j in range(1, J):
            bucket[w >= wmin * 2 ** j] = j
        self.bucket = torch.tensor(bucket, device=dev)
        self.w = torch.tensor(w, device=dev)
        self.e = torch.tensor(np.minimum(np.arange(B) * E // B, E - 1), device=dev)
        # tables per set s = bucket * E + e: thresholds [s][p][h], free energy
        # [s][p], contributions 2^Q G [s][hp][k], visible thresholds [q]
        L = None
        ph, fe, gq = [], [], []
        for j in range(J):
            for e in range(E):
                st = [x for x in sets if x["len"] == K and x["bucket"] == j and x["temp"] == e][0]
                W, b = np.asarray(st["W"]), np.asarray(st["b"])
                L = W.shape[1]
                V = np.array([[(p >> k) & 1 for k in range(K)] for p in range(2 ** K)], float)
                a = V @ W + b
                ph.append(np.rint(65536.0 / (1.0 + np.exp(-a))))
                fe.append(-np.logaddexp(0, a).sum(1))
                Hp = np.array([[(hp >> h) & 1 for h in range(L)] for hp in range(2 ** L)], float)
                gq.append(np.rint(Hp @ W.T * 2 ** Q))
        self.L, self.Q = L, Q
        self.ph = torch.tensor(np.stack(ph), dtype=torch.float32, device=dev)
        self.fe = torch.tensor(np.stack(fe), dtype=torch.float32, device=dev)
        self.gq = torch.tensor(np.stack(gq), dtype=torch.float32, device=dev)
        qmax = 12 << Q
        qs = np.arange(-qmax, qmax + 1)
        self.qmax = qmax
        self.pv = torch.tensor(np.rint(65536.0 / (1.0 + np.exp(-qs / 2.0 ** Q))), dtype=torch.float32,
                               device=dev)
        self.sidx = self.bucket[None, :] * E + self.e[:, None]  # B x m
        self.gen = torch.Generator(device=dev).manual_seed(0)
        self.x = (torch.rand(B, n, device=dev, generator=self.gen) < 0.5).float()
        self.nu = torch.full((B, n), 0.25, device=dev)
        self.best = torch.full((B,), 2 ** 62, dtype=torch.int64, device=dev)

    def round(self, alpha=0.01):
        t = self.t
        D = (2.0 * self.x - 1.0) @ self.A.T  # B x m: 2 p - (2^K - 1)
        p = ((D + (2 ** self.K - 1)) * 0.5).round().long()
        cost = ((p == 0).long() * self.w[None, :]).sum(1)
        self.best = t.minimum(self.best, cost)
        Fb = self.fe[self.sidx, p].sum(1)
        thr = self.ph[self.sidx, p]  # B x m x L
        h = (t.rand(thr.shape, device="cuda", generator=self.gen) * 65536.0 < thr).long()
        hp = (h << t.arange(self.L, device="cuda")).sum(-1)
        G = self.gq[self.sidx, hp].reshape(self.B, self.m * self.K)  # 2^Q G per literal
        z = G @ self.P  # B x n, units of 2^-Q
        q = z.round().long().clamp(-self.qmax, self.qmax) + self.qmax
        P = self.pv[q]
        rho = P / 65536.0
        self.nu = (1 - alpha) * self.nu + alpha * rho * (1 - rho)
        self.x = (t.rand(P.shape, device="cuda", generator=self.gen) * 65536.0 < P).float()
        return Fb


def fp32_form_probe(ms, torch, n, off, lits, w, B, stream, sets, seed, args, ours_ms_round):
    """Device time per round of the plain FP32 form, and the best exact cost
    each implementation reaches in the same wall time."""
    lens = np.diff(off)
    if not (lens == lens[0]).all():
        return dict(unavailable="plain FP32 form written for uniform clause length")
    f = Fp32Form(torch, n, off, lits, w, B, sets)
    for _ in range(3):
        f.round()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    R = 20
    a.record()
    for _ in range(R):
        f.round()
    b.record()
    b.synchronize()
    ms_round = a.elapsed_time(b) / R
    # equal wall time (seconds of rounds on each side, fresh chains, same seed)
    budget = float(args.fixed_seconds)
    f = Fp32Form(torch, n, off, lits, w, B, sets)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rounds_fp32 = 0
    while time.perf_counter() - t0 < budget:
        for _ in range(10):
            f.round()
        torch.cuda.synchronize()
        rounds_fp32 += 10
    best_fp32 = int(f.best.min())
    ctx = ms.maxsat_create(n, off, lits, w, ms.maxsat_default_params(sets=sets), stream)
    ms.maxsat_reset(ctx, B, seed)
    rounds_ours = 0
    chunk = max(10, int(0.05 / max(ours_ms_round / 1e3, 1e-6)))
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget:
        ms.maxsat_step(ctx, chunk)
        stream.synchronize()
        rounds_ours += chunk
    ms.maxsat_score(ctx)
    best_ours = int(ms.maxsat_get_state(ctx)["best_cost"].min())
    ms.maxsat_destroy(ctx)
    return dict(ms_per_round=ms_round, speedup=ms_round / ours_ms_round,
                fixed_time_s=budget, rounds_fp32=rounds_fp32, rounds_ours=rounds_ours,
                best_cost_fp32=best_fp32, best_cost_ours=best_ours,
                note="FP32 torch matmuls (TF32 off) + lookups, torch generator draws")


def _features(n, off, lits):
    """The network's variable input features without the constant:
    positive-occurrence share minus 1/2 and log(1 + degree) / 4 (0 share for
    a variable without occurrences)."""
    var = np.abs(lits.astype(np.int64)) - 1
    deg = np.bincount(var, minlength=n).astype(np.float64)
    pos = np.bincount(var[lits > 0], minlength=n).astype(np.float64)
    share = np.where(deg > 0, pos / np.maximum(deg, 1.0), 0.5) - 0.5
    return np.stack([share, np.log1p(deg) / 4.0, np.ones(n)], axis=1)


def _logistic_fit(X, y, iters=12):
    """Logistic regression by Newton's method (a features-only baseline)."""
    w = np.zeros(X.shape[1])
    for _ in range(iters):
        p = 1.0 / (1.0 + np.exp(-X @ w))
        g = X.T @ (p - y)
        H = (X * (p * (1 - p))[:, None]).T @ X + 1e-9 * np.eye(X.shape[1])
        w -= np.linalg.solve(H, g)
    return w


def _bce_acc(p, y):
    p = np.clip(p.astype(np.float64), 1e-7, 1 - 1e-7)
    return (float(-np.mean(y * np.log(p) + (1 - y) * np.log(1 - p))),
            float(np.mean((p >= 0.5) == (y == 1))))


def proposal_probe(ms, torch, stream, sets, args):
    """Learned proposal (config 5): a 3-layer, 64-wide message-passing network
    trained by the library's kernels on solver-labelled random weighted
    3-SAT formulas (n uniform in [500, 2000], m = 6 n, weights uniform in
    [1, 1000]; label = best assignment of 256 chains after 500 rounds).
    On held-out formulas (n = 2000, m = 12000, labelled the same way):
    binary cross entropy and per-variable accuracy of the network and of a
    features-only logistic regression on the network's own input features;
    then each held-out formula is solved from uniform starts (plain), from
    the network's starts, from the network's starts with flip proposals
    every 200 rounds, and from the features-only model's starts, the same
    seed and chains, best cost read every 50
    rounds; per formula the fraction of plain's rounds and wall time the
    learned modes need to reach plain's best after 2000 rounds. The share of
    the network's dense layers in its training time comes from CUDA events
    around every training launch of one batch."""
    from paper_2311_02101_gb300 import proposal as P
    rng = np.random.default_rng(args.seed + 17)

    def gen(k, n_lo, n_hi):
        out = []
        for _ in range(k):
            nv = int(rng.integers(n_lo, n_hi + 1))
            out.append(workloads.random_ksat(nv, 6 * nv, 3, int(rng.integers(1 << 30)), 1000))
        return out

    p = ms.maxsat_default_params(sets=sets)
    t0 = time.perf_counter()
    train = gen(args.proposal_train, 500, 2000)
    labels = P.label_with_solver(train, p, restarts=256, steps=500, seed=3, batch=512,
                                 stream=stream)
    t1 = time.perf_counter()
    model = ms.maxsat_mp_create(3, seed=0)
    losses = P.train(model, train, labels, p, epochs=args.proposal_epochs, batch=32, lr=2e-3,
                     stream=stream)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # the training launches of one batch of 32 formulas, each timed by CUDA events
    ctx = ms.maxsat_create_batch(train[:32], p, stream)
    y = torch.tensor(np.concatenate(labels[:32]).astype(np.uint8), device="cuda")
    torch.cuda.synchronize()
    ms.maxsat_set_profiling(ctx, True)
    for _ in range(10):
        ms.maxsat_mp_gradient(model, ctx, y)
        ms.maxsat_mp_adam(model, ctx, 1e-12)
    kt = ms.maxsat_kernel_times(ctx)
    ms.maxsat_set_profiling(ctx, False)
    ms.maxsat_destroy(ctx)
    tot = sum(v[1] for v in kt.values())
    dense_share = sum(v[1] for k, v in kt.items() if k.startswith("mp_dense")) / tot
    # features-only baseline, fitted on (a sample of) the training variables
    Xtr = np.concatenate([_features(f[0], f[1], f[2]) for f in train[:2000]])
    ytr = np.concatenate(labels[:2000]).astype(np.float64)
    wlog = _logistic_fit(Xtr, ytr)
    held = gen(args.proposal_held_out, 2000, 2000)
    held_labels = P.label_with_solver(held, p, restarts=256, steps=500, seed=5, batch=32,
                                      stream=stream)
    cps = list(range(0, 2001, 50))
    modes = ("plain", "learned", "learned+flips", "features")
    mean = {k: np.zeros(len(cps)) for k in modes}
    fr = {k: [] for k in modes[1:]}
    ft = {k: [] for k in modes[1:]}
    net_bce, net_acc, feat_bce, feat_acc = [], [], [], []
    for f, yl in zip(held, held_labels):
        ctx = ms.maxsat_create(*f, p, stream)
        prob = P.propose(model, ctx)
        b, a = _bce_acc(prob, yl)
        net_bce.append(b)
        net_acc.append(a)
        pfeat = (1.0 / (1.0 + np.exp(-_features(f[0], f[1], f[2]) @ wlog))).astype(np.float32)
        b, a = _bce_acc(pfeat, yl)
        feat_bce.append(b)
        feat_acc.append(a)
        curves, times = {}, {}
        for mode in modes:
            torch.cuda.synchronize()
            ts = time.perf_counter()
            if mode == "plain":
                ms.maxsat_reset(ctx, 256, 11)
            elif mode == "features":  # starts from the features-only model
                ms.maxsat_reset_probs(ctx, 256, 11, pfeat)
            else:
                prob = P.propose(model, ctx)
                ms.maxsat_reset_probs(ctx, 256, 11, prob)
            cur, tt, done = [], [], 0
            for T in cps:
                while done < T:  # flip proposals every 200 rounds in the third mode
                    k = min(T, (done // 200 + 1) * 200) - done
                    ms.maxsat_step(ctx, k)
                    done += k
                    if mode == "learned+flips" and done % 200 == 0:
                        ms.maxsat_propose_flips(ctx, prob, 0.2)
                ms.maxsat_score(ctx)  # scores the current state too (keeps the best)
                st = ms.maxsat_get_state(ctx)
                tt.append(time.perf_counter() - ts)
                cur.append(int(st["best_cost"].min()))
            curves[mode], times[mode] = cur, tt
            mean[mode] += np.array(cur, float) / len(held)
        target = curves["plain"][-1]
        for mode in fr:
            k = next((i for i, c in enumerate(curves[mode]) if c <= target), None)
            fr[mode].append(cps[k] / cps[-1] if k is not None else None)
            ft[mode].append(times[mode][k] / times["plain"][-1] if k is not None else None)
        ms.maxsat_destroy(ctx)
    ms.maxsat_mp_destroy(model)

    def med(xs):
        ok = [x for x in xs if x is not None]
        return float(np.median(ok)) if len(ok) == len(xs) else None

    return dict(formulas=len(train), label_rounds=500, label_s=t1 - t0, train_s=t2 - t1,
                epochs=args.proposal_epochs, train_steps=len(losses), loss_first=losses[0],
                loss_last=float(np.mean(losses[-64:])), held_out=len(held),
                held_out_bce=float(np.mean(net_bce)), held_out_accuracy=float(np.mean(net_acc)),
                features_only=dict(weights=wlog.tolist(), bce=float(np.mean(feat_bce)),
                                   accuracy=float(np.mean(feat_acc))),
                dense_layer_share_of_training=dense_share,
                training_kernels_us={k: 1e3 * v[1] / v[0] for k, v in kt.items()},
                checkpoint_every=50,
                mean_best_plain=[int(x) for x in mean["plain"][::4]],
                mean_best_learned=[int(x) for x in mean["learned"][::4]],
                mean_best_learned_flips=[int(x) for x in mean["learned+flips"][::4]],
                rounds_fraction_learned=fr["learned"], wall_fraction_learned=ft["learned"],
                rounds_fraction_flips=fr["learned+flips"], wall_fraction_flips=ft["learned+flips"],
                mean_best_features_start=[int(x) for x in mean["features"][::4]],
                wall_fraction_features_start=ft["features"],
                median_wall_fraction=med(ft["learned"]),
                flips_median_wall_fraction=med(ft["learned+flips"]),
                features_start_median_wall_fraction=med(ft["features"]),
                note="mean_best_* every 200 rounds; a fraction is None when the mode does not "
                     "reach plain's final best by round 2000 (then the median is None); "
                     "checkpoint scoring (maxsat_score + state copy) is inside every wall time")


def pt_probe(ms, torch, n, off, lits, w, B, stream, args, E=8, period=10):
    """Parallel tempering on an ensemble of E = 8 temperatures (F* from 0.35 to
    0.528, geometric: neighbours close enough for the free energies of m =
    6000 clauses to overlap; sets fitted by the library): Gibbs alone vs Gibbs
    with a swap round every `period` rounds (alternating parity), same
    seconds, same seed; lowest best cost over all chains, swap acceptance."""
    secs = args.fixed_seconds
    fstar = list(np.geomspace(0.35, 0.528, E))
    p = ms.maxsat_default_params(fstar=fstar, fit_iters=5000, path=ms.MAXSAT_PATH_SPARSE)
    out = dict(temperatures=E, period=period, seconds=secs, chains=B)
    for mode in ("gibbs", "gibbs+swaps"):
        ctx = ms.maxsat_create(n, off, lits, w, p, stream)
        ms.maxsat_reset(ctx, B, 99)
        rounds, acc, tried = 0, 0, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < secs:
            ms.maxsat_step(ctx, period)
            stream.synchronize()  # the host clock bounds the GPU's work
            rounds += period
            if mode == "gibbs+swaps":
                par = (rounds // period) & 1
                acc += ms.maxsat_pt_swap(ctx, par)
                tried += (E - par) // 2 * (B // E)
        ms.maxsat_score(ctx)
        st = ms.maxsat_get_state(ctx)
        ms.maxsat_destroy(ctx)
        out[mode] = dict(rounds=rounds, best_cost=int(st["best_cost"].min()))
        if tried:
            out[mode]["swap_acceptance"] = acc / tried
    return out


def up_probe(ms, torch, n, off, lits, w, B, stream, sets, args, upp=200, upw=20):
    """The paper's unit-propagation ablation at equal wall time (Sec. 4.4,
    Table "RbmSAT - UP"): Gibbs alone vs Gibbs with a unit-propagation round
    sent every `upp` rounds and merged `upw` rounds later (the host works
    while the GPU samples). Same seed, same seconds; lowest best cost over
    all chains. Propagation and merge on the GPU ("gibbs+up") and on host
    threads as in the paper ("gibbs+up_host"); the wall time of one
    propagation round (begin to end, including the upw rounds between)."""
    secs = args.fixed_seconds
    out = dict(upp=upp, upw=upw, seconds=secs, chains=B)
    for mode in ("gibbs", "gibbs+up", "gibbs+up_host"):
        p = ms.maxsat_default_params(sets=sets, up_device=0 if mode == "gibbs+up_host" else 1)
        ctx = ms.maxsat_create(n, off, lits, w, p, stream)
        ms.maxsat_reset(ctx, B, 99)
        rounds, ups, t_up = 0, 0, 0.0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < secs:
            if mode != "gibbs":
                ms.maxsat_step(ctx, upp - upw)
                stream.synchronize()  # the propagation round alone is timed
                ta = time.perf_counter()
                ms.maxsat_up_begin(ctx)
                ms.maxsat_step(ctx, upw)
                ms.maxsat_up_end(ctx)
                stream.synchronize()
                t_up += time.perf_counter() - ta
                ups += 1
            else:
                ms.maxsat_step(ctx, upp)
                stream.synchronize()  # the host clock bounds the GPU's work
            rounds += upp
        ms.maxsat_score(ctx)
        st = ms.maxsat_get_state(ctx)
        ms.maxsat_destroy(ctx)
        out[mode] = dict(rounds=rounds, best_cost=int(st["best_cost"].min()))
        if ups:
            out[mode]["up_rounds"] = ups
            out[mode]["ms_per_up_round"] = 1e3 * t_up / ups
    return out


def ragged_probe(ms, torch, stream, sets, args):
    """Batched ragged instances: 512 weighted 3-SAT formulas (n log-uniform
    in [100, 5000], m / n uniform in [4, 8]) with 256 restarts each, all in
    every launch of one context (maxsat_create_batch). Device time of K
    graph-replayed rounds with CUDA events on the library's stream, then the
    per-kernel split from a profiled region."""
    spec = workloads.WORKLOADS["ragged-512"]
    insts = spec["gen"](args.seed)
    B = spec["B"]
    m_tot = sum(len(i[1]) - 1 for i in insts)
    p = ms.maxsat_default_params(sets=sets, tune_blocks=1)
    try:
        ctx = ms.maxsat_create_batch(insts, p, stream)
    except ms.MaxsatError as e:
        return dict(unavailable=str(e))
    K = max(20, min(200, args.steps))
    ms.maxsat_reset(ctx, B, 7)
    cb = ms.maxsat_get_clause_block(ctx)
    ms.maxsat_step(ctx, max(3, min(args.warmup, 20)))
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    ms.maxsat_step(ctx, K)
    stop.record(stream)
    torch.cuda.synchronize()
    ms_round = start.elapsed_time(stop) / K
    ms.maxsat_set_profiling(ctx, True)
    ms.maxsat_step(ctx, max(10, K // 4))
    kt = ms.maxsat_kernel_times(ctx)
    ms.maxsat_set_profiling(ctx, False)
    best, _ = ms.maxsat_solve(ctx, B, 50, 7)
    ms.maxsat_destroy(ctx)
    out = dict(workload="ragged-512", instances=len(insts), clauses=m_tot, clause_block=cb,
               variables=int(sum(i[0] for i in insts)), B=B, rounds=K, ms_per_round=ms_round,
               evals_per_s=m_tot * B / (ms_round / 1e3), unit="evals/s",
               kernels_us={k: 1e3 * v[1] / v[0] for k, v in kt.items()},
               launches_per_round=sum(v[0] for k, v in kt.items()) / max(10, K // 4),
               best_cost_sum_50_rounds=int(np.sum(best)))
    # the comparator: the same formulas, one (sparse) context each, the same
    # K rounds from one CUDA graph per context; issued on one stream, then
    # round-robin over 16 streams so that small formulas can run side by side
    streams = [stream] + [torch.cuda.Stream() for _ in range(15)]
    for label, nstreams in (("per_instance", 1), ("per_instance_16_streams", 16)):
        try:
            ctxs = [ms.maxsat_create(*inst, ms.maxsat_default_params(
                        sets=sets, path=ms.MAXSAT_PATH_SPARSE, steps_per_graph=K),
                        streams[k % nstreams])
                    for k, inst in enumerate(insts)]
        except ms.MaxsatError as e:
            out[label] = dict(unavailable=str(e))
            continue
        for c in ctxs:
            ms.maxsat_reset(c, B, 7)
            ms.maxsat_step(c, K)  # captures each context's graph, warms up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in ctxs:
            ms.maxsat_step(c, K)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        for c in ctxs:
            ms.maxsat_destroy(c)
        out[label] = dict(ms_per_round=1e3 * wall / K, evals_per_s=m_tot * B * K / wall,
                          graphs=len(ctxs), streams=nstreams,
                          note="host wall clock around all contexts' graph launches")
    if "ms_per_round" in out.get("per_instance", {}):
        out["per_instance_evals_per_s"] = out["per_instance"]["evals_per_s"]
    # the persistent round on the same batch
    out["persistent_round"] = persistent_probe(
        ms, torch, stream,
        lambda pr: ms.maxsat_create_batch(insts, ms.maxsat_default_params(
            sets=sets, tune_blocks=1, persistent_round=pr), stream),
        B, m_tot, args)
    return out


def persistent_probe(ms, torch, stream, make, B, m_tot, args):
    """The persistent round (one cooperative launch per 100 rounds, grid
    barriers between the gather and the visible update) against the
    two-launch round replayed from CUDA graphs of 100 rounds, on contexts of
    the same formula(s) made by make(persistent_round): K rounds each between
    one pair of CUDA events after warm-up rounds, state carried in L2 from
    round to round in both (as the steady-state rate)."""
    K = 200
    out = {}
    for label, p in (("two_launch", 0), ("persistent", 1)):
        try:
            ctx = make(p)
        except ms.MaxsatError as e:
            return dict(unavailable=str(e))
        try:
            ms.maxsat_reset(ctx, B, 7)
            active = ms.maxsat_get_persistent_round(ctx)
            ms.maxsat_step(ctx, 100)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            ms.maxsat_step(ctx, K)
            b.record(stream)
            torch.cuda.synchronize()
            ms_round = a.elapsed_time(b) / K
            st = ms.maxsat_get_state(ctx)  # reads the device error code of the persistent form
        except ms.MaxsatError as e:
            ms.maxsat_destroy(ctx)
            return dict(unavailable=f"{label}: {e}")
        out[label] = dict(ms_per_round=ms_round, evals_per_s=m_tot * B / (ms_round / 1e3),
                          persistent_active=active, clause_block=ms.maxsat_get_clause_block(ctx),
                          visible_batch=ms.maxsat_get_visible_batch(ctx) if not active else 4,
                          best_cost_sum=int(np.sum(st["best_cost"])))
        ms.maxsat_destroy(ctx)
    out.update(rounds=K, launches_per_100_rounds=dict(two_launch=200, persistent=1),
               persistent_over_two_launch_time=out["persistent"]["ms_per_round"]
               / out["two_launch"]["ms_per_round"])
    return out


def dense_eval_probe(ms, torch, n, off, lits, w, B, stream, sets, args):
    """Exact cost evaluation of B random assignments on the FP8 tensor-core
    gather (maxsat_eval on the dense path: the FP8 conversion of the
    assignments, then the product with its cost epilogue as a programmatic
    dependent launch). `avg_eval_us` is the mean over back-to-back
    evaluations between one pair of CUDA events, and `frac` charges that
    whole time to the product's 2 m n B FLOPs against the FP8 dense peak
    measured in this run (cuBLAS, burst); `eval_us` splits one evaluation
    per kernel from a profiled region (events around every launch)."""
    m = len(off) - 1
    p = ms.maxsat_default_params(sets=sets, path=ms.MAXSAT_PATH_DENSE)
    try:
        ctx = ms.maxsat_create(n, off, lits, w, p, stream)
    except ms.MaxsatError as e:
        return dict(unavailable=str(e))
    g = torch.Generator(device="cuda").manual_seed(1)
    with torch.cuda.stream(stream):
        X = torch.randint(0, 2, (B, n), dtype=torch.uint8, device="cuda", generator=g)
        cost = torch.zeros(B, dtype=torch.int64, device="cuda")
    for _ in range(5):
        ms.maxsat_eval(ctx, X, cost)
    reps = max(20, min(500, args.steps))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    a.record(stream)
    for _ in range(reps):
        ms.maxsat_eval(ctx, X, cost)
    b.record(stream)
    b.synchronize()
    avg = a.elapsed_time(b) / reps / 1e3
    ms.maxsat_set_profiling(ctx, True)
    for _ in range(reps):
        ms.maxsat_eval(ctx, X, cost)
    kt = ms.maxsat_kernel_times(ctx)
    ms.maxsat_set_profiling(ctx, False)
    ms.maxsat_destroy(ctx)
    flops = 2.0 * m * n * B
    peaks, src = measured_peaks()
    burst, _, fsrc = fp8_peak(torch, peaks)
    g_launches, g_tot = kt["gemm1_eval"]
    g_avg = g_tot / g_launches / 1e3
    return dict(kernel="gemm1_eval (tcgen05 kind::f8f6f4) after assign_fp8", avg_eval_us=avg * 1e6,
                evals_per_s=m * B / avg, achieved_tflops=flops / avg / 1e12, peak_tflops=burst,
                frac=flops / avg / 1e12 / burst, bound="tensor", peak_source=fsrc + ", burst",
                flops_per_eval=flops, eval_us={k: 1e3 * v[1] / v[0] for k, v in kt.items()},
                gemm1_eval_frac_events=flops / g_avg / 1e12 / burst)


def compare_paths(ms, torch, n, off, lits, w, B, stream, sets, seed, args):
    """Device time per Gibbs round of both paths on the same workload (CUDA
    graphs, CUDA events), with the per-kernel split from a profiled region."""
    out = {}
    K = max(20, min(200, args.steps))
    for name, code in [("sparse", ms.MAXSAT_PATH_SPARSE), ("dense", ms.MAXSAT_PATH_DENSE)]:
        try:
            ctx = ms.maxsat_create(n, off, lits, w, ms.maxsat_default_params(sets=sets, path=code,
                                                                             steps_per_graph=K),
                                   stream)
        except ms.MaxsatError as e:
            out[name] = dict(unavailable=str(e))
            continue
        ms.maxsat_reset(ctx, B, seed)
        ms.maxsat_step(ctx, K)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ms.maxsat_step(ctx, K)
        b.record(stream)
        b.synchronize()
        ms_round = a.elapsed_time(b) / K
        ms.maxsat_set_profiling(ctx, True)
        ms.maxsat_step(ctx, min(K, 50))
        kt = ms.maxsat_kernel_times(ctx)
        ms.maxsat_set_profiling(ctx, False)
        ms.maxsat_get_state(ctx)  # surfaces a device-side wait timeout, if any
        ms.maxsat_destroy(ctx)
        out[name] = dict(ms_per_round=ms_round, evals_per_s=(len(off) - 1) * B / (ms_round / 1e3),
                         kernels_us={k: 1e3 * v[1] / v[0] for k, v in kt.items()})
    return out


def _rounds_ms(ms, torch, ctx, stream, K):
    """Device ms per Gibbs round over K rounds (CUDA events on the library's
    stream), after the chains ran K rounds once."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ms.maxsat_step(ctx, K)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / K


def config_probe(ms, torch, stream, args):
    """The other configurations on this GPU (they are not the headline):
    config 1, uniform 3-SAT n = 50, m = 215, 256 chains, 200 rounds (launch
    and latency bound): evals/s of the rounds replayed from one CUDA graph and
    of whole create + solve + destroy calls; config 3, mixed lengths 2..12,
    n = 20000, m = 100000, 1024 chains: both paths (device ms per round, per
    kernel) and the path MAXSAT_PATH_AUTO picks."""
    out = {}
    n, off, lits, w, B = workload("3sat-n50-m215", 0)
    m = len(off) - 1
    T = workloads.WORKLOADS["3sat-n50-m215"]["steps"]
    p = ms.maxsat_default_params(n_buckets=1)
    sets = ms_fitted_sets(ms, off, p)
    p = ms.maxsat_default_params(sets=sets, n_buckets=1, steps_per_graph=T)
    ctx = ms.maxsat_create(n, off, lits, w, p, stream)
    ms.maxsat_reset(ctx, B, 0)
    ms.maxsat_step(ctx, T)
    ms_r = _rounds_ms(ms, torch, ctx, stream, T)
    ms.maxsat_destroy(ctx)
    t0 = time.perf_counter()
    for _ in range(5):
        c = ms.maxsat_create(n, off, lits, w, p, stream)
        best, _ = ms.maxsat_solve(c, B, T, 0)
        ms.maxsat_destroy(c)
    solve_s = (time.perf_counter() - t0) / 5
    out["config1"] = dict(workload="3sat-n50-m215", B=B, rounds=T, path="auto",
                          us_per_round=1e3 * ms_r, evals_per_s=m * B / (ms_r / 1e3),
                          solve_ms=1e3 * solve_s, solve_evals_per_s=m * B * T / solve_s,
                          best_cost=int(best))
    if args.no_config3:
        return out
    n, off, lits, w, B = workload("mixed-n20000-m100000", 0)
    m = len(off) - 1
    t0 = time.perf_counter()
    p = ms.maxsat_default_params()
    sets = ms_fitted_sets(ms, off, p)
    c3 = dict(workload="mixed-n20000-m100000", B=B, fit_s=time.perf_counter() - t0)
    for name, code in [("sparse", ms.MAXSAT_PATH_SPARSE), ("dense", ms.MAXSAT_PATH_DENSE)]:
        try:
            t0 = time.perf_counter()
            ctx = ms.maxsat_create(n, off, lits, w, ms.maxsat_default_params(sets=sets, path=code,
                                                                             steps_per_graph=5),
                                   stream)
            create_s = time.perf_counter() - t0
        except ms.MaxsatError as e:
            c3[name] = dict(unavailable=str(e))
            continue
        ms.maxsat_reset(ctx, B, 1)
        ms.maxsat_step(ctx, 5)
        ms_r = _rounds_ms(ms, torch, ctx, stream, 10)
        ms.maxsat_set_profiling(ctx, True)
        ms.maxsat_step(ctx, 3)
        kt = ms.maxsat_kernel_times(ctx)
        ms.maxsat_set_profiling(ctx, False)
        ms.maxsat_get_state(ctx)  # surfaces a device-side wait timeout, if any
        ms.maxsat_destroy(ctx)
        c3[name] = dict(ms_per_round=ms_r, evals_per_s=m * B / (ms_r / 1e3), create_s=create_s,
                        kernels_us={k: 1e3 * v[1] / v[0] for k, v in kt.items()})
        if name == "dense":
            us = c3[name]["kernels_us"].get("gemm1_step")
            if us:
                burst, sust, fsrc = fp8_peak(torch, measured_peaks()[0])
                m_pad, n_pad = (m + 127) // 128 * 128, (n + 127) // 128 * 128
                Bp = (B + 255) // 256 * 256
                c3[name]["gemm1_tflops"] = 2.0 * m_pad * n_pad * Bp / (us / 1e6) / 1e12
                c3[name]["gemm1_frac_fp8"] = c3[name]["gemm1_tflops"] / sust
    t0 = time.perf_counter()
    ctx = ms.maxsat_create(n, off, lits, w, ms.maxsat_default_params(sets=sets), stream)
    ms.maxsat_reset(ctx, B, 1)
    stream.synchronize()
    c3["auto"] = dict(choice={1: "dense", 2: "sparse"}[ms.maxsat_get_path(ctx)],
                      create_and_reset_s=time.perf_counter() - t0)
    ms.maxsat_destroy(ctx)
    out["config3"] = c3
    return out


def summary_of(line):
    """The figures a reader needs first, kept short: the line's end survives a
    truncated log."""
    r, e2e = line["roofline"], line["e2e"]
    out = dict(value=line["value"], roofline=dict(kernel=r["kernel"], frac=round(r["frac"], 3),
                                                    us=round(r["avg_launch_us"], 1)),
               e2e_over_value=round(line["value"] / e2e["value"], 2) if e2e else None)
    st = line.get("steady_state")
    if st:
        out["steady_state"] = st["value"]
    de = line.get("dense_eval")
    if de and "frac" in de:
        out["dense_eval"] = dict(frac_fp8=round(de["frac"], 3), us=round(de["avg_eval_us"], 1),
                                 pflops=round(de["achieved_tflops"] / 1e3, 3),
                                 fp8_peak_pflops=round(de["peak_tflops"] / 1e3, 3),
                                 evals_per_s=de["evals_per_s"])
    pa = line.get("paths")
    if pa:
        out["paths_ms"] = {k: round(v["ms_per_round"], 4) for k, v in pa.items() if "ms_per_round" in v}
    cf = line.get("configs") or {}
    if "config1" in cf:
        out["config1"] = dict(evals_per_s=cf["config1"]["evals_per_s"],
                              solve_evals_per_s=cf["config1"]["solve_evals_per_s"])
    c3 = cf.get("config3")
    if c3:
        out["config3"] = {k: (dict(ms=round(v["ms_per_round"], 3), evals_per_s=v["evals_per_s"],
                                   **({"gemm1_frac_fp8": round(v["gemm1_frac_fp8"], 3)}
                                      if "gemm1_frac_fp8" in v else {}))
                              if isinstance(v, dict) and "ms_per_round" in v else v)
                          for k, v in c3.items() if k in ("sparse", "dense")}
        out["config3"]["auto"] = c3.get("auto", {}).get("choice")
    rg = line.get("ragged")
    if rg and "evals_per_s" in rg:
        out["ragged"] = {k: rg[k] for k in ("evals_per_s", "per_instance_evals_per_s") if k in rg}
    for key, pr in (("persistent", line.get("persistent_round")),
                    ("ragged_persistent", (rg or {}).get("persistent_round"))):
        if pr and "persistent" in pr:
            out[key] = dict(ms=round(pr["persistent"]["ms_per_round"], 4),
                            two_launch_ms=round(pr["two_launch"]["ms_per_round"], 4),
                            active=pr["persistent"]["persistent_active"])
    pr = line.get("proposal")
    if pr:
        out["proposal"] = {k: (round(pr[k], 4) if isinstance(pr[k], float) else pr[k])
                           for k in ("median_wall_fraction", "flips_median_wall_fraction",
                                     "held_out", "formulas", "held_out_bce", "held_out_accuracy",
                                     "dense_layer_share_of_training",
                                     "features_start_median_wall_fraction") if k in pr}
        if "features_only" in pr:
            out["proposal"]["features_only_bce"] = round(pr["features_only"]["bce"], 4)
    return out


KERNEL_SOURCES = {
    "gather_hidden": ["sparse.cu", "philox.cuh", "internal.h"],
    "visible": ["sparse.cu", "philox.cuh", "internal.h"],
    "gemm1_step": ["dense_step.cu", "dense_common.cuh", "tc_ptx.cuh", "philox.cuh", "internal.h"],
    "gemm2": ["dense_step.cu", "dense_common.cuh", "tc_ptx.cuh", "philox.cuh", "internal.h"],
    "gemm1_eval": ["dense.cu", "dense_common.cuh", "tc_ptx.cuh", "internal.h"],
}


def kernel_source_hash(kernel):
    """Hash of the sources a kernel is built from: a recorded DRAM traffic
    figure is used only while it matches."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2311_02101_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, []):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


def ms_fitted_sets(ms, off, params):
    """The library's own fitted sets for this formula's clause lengths and
    weight buckets (host fitting, outside the timed region), with the
    iteration count the library uses at create (beyond 7 literals the fit
    enumerates 2^K inputs per step, so the count is divided by 2^(K - 7), at
    least 2000), fitted on every host core."""
    from concurrent.futures import ThreadPoolExecutor
    lengths = sorted(set(np.diff(off).tolist()) - {0})
    fstar = [0.068, 0.528]
    jobs = [(e, fs, j, K) for e, fs in enumerate(fstar) for j in range(params.n_buckets)
            for K in lengths]

    def fit(job):
        e, fs, j, K = job
        L = 3 if K <= 3 else K + 1
        iters = params.fit_iters
        if K > 7:
            iters = max(min(2000, iters), iters >> (K - 7))
        W, b = ms.maxsat_fit_or_rbm(K, L, fs * (1 + j * params.bucket_gamma),
                                    params.quant_bits, iters)
        return dict(len=K, bucket=j, temp=e, W=W, b=b)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(fit, jobs))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
