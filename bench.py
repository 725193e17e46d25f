"""Benchmark: nested MLMC level estimation with FP16 + Kahan approximate
random variables (piecewise-linear table) on GB300.

Workload (one step): GBM dX = 0.05 X dt + 0.2 X dW, X0 = 1, T = 1, discounted
European call K = 1; levels l = 0..12, N = 2^20 samples per level and
estimator; for every level the two-way approximate difference (FP16 + Kahan,
table) and the four-way nested difference (exact FP32 + Kahan vs FP16 + Kahan
table).  One step = 2 x 2^20 x (2^13 - 1) = 1.718e10 fine Euler path-steps.
Beside it, the plain FP32 exact-normal two-way MLMC over the same levels.

A step is two batched launches (mlmc_batch_async): the 13 two-way items and
the 13 four-way items, each one persistent kernel over all levels in the
tuned tile order, replayed from a captured graph.  value: fine path-steps per
second of that step, timed on the device with CUDA events; e2e: the same
through the synchronous mlmc_batch call with host items and host sums, new
path offsets every step (the descriptors are re-staged).  The same step
through one mlmc_level_async call per level and estimator is reported beside
it.  `--impl reference` times the CPU oracle on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LEVELS = list(range(13))
N_PER_LEVEL = 1 << 20
SEED = 1234
WORKLOAD = "GBM call, levels 0..12, N=2^20 per level, two-way + four-way, FP16+Kahan table vs FP32"

# Algorithmic lane-instructions per fine path-step (one sample of one
# estimator), counted from the method's operations in their minimal form on
# this ISA (a wide 32x32 multiply and a three-input XOR count one each;
# binary16 work per f16x2 operation, i.e. half per sample):
#   Philox (1/5 call x (10 rounds x (2 multiplies + 2 XOR) + 2 byte
#     permutes for the call's fifth uniform); the levels 0..2 of the
#     workload, 0.1 % of its path-steps, take 1/4 call)            8.4
#   uniform and mirror (funnel shift, three adds)                 4
#   table normal (exponent, lookup, v -> f16, mul, add, sign)     4
#   fine Euler + Kahan (8 f16x2 ops per pair)                     4
#   coarse Euler + Kahan (9 per pair per 2 fine steps)            2.25
#   four-way only: exact normal in FP32 (binade lookup, local
#     variable, 7 FMA Horner, centring, sign)                    14
#   four-way only: hat fine + coarse Euler + Kahan in FP32       12.5
OPS_FOURWAY_F16K_TABLE = 49.15
OPS_TWOWAY_F16K_TABLE = 22.65
# DRAM bytes (read + write) of the timed four-way batched launch over levels
# 0..12 at N = 2^20, from an ncu capture of the bench command
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass): the descriptors
# and the tables, 0.07 to 0.74 MB read over the 36 launches captured (the
# tuner's candidates, the replays; ncu starts each from cold caches), 2 KB
# written (the group partials stay in L2).  The traffic does not grow with
# the path-steps.
TRAFFIC_FOURWAY_BYTES = 614656
# Pipe utilisation of the same kernel from the committed ncu capture (the
# small case of the batch-kernel profile: levels 0..12, N = 2^18, full
# section set), of peak over active cycles; the non-tensor pipes bound it.
PIPES_FOURWAY_NCU = {"issue_active": 0.779, "fma_pipe_cycles_active": 0.651, "fmaheavy_cycles_active": 0.608,
                     "alu_pipe_cycles_active": 0.425, "thread_instructions_per_path_step": 55.7,
                     "source": "profiles/batch_kernels_gbm_call_l0-12_N2e20.md"}


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_step_items(M, icdf=None):
    """(four, level, prec, kahan, icdf) of every level in one FP16+Kahan nested step."""
    icdf = M.MLMC_ICDF_TABLE if icdf is None else icdf
    items = []
    for l in LEVELS:
        items.append((0, l, M.MLMC_F16, True, icdf))
        items.append((1, l, M.MLMC_F16, True, icdf))
    return items


def batch_items(M, params, kind, prec, kahan, icdf, offset):
    """The step's items of one estimator (kind 0 two-way, 1 four-way), levels 0..12."""
    return [M.mlmc_work(params, l, kind, prec, int(kahan), icdf, 0, N_PER_LEVEL, offset) for l in LEVELS]


def launches_per_batch_call(items):
    """Kernel launches of one mlmc_batch(_async) replay: one persistent batch
    kernel per group of items sharing estimator, variant and SDE scheme, the
    finalize's span pass when an item has more than 8192 chunk-group partials
    (chunks of 32 sample pairs, chunk_group(l, chunks) of them per partial:
    1 from level 6, else up to 64 >> l keeping at least 16384 groups), and the
    finalize kernel."""
    groups = {(w.kind, w.prec, w.kahan, w.icdf, w.params.sde, w.params.scheme) for w in items}

    def partials(w):
        # lane slots: pairs, or units of 4 / 8 samples at the coarsest two-way levels
        unit = 1 if w.kind else ((4 if w.l == 0 else 2 if w.l == 1 else 1) if w.icdf == 3 else (2 if w.l == 0 else 1))
        chunks = ((w.N + 2 * unit - 1) // (2 * unit) + 31) // 32
        g = 1 if w.l >= 6 else max(1, min(chunks // 16384, 64 >> w.l))
        return (chunks + g - 1) // g
    spans = any(partials(w) > 8192 for w in items)
    return len(groups) + (1 if spans else 0) + 1


def path_steps(levels, n):
    return sum(n * (1 << l) for l in levels)


def run_gpu(args):
    import torch
    import paper_2012_09739_gb300 as M

    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    M.mlmc_icdf_table()                  # first call on the device: state and tables
    init_s = time.perf_counter() - t0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # 256 MiB > 129 MB L2
    # each rank simulates its own disjoint path range (weak scaling)
    offset = rank * N_PER_LEVEL
    F16, T, T16 = M.MLMC_F16, M.MLMC_ICDF_TABLE, M.MLMC_ICDF_TABLE16
    two = batch_items(M, params, 0, F16, True, T, offset)
    four = batch_items(M, params, 1, F16, True, T, offset)
    plain = batch_items(M, params, 0, M.MLMC_F32, False, M.MLMC_ICDF_EXACT, offset)
    two16 = batch_items(M, params, 0, F16, True, T16, offset)
    four16 = batch_items(M, params, 1, F16, True, T16, offset)
    sums = torch.zeros(2 * 2 * len(LEVELS), dtype=torch.float64, device=dev)
    n2 = 2 * len(LEVELS)

    def step(e=None):
        """One step: the two-way and the four-way batched launches."""
        if e:
            e[0].record(stream)
        M.mlmc_batch_async(two, SEED, sums[:n2], stream.cuda_stream)
        if e:
            e[1].record(stream)
        M.mlmc_batch_async(four, SEED, sums[n2:], stream.cuda_stream)
        if e:
            e[2].record(stream)

    # warm-up; the first call of each item-list shape tunes and captures its graph
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        step()
        if not args.no_fp32:
            M.mlmc_batch_async(plain, SEED, sums[:n2], stream.cuda_stream)
        if not args.no_table16:
            M.mlmc_batch_async(two16, SEED, sums[:n2], stream.cuda_stream)
            M.mlmc_batch_async(four16, SEED, sums[n2:], stream.cuda_stream)
    torch.cuda.synchronize()

    # --- device-timed FP16+Kahan nested step
    step_ms, two_ms, four_ms = [], 0.0, 0.0
    with ClockSampler(local) as clocks:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step(e)
            torch.cuda.synchronize()
            two_ms += e[0].elapsed_time(e[1])
            four_ms += e[1].elapsed_time(e[2])
            step_ms.append(e[0].elapsed_time(e[2]))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    ms_total = sum(step_ms)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ps_step = 2 * path_steps(LEVELS, N_PER_LEVEL)
    value = ps_step * args.steps * world / (ms_total / 1e3)

    def timed(calls):
        """Device time (ms) of `calls` per step, summed over the steps, L2 flushed before each."""
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            calls()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total

    # --- plain FP32 exact-normal MLMC over the same levels (comparison)
    fp32_ms = 0.0 if args.no_fp32 else timed(
        lambda: M.mlmc_batch_async(plain, SEED, sums[:n2], stream.cuda_stream))
    fp32_value = path_steps(LEVELS, N_PER_LEVEL) * args.steps * world / (fp32_ms / 1e3) if fp32_ms else None

    # --- the same nested step with 16-bit uniforms for the approximate normals
    t16_kind = [0.0, 0.0]
    for _ in range(0 if args.no_table16 else args.steps):
        flush.fill_(1)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        M.mlmc_batch_async(two16, SEED, sums[:n2], stream.cuda_stream)
        e[1].record(stream)
        M.mlmc_batch_async(four16, SEED, sums[n2:], stream.cuda_stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        t16_kind[0] += e[0].elapsed_time(e[1])
        t16_kind[1] += e[1].elapsed_time(e[2])
    t16_ms = sum(t16_kind)
    t16_value = ps_step * args.steps * world / (t16_ms / 1e3) if t16_ms else None

    # --- the same step through one mlmc_level_async call per level and estimator
    lvl_items = gpu_step_items(M)

    def level_step():
        for i, (k, l, prec, kahan, icdf) in enumerate(lvl_items):
            M.mlmc_level_async(k, l, N_PER_LEVEL, prec, kahan, icdf, params, SEED, offset, sums[2 * i:],
                               stream.cuda_stream)
    lvl_ms = 0.0
    if not args.no_level_calls:
        level_step()                     # untimed warm-up of this leg
        lvl_ms = timed(level_step)
    lvl_value = ps_step * args.steps * world / (lvl_ms / 1e3) if lvl_ms else None

    # --- end to end through the synchronous C-ABI call: host items in, host
    # sums out, new path offsets every step (the descriptors are re-staged)
    e2e_value, h2d = None, 0
    if not args.no_e2e:
        def e2e_items(k):
            off = (k * world + rank + 1) * N_PER_LEVEL
            return (batch_items(M, params, 0, F16, True, T, off) + batch_items(M, params, 1, F16, True, T, off))
        M.mlmc_batch(e2e_items(args.steps + 1), SEED)          # tunes and captures this shape (setup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            M.mlmc_batch(e2e_items(k), SEED, stream.cuda_stream)
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e_value = ps_step * args.steps * world / e2e_s
        h2d = 2 * len(LEVELS) * M.mlmc_batch_descriptor_bytes()

    # --- batching workload: 128 sets x 17 levels x (two-way + four-way), one launch
    batch = None if args.no_batch else batch_leg(M, torch, stream)

    # --- time to RMSE eps through mlmc_run: nested FP16+Kahan vs plain FP32
    mlp = None if args.no_mlp else mlp_leg(M, torch, params)
    tte = None if args.no_tte else time_to_eps(M, params, [args.eps, 3e-4, 1e-5, 3e-6], with_mlp=mlp is not None)

    # --- roofline of the dominant kernel (four-way FP16+Kahan table, all levels in one launch)
    clk = clocks.summary()
    four_ps = path_steps(LEVELS, N_PER_LEVEL) * args.steps
    achieved = OPS_FOURWAY_F16K_TABLE * four_ps / (four_ms / 1e3) / 1e9     # Gop/s (lane-instructions)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clk["sm_mhz"] or 1477.0
    peak = sm_count * 128 * clk_mhz * 1e6 / 1e9                              # Gop/s issue peak

    line = {
        "metric": "EM path-steps/s and time-to-RMSE 1e-3: FP16+Kahan vs plain FP32, one GB300",
        "value": value,
        "unit": "path-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f16",
        "data": "synthetic (Philox4x32-10 seed 1234; counter-based, generated in-kernel)",
        "config": {"workload": WORKLOAD, "levels": [min(LEVELS), max(LEVELS)], "N_per_level": N_PER_LEVEL,
                   "path_steps_per_step": ps_step, "estimators": "two-way FP16+Kahan table + four-way nested",
                   "launch": "one batched persistent launch per estimator over all levels (mlmc_batch_async, "
                             "graph replay)",
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "fp32_plain": {"value": fp32_value, "unit": "path-steps/s", "ms_per_step": fp32_ms / args.steps,
                       "ratio": (value / fp32_value) if fp32_value else None,
                       "path_steps_per_step": path_steps(LEVELS, N_PER_LEVEL)},
        "kernel_ms_per_step": {"fourway_f16_kahan_table": four_ms / args.steps,
                               "twoway_f16_kahan_table": two_ms / args.steps},
        "level_calls": None if not lvl_ms else {
            "value": lvl_value, "unit": "path-steps/s", "ms_per_step": lvl_ms / args.steps,
            "note": "the same step as one mlmc_level_async call per level and estimator (26 launches of "
                    "the level kernels plus finalizes)"},
        "table16": None if not t16_ms else {
            "value": t16_value, "unit": "path-steps/s", "ms_per_step": t16_ms / args.steps,
            "ratio_vs_table": t16_value / value,
            "kernel_ms_per_step": {"fourway_f16_kahan_table16": t16_kind[1] / args.steps,
                                   "twoway_f16_kahan_table16": t16_kind[0] / args.steps},
            "note": "approximate normals from 16-bit uniforms (two per Philox word on two-way paths)"},
        "roofline": {"bound": "alu", "kernel": "batch_kernel<FOUR,F16,kahan,TABLE,GBM> (levels 0..12)",
                     "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                     "traffic": TRAFFIC_FOURWAY_BYTES,
                     "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the timed full-size "
                                      "launch of the bench command; independent of the path-steps",
                     "ops_per_path_step": OPS_FOURWAY_F16K_TABLE,
                     "peak_basis": f"{sm_count} SMs x 128 lanes x {clk_mhz:.0f} MHz (median SM clock sampled)",
                     "launches": args.steps,
                     "pipes_ncu": PIPES_FOURWAY_NCU},
        "e2e": {"value": e2e_value, "unit": "path-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 2 * len(LEVELS) * 16,
                "note": "synchronous mlmc_batch over the 26 items; new path offsets each step"},
        "time_to_eps": tte,
        "batching": batch,
        "mlp": mlp,
        "setup": {"library_init_seconds": init_s,
                  "step_tune_and_capture_seconds": capture_s,
                  "batch_tune_and_capture_seconds": batch["first_call_seconds"] if batch else None,
                  "mlp_train_seconds": mlp["train_seconds"] if mlp else None,
                  "note": "one-time costs, outside every timed region"},
        "gpu_launches": args.steps * (launches_per_batch_call(two) + launches_per_batch_call(four)),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.cpu_seconds)
        line["cpu_baseline"] = cb
        if tte:
            # the oracle's time to the same RMSE, from its path-steps/s on the
            # nested workload and the path-steps each GPU run drew
            line["time_to_eps_cpu_extrapolated"] = {
                e: {k: r[k]["path_steps"] / cb["value"] for k in ("plain_fp32_exact", "nested_f16_kahan_table")
                    if isinstance(r.get(k), dict)}
                for e, r in tte.items()}
            line["time_to_eps_cpu_extrapolated"]["note"] = ("seconds, extrapolated: path-steps of the GPU run / "
                                                            "the oracle's path-steps/s on all host cores")
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def batch_leg(M, torch, stream, repeats=5):
    """The batching workload (64 GBM + 64 OU sets, levels 0..16, uneven N_l,
    FP16 + Kahan table, two-way + four-way) through mlmc_batch (one persistent
    launch replayed from a captured graph), against the same items launched
    one by one through mlmc_level_async."""
    from workloads import batching_sets, batch_level_samples
    sets = batching_sets()
    Ns = batch_level_samples()
    items = []
    for k, s in enumerate(sets):
        if s["kind"] == "gbm":
            p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=s["mu"], p1=s["sigma"], K=s["K"])
        else:
            p = M.sde_params(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=s["theta"], p1=s["m"], p2=s["s"], disc=1.0)
        for l in range(len(Ns)):
            for kind in (0, 1):
                items.append(M.mlmc_work(p, l, kind, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, k, Ns[l], 0))
    ps = sum(it.N * (1 << it.l) for it in items)
    t0 = time.perf_counter()
    M.mlmc_batch(items, SEED)            # tunes, captures the graph
    first_s = time.perf_counter() - t0
    M.mlmc_batch(items, SEED)
    times, devs = [], []
    for _ in range(repeats):
        t0 = time.perf_counter()
        r = M.mlmc_batch(items, SEED)
        times.append(time.perf_counter() - t0)
        devs.append(sum(x.cost_ns for x in r) * 1e-9)
    t_batch = statistics.median(times)
    dev_s = statistics.median(devs)
    sums = torch.zeros(2 * len(items), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    seq = []
    for _ in range(2):
        t0 = time.perf_counter()
        for i, it in enumerate(items):
            M.mlmc_level_async(it.kind, it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED, 0, sums[2 * i:],
                               stream.cuda_stream)
        torch.cuda.synchronize()
        seq.append(time.perf_counter() - t0)
    t_seq = min(seq)
    return {"items": len(items), "path_steps": ps, "seconds": t_batch, "path_steps_per_s": ps / t_batch,
            "first_call_seconds": first_s,
            "device_seconds": dev_s,
            "one_launch_per_item_seconds": t_seq, "speedup_vs_one_launch_per_item": t_seq / t_batch,
            "timing": "wall clock around the synchronous mlmc_batch call (graph replay), median of 5; "
                      "device_seconds from CUDA events around the graph launch of the same 5 calls, median"}


def time_to_eps(M, params, eps_list, repeats=5, with_mlp=False):
    """Wall time of mlmc_run to RMSE eps (Sec. 3 adaptive MLMC): the standard
    estimator (FP32, exact normals, plain Euler) against the nested estimator
    with FP16 + Kahan table normals, FP32 table normals, and the per-level
    automatic choice; the same with 16-bit uniforms for the approximate
    normals, and with the Milstein scheme.  Median of `repeats` runs with
    different seeds, after one untimed run.  Beside the wall time: the cost
    model's device time of the samples drawn (sum of N_t C_t, Sec. 3) and the
    measured device time of the rounds (their difference to the wall time is
    the host's share: planning, launches, waits)."""
    T, T16 = M.MLMC_ICDF_TABLE, M.MLMC_ICDF_TABLE16
    E, MIL = M.MLMC_EULER, M.MLMC_MILSTEIN
    variants = (("plain_fp32_exact", 0, M.MLMC_F32, 0, T, E), ("nested_f16_kahan_table", 1, M.MLMC_F16, 1, T, E),
                ("nested_f32_table", 1, M.MLMC_F32, 0, T, E), ("nested_auto_table", 1, -1, 0, T, E),
                ("nested_f16_kahan_table16", 1, M.MLMC_F16, 1, T16, E), ("nested_auto_table16", 1, -1, 0, T16, E),
                ("plain_fp32_exact_milstein", 0, M.MLMC_F32, 0, T, MIL),
                ("nested_f16_kahan_table16_milstein", 1, M.MLMC_F16, 1, T16, MIL),
                ("nested_auto_table16_milstein", 1, -1, 0, T16, MIL))
    if with_mlp:       # the network trained by the MLP leg
        variants += (("nested_f16_kahan_mlp", 1, M.MLMC_F16, 1, M.MLMC_ICDF_MLP, E),)
    out = {}
    for eps in eps_list:
        row = {}
        for name, est, prec, kahan, icdf, scheme in variants:
            times, model, device, res = [], [], [], None
            p = M.mlmc_sde_params.from_buffer_copy(params)
            p.scheme = scheme
            for rep in range(repeats + 1):
                o = M.mlmc_run_opts(estimator=est, prec=prec, kahan=kahan, icdf=icdf, max_level=18,
                                    min_levels=3, n0=10000, seed=1000 + rep, alpha=1.0, timeout_s=600.0)
                t0 = time.perf_counter()
                r = M.mlmc_run(eps, p, o)
                dt = time.perf_counter() - t0
                if rep > 0:
                    times.append(dt)
                    model.append(r.model_s)
                    device.append(r.device_s)
                    res = r
            row[name] = {"seconds": statistics.median(times), "model_device_seconds": statistics.median(model),
                         "device_seconds": statistics.median(device), "estimate": res.estimate,
                         "rmse_est": math.sqrt(res.variance), "levels": res.levels, "rounds": res.rounds,
                         "path_steps": res.path_steps, "runs": repeats}
            if est == 1 and prec == -1:
                row[name]["prec_per_level"] = ["f16" if res.prec[l] == M.MLMC_F16 else "f32"
                                               for l in range(res.levels)]
                row[name]["kahan_per_level"] = [int(res.kahan[l]) for l in range(res.levels)]
                row[name]["efficiency_per_level"] = [round(res.efficiency[l], 3) for l in range(res.levels)]
        row["speedup_auto_table16_vs_plain"] = (row["plain_fp32_exact"]["seconds"]
                                                / row["nested_auto_table16"]["seconds"])
        row["model_ratio_auto_table16_vs_plain"] = (row["nested_auto_table16"]["model_device_seconds"]
                                                    / row["plain_fp32_exact"]["model_device_seconds"])
        row["speedup_f16_kahan_vs_plain"] = row["plain_fp32_exact"]["seconds"] / row["nested_f16_kahan_table"]["seconds"]
        row["speedup_f16_kahan_table16_vs_plain"] = (row["plain_fp32_exact"]["seconds"]
                                                     / row["nested_f16_kahan_table16"]["seconds"])
        row["speedup_milstein_f16_kahan_table16_vs_plain_milstein"] = (
            row["plain_fp32_exact_milstein"]["seconds"] / row["nested_f16_kahan_table16_milstein"]["seconds"])
        out[f"{eps:g}"] = row
    # the per-level efficiency map (Sec. 3, Fig. 4): every candidate measured on every level
    if 1e-5 in eps_list:
        o = M.mlmc_run_opts(estimator=1, prec=-1, kahan=0, icdf=T16, max_level=18, min_levels=3, n0=10000,
                            seed=999, alpha=1.0, timeout_s=600.0, trial_all=1)
        r = M.mlmc_run(1e-5, params, o)
        out["efficiency_map_1e-05_table16"] = {
            "prec_per_level": ["f16" if r.prec[l] == M.MLMC_F16 else "f32" for l in range(r.levels)],
            "kahan_per_level": [int(r.kahan[l]) for l in range(r.levels)],
            "nested_per_level": [int(r.nested[l]) for l in range(r.levels)],
            "efficiency_per_level": [round(r.efficiency[l], 3) for l in range(r.levels)],
            "note": "trial_all: all candidates measured on every level; efficiency (v c / v^ c^)(1 + sqrt(V C / v c))^2 "
                    "against the standard FP32 exact term (< 1: the nested pair saves at that level)"}
    return out


def mlp_leg(M, torch, params, steps=20000, level=10, n=1 << 20, workload=True):
    """The learned part: train the FP16 tensor-core MLP surrogate on 2^24
    (u, |Phi^-1|) pairs (targets computed on the device in FP64), then its
    E|Z - Z~|^2 against the table's, the four-way throughput with it, and the
    learned-part workload: the nested step (two-way + four-way, FP16+Kahan)
    over levels 0..10 with N = 2^22 per level with the network and with the
    table, beside the plain FP32 exact two-way over the same levels."""
    from workloads import mlp_initial_weights, uniform_grid_sample
    dev = torch.device("cuda")
    M.mlmc_mlp_set_weights(mlp_initial_weights(1234))
    u = torch.tensor(uniform_grid_sample(1 << 24, 31), dtype=torch.float32, device=dev)
    opts = M.mlmc_train_opts(steps=steps, batch=8192, lr0=1e-2, lr_min=1e-5, beta1=0.9, beta2=0.999, eps=1e-8,
                             seed=SEED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = M.mlmc_mlp_train(u, None, opts)
    train_s = time.perf_counter() - t0
    ue = torch.tensor(uniform_grid_sample(1 << 22, 41), dtype=torch.float64, device=dev)
    ref = torch.special.ndtri(ue)
    err = {}
    for name, kind in (("mlp", M.MLMC_ICDF_MLP), ("table", M.MLMC_ICDF_TABLE)):
        z = torch.empty(ue.numel(), dtype=torch.float32, device=dev)
        M.approx_icdf(ue.float(), z, kind, M.MLMC_F32)
        err[name] = float(((z.double() - ref) ** 2).mean())
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream()
    rates = {}
    for name, kind in (("mlp", M.MLMC_ICDF_MLP), ("table", M.MLMC_ICDF_TABLE)):
        M.mlmc_level_async(1, level, n, M.MLMC_F16, 1, kind, params, SEED, 0, sums, s.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(3):
            M.mlmc_level_async(1, level, n, M.MLMC_F16, 1, kind, params, SEED, 0, sums, s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize()
        rates[name] = 3 * n * (1 << level) / (e0.elapsed_time(e1) / 1e3)
    # learned-part workload: levels 0..10, N = 2^22
    n4, levels4 = 1 << 22, (range(0, 11) if workload else range(0))
    steps4 = sum(n4 * (1 << l) for l in levels4)
    legs = {}
    for name, kind, prec, kahan, icdf in (("nested_f16_kahan_mlp", 2, M.MLMC_F16, 1, M.MLMC_ICDF_MLP),
                                          ("nested_f16_kahan_table", 2, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE),
                                          ("plain_fp32_exact", 1, M.MLMC_F32, 0, M.MLMC_ICDF_EXACT)):
        def one():
            for l in levels4:
                M.mlmc_level_async(0, l, n4, prec, kahan, icdf, params, SEED, 0, sums, s.cuda_stream)
                if kind == 2:
                    M.mlmc_level_async(1, l, n4, prec, kahan, icdf, params, SEED, 0, sums, s.cuda_stream)
        one()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        one()
        e1.record(s)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        legs[name] = {"seconds": sec, "path_steps": kind * steps4, "path_steps_per_s": kind * steps4 / sec}
    return {"train_seconds": train_s, "steps": steps, "batch": 8192, "pairs": 1 << 24, "final_loss": loss,
            "l2_error_mlp": err["mlp"], "l2_error_table": err["table"],
            f"fourway_l{level}_path_steps_per_s": {"mlp": rates["mlp"], "table": rates["table"]},
            "levels_0_10_N_2e22": legs}


def _cpu_sample(target_s: float, nthreads: int):
    """Times the oracle on a bounded sample of the same workload: every level,
    the two-way (FP16+Kahan emulated) and four-way (FP64 exact vs FP16+Kahan
    emulated) estimators, with n samples per level scaled to ~target_s."""
    import oracle as O
    from oracle import table
    tab = table.build_table()
    sde = O.gbm(payoff=O.PAYOFF_CALL)
    bar = O.variant(prec=O.F16, kahan=True, rv=O.RV_TABLE)
    hat = O.variant()

    def run(n):
        t0 = time.perf_counter()
        for l in LEVELS:
            O.level_sums(l, n, 0, bar, sde, SEED, O.make_tag(O.KIND_APPROX, l), table=tab, nthreads=nthreads)
            O.level_sums(l, n, 0, hat, sde, SEED, O.make_tag(O.KIND_FOUR, l), table=tab, four=True, var2=bar,
                         nthreads=nthreads)
        return time.perf_counter() - t0

    n = 16 * nthreads
    dt = run(n)
    n2 = max(n, int(n * target_s / max(dt, 1e-3)))
    dt = run(n2)
    ps = 2 * path_steps(LEVELS, n2)
    return ps / dt, n2, dt


def _config1_full(nthreads: int) -> float:
    """Seconds of the oracle on the plain-MLMC workload in full: GBM, P = X_T,
    levels 0..6, 1e5 samples per level, two-way FP64 with exact normals."""
    import oracle as O
    sde = O.gbm(payoff=O.PAYOFF_X)
    t0 = time.perf_counter()
    for l in range(7):
        O.level_sums(l, 100000, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_STD, l), nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_baseline(target_s: float):
    import oracle as O
    threads = os.cpu_count() or 1
    O.build()
    rate, n, dt = _cpu_sample(target_s, threads)
    rate1, n1, dt1 = _cpu_sample(target_s / 4, 1)
    return {"value": rate, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"levels 0..12, {n} samples per level and estimator (two-way + four-way), {dt:.1f} s",
            "single_thread": {"value": rate1, "unit": "path-steps/s", "cores": 1,
                              "sample": f"levels 0..12, {n1} samples per level and estimator, {dt1:.1f} s"},
            "plain_mlmc_full": {"seconds": _config1_full(threads), "path_steps": 100000 * 127, "cores": threads,
                                "workload": "GBM P=X_T, levels 0..6, N=1e5 per level, two-way FP64 exact normals"}}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    rates = []
    for _ in range(args.warmup):
        _cpu_sample(args.cpu_seconds / 4, threads)
    t_total, ps_total, ns = 0.0, 0, []
    for _ in range(args.steps):
        rate, n, dt = _cpu_sample(args.cpu_seconds / 2, threads)
        rates.append(rate)
        ns.append(n)
        t_total += dt
        ps_total += 2 * path_steps(LEVELS, n)
    value = ps_total / t_total
    line = {
        "impl": "reference",
        "metric": "EM path-steps/s and time-to-RMSE 1e-3: FP16+Kahan vs plain FP32, one GB300",
        "value": value, "unit": "path-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16 (emulated in FP64)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "levels": [min(LEVELS), max(LEVELS)], "N_per_level": N_PER_LEVEL,
                   "path_steps_per_step": 2 * path_steps(LEVELS, N_PER_LEVEL),
                   "estimators": "two-way FP16+Kahan table + four-way nested",
                   "sample": f"each step a bounded sample of the workload: {min(ns)}-{max(ns)} samples per level "
                             f"and estimator instead of {N_PER_LEVEL}",
                   "parallelism": f"OpenMP over paths, {threads} host threads"},
        "cpu_baseline": {"value": value, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
                         "sample": f"per step: levels 0..12, {min(ns)}-{max(ns)} samples per level and estimator "
                                   f"(two-way + four-way), ~{args.cpu_seconds / 2:.0f} s"},
        "e2e": {"value": value, "unit": "path-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 comparison leg (profiling runs)")
    ap.add_argument("--no-table16", action="store_true", help="skip the 16-bit-uniform leg (profiling runs)")
    ap.add_argument("--no-level-calls", action="store_true", help="skip the per-level-call leg (profiling runs)")
    ap.add_argument("--no-tte", action="store_true", help="skip the time-to-eps leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batching leg")
    ap.add_argument("--no-mlp", action="store_true", help="skip the MLP leg")
    ap.add_argument("--mlp-only", action="store_true", help="run only the MLP leg (profiling)")
    ap.add_argument("--tte-only", action="store_true", help="run only the time-to-eps leg at --eps (profiling)")
    ap.add_argument("--mlp-steps", type=int, default=20000)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--levels", type=str, default=None, help="comma-separated levels (profiling runs)")
    ap.add_argument("--n", type=int, default=None, help="samples per level (profiling runs)")
    args = ap.parse_args()
    global LEVELS, N_PER_LEVEL
    if args.levels:
        LEVELS = [int(x) for x in args.levels.split(",")]
    if args.n:
        N_PER_LEVEL = args.n
    if args.impl == "reference":
        run_reference(args)
    elif args.mlp_only:
        # profiling mode: the learned part alone (training steps, one four-way MLP level)
        import torch
        import paper_2012_09739_gb300 as M
        params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
        print(json.dumps(mlp_leg(M, torch, params, steps=args.mlp_steps, level=LEVELS[-1], n=N_PER_LEVEL,
                                 workload=args.n is None)))
    elif args.tte_only:
        # profiling mode: the adaptive runs of the time-to-eps leg at one RMSE
        import paper_2012_09739_gb300 as M
        params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
        print(json.dumps(time_to_eps(M, params, [args.eps])))
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
