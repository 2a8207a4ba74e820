#!/usr/bin/env python3
"""Throughput of the exact FSI hot path on GB300.

Workload: d = 20 players, order l = 3, 16 games per batch (2^20 coalitions
and 1351 scores each); the value vectors come from 16 instances of a
random-init 20-128-128-1 GELU MLP evaluated with absent features set to 0.
One step = tt_fsi_apply on the 16-game batch (Moebius + correction +
assembly of every score).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--arith exact|f64|f32]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

Under torchrun every rank processes its own 16-game batch (weak scaling,
no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact FSI coalitions/s (B·2^d/s, d=20 ℓ=3) and % HBM roofline; student inst/s"
D, ELL, BATCH, HIDDEN = 20, 3, 16, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arith", default="exact", choices=["exact", "f64", "f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=1000, help="student mode: training epochs")
    ap.add_argument("--no-variants", action="store_true",
                    help="headline mode: skip the float64 / float32 variants and the peak measurement")
    ap.add_argument("--no-student", action="store_true", help="headline mode: skip the student fields")
    ap.add_argument("--student-epochs", type=int, default=1000,
                    help="headline mode: epochs of the student run reported beside the headline")
    ap.add_argument("--student-lr", type=float, default=1e-3, help="student: peak learning rate")
    ap.add_argument("--student-schedule", default="cosine", choices=["cosine", "constant"],
                    help="student: learning-rate schedule")
    ap.add_argument("--workload", default="mlp_d20_l3_b16",
                    choices=["mlp_d20_l3_b16", "uneven_1024", "student", "student_step", "configs",
                             "value_function", "peaks"],
                    help="mlp_d20_l3_b16: the headline batch; uneven_1024: 1024 Moebius-sparse "
                         "games with d in 10..20 and l in 1..3, one persistent launch vs "
                         "per-game launches vs a CUDA graph of them; student: the amortised "
                         "explainer; configs: device time of every single-plan configuration "
                         "(each arithmetic, order 4, the other indices), one JSON line; "
                         "value_function: the masked-model value function on each path; "
                         "student_step: the explainer's training step alone (synthetic batch); "
                         "peaks: float64 and integer add / multiply-add throughput of this GPU")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region (NVML through ctypes; reading only)
# ---------------------------------------------------------------------------
REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
           0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
           0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
           0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index: int):
        self.samples, self.reasons = [], 0
        self.max_mhz = None
        self._stop = threading.Event()
        self._nvml = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(h)) != 0:
                raise OSError
            self._nvml, self._h = nv, h
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
        except OSError:
            self._nvml = None

    def _run(self):
        nv, h = self._nvml, self._h
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if nv.nvmlDeviceGetCurrentClocksEventReasons(h, ctypes.byref(rs)) == 0:
                self.reasons |= rs.value & ~0x1
            time.sleep(0.0005)

    def __enter__(self):
        if self._nvml is not None:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *exc):
        if self._nvml is not None:
            self._stop.set()
            self._t.join()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in REASONS.items() if self.reasons & b],
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def shard_workload(rank: int):
    """The d=20 masked-MLP workload of one rank: the same model, instances
    [16 rank, 16 rank + 16) of the seeded instance stream (rank 0 is the
    named 16-game batch), so ranks explain disjoint instances."""
    from paper_2601_01903_gb300 import synthetic
    w = synthetic.workload_mlp_d20()
    if rank:
        w.x = synthetic.gaussian_instances(BATCH, D, 2, first=rank * BATCH)
    return w


def max_over_ranks(value: float, device) -> float:
    """Largest value over all ranks (the job takes as long as its slowest
    rank); the value itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units all ranks processed per second, over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def make_inputs(device, rank: int = 0):
    """16 value vectors of the d=20 masked-MLP workload, float64 on device."""
    import numpy as np
    import torch
    import paper_2601_01903_gb300 as fsi
    w = shard_workload(rank)
    v = torch.empty((BATCH, 1 << D), dtype=torch.float64, device=device)
    fsi.masked_game_into(w.mlp, torch.as_tensor(w.x, device=device),
                         torch.as_tensor(w.baseline, device=device), v)
    torch.cuda.synchronize(device)
    return v, w


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(entry=None):
    """dram bytes per launch of the tile kernel (or of the kernel under
    `entry` in the file) from the committed ncu summary, if the kernel's
    source files still match the ones profiled."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if entry is not None:
            t = t[entry]
        h = hashlib.sha256()
        for src in t["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest()[:16] != t.get("sources_sha256_16"):
        return None
    return t.get("dram_bytes_per_launch")


def committed_record(name, entry=None):
    """A committed ncu figure (profiles/<name>), or None once the kernel's
    source files differ from the ones profiled."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            t = json.load(f)
        if entry is not None:
            t = t[entry]
        h = hashlib.sha256()
        for src in t["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest()[:16] != t.get("sources_sha256_16"):
        return None
    return t


def measure_alu_peaks(dev, reps=3):
    """Throughput of float64 add, float64 multiply-add, 32-bit and 64-bit
    integer add on this GPU (tt_fsi_peak_launch: 8 independent chains per
    thread, 8 CTAs of 256 threads per SM), best of `reps` launches timed with
    CUDA events on the launching stream, with the SM clock sampled."""
    import torch
    import paper_2601_01903_gb300 as fsi
    lib = fsi.native.load()
    props = torch.cuda.get_device_properties(dev)
    blocks = props.multi_processor_count * 8
    out = torch.zeros(blocks * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"sms": props.multi_processor_count, "how": "tt_fsi_peak_launch, 8 independent chains per thread, "
           f"{blocks} CTAs x 256 threads, best of {reps} launches (CUDA events)"}
    with ClockSampler(dev.index or 0) as clocks:
        for kind, name, iters in ((0, "f64_add", 64), (1, "f64_fma", 64), (2, "i32_add", 2048),
                                  (3, "i64_add", 512)):
            ops = ctypes.c_int64()
            best = None
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = lib.tt_fsi_peak_launch(kind, blocks, iters, ctypes.c_void_p(out.data_ptr()),
                                            ctypes.byref(ops), ctypes.c_void_p(stream.cuda_stream))
                if st != 0:
                    raise RuntimeError(f"tt_fsi_peak_launch failed ({st})")
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if r:
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
            res[name + "_per_s"] = ops.value / (best * 1e-3)
    res["clocks"] = clocks.summary()
    return res


def time_plan(plan, copies, phi, steps, stream, warmup=3, nprof=None):
    """Device time per step of plan.apply over the rotating input copies
    (CUDA events on the launching stream), then the tile / combine split of
    the plan's own tracing over nprof further calls."""
    import torch
    import paper_2601_01903_gb300 as fsi
    for i in range(warmup):
        plan.apply(copies[i % len(copies)], out=phi)
    plan.check()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        plan.apply(copies[i % len(copies)], out=phi)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.check()
    lib = fsi.native.load()
    nprof = nprof or min(steps, 100)
    lib.tt_fsi_plan_profile(plan.handle, 1)
    for i in range(nprof):
        plan.apply(copies[i % len(copies)], out=phi)
    lib.tt_fsi_plan_profile(plan.handle, 0)
    t_a, t_b, ncalls = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    lib.tt_fsi_plan_profile_read(plan.handle, ctypes.byref(t_a), ctypes.byref(t_b), ctypes.byref(ncalls))
    plan.check()
    n = max(1, ncalls.value)
    return e0.elapsed_time(e1) / steps, t_a.value / n, t_b.value / n


def cpu_baseline(v_host_games, budget_s=12.0):
    """The oracle as it stands, on this host's cores, over whole games of the
    same workload until about budget_s seconds of work."""
    import oracle
    import numpy as np
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    for g in range(v_host_games.shape[0]):
        oracle.fsi(v_host_games[g], D, ELL)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done * (1 << D) / dt, "unit": "coalitions/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{done} of the {BATCH} d=20 l=3 masked-MLP games, whole games "
                      f"(closed form, explicit superset sums, OpenMP over scores)"}


def cpu_baseline_fast(v_host_games, reps=3):
    """A fair CPU program on this host's cores (oracle/fsi_cpu_fast.c:
    Moebius butterflies and weighted pruned superset sums, float64, OpenMP
    over games) on the whole batch, best of `reps` runs."""
    import oracle
    oracle.build()
    oracle.cpu_fast_fsi(v_host_games[:1], D, ELL)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.cpu_fast_fsi(v_host_games, D, ELL)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return {"value": v_host_games.shape[0] * (1 << D) / best, "unit": "coalitions/s",
            "cores": oracle.num_threads(), "kind": "fast CPU program (not the oracle)",
            "sample": f"the whole {v_host_games.shape[0]}-game batch, best of {reps} runs "
                      "(Moebius butterflies + weighted pruned superset sums, blocked for cache, "
                      "float64, OpenMP over games)"}


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    import numpy as np
    import oracle
    if rank != 0:
        return
    from paper_2601_01903_gb300 import synthetic
    oracle.build()
    w = synthetic.workload_mlp_d20()
    # one whole game per step, its value vector from the oracle's masked game
    v = oracle.masked_game(w.mlp, w.x[0], w.baseline)
    for _ in range(args.warmup):
        oracle.fsi(v, D, ELL)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fsi(v, D, ELL)
    dt = time.perf_counter() - t0
    value = args.steps * (1 << D) / dt
    line = {"metric": METRIC, "value": value, "unit": "coalitions/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "mlp_d20_l3_b16", "d": D, "ell": ELL, "global_batch": BATCH,
                       "reference_step": "one whole game of the batch per step"},
            "cpu_baseline": {"value": value, "unit": "coalitions/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": "one d=20 l=3 masked-MLP game per step"},
            "e2e": {"value": value, "unit": "coalitions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2601_01903_gb300 as fsi

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    v, w = make_inputs(dev, rank)
    n = 1 << D
    # Three copies of the batch rotate so that every step reads its inputs
    # from HBM (3 x 128 MiB is larger than the 126 MiB L2).
    copies = [v] + [v.clone() for _ in range(2)]
    plan = fsi.Plan(D, ELL, args.arith, max_batch=BATCH)
    phi = torch.empty((BATCH, plan.n_scores), dtype=v.dtype, device=dev)
    if args.arith == "f32":
        copies = [c.float() for c in copies]
        phi = phi.float()
    stream = torch.cuda.current_stream(dev)

    def step(i):
        plan.apply(copies[i % len(copies)], out=phi)

    for i in range(args.warmup):
        step(i)
    plan.check()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clocks:
        start.record(stream)
        for i in range(args.steps):
            step(i)
        stop.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(start.elapsed_time(stop), dev)
    plan.check()
    ms_per_step = ms / args.steps
    value = whole_job_rate(BATCH * n, world, ms_per_step)

    # per-kernel device time (the plan's tracing events on the launching
    # stream) of the split schedule the timed steps ran (tile launch, then
    # combine launch), and for comparison the fused persistent schedule
    lib = fsi.native.load()
    nprof = min(args.steps, 100)

    def kernel_ms(fused):
        plan.set_schedule(fused=fused)
        for i in range(3):
            step(i)
        lib.tt_fsi_plan_profile(plan.handle, 1)
        for i in range(nprof):
            step(i)
        lib.tt_fsi_plan_profile(plan.handle, 0)
        t_a, t_b, ncalls = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        lib.tt_fsi_plan_profile_read(plan.handle, ctypes.byref(t_a), ctypes.byref(t_b), ctypes.byref(ncalls))
        return t_a.value / max(1, ncalls.value), t_b.value / max(1, ncalls.value)

    fused_ms, _ = kernel_ms(True)
    tile_ms, comb_ms = kernel_ms(False)
    plan.check()
    elem = 4 if args.arith == "f32" else 8
    # algorithmic traffic of the tile launch, the dominant kernel: one read of v
    alg_bytes = BATCH * n * elem
    peak, peak_kind = peaks()
    achieved = alg_bytes / (tile_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers
    v_host = copies[0].cpu().pin_memory()
    phi_host = torch.empty(phi.shape, dtype=phi.dtype).pin_memory()

    def e2e_rate(zero_copy):
        # zero_copy: the tile kernel reads the page-locked input in place over
        # the host link; otherwise staged chunked copies on the plan's copy stream
        plan.set_host_zero_copy(zero_copy)
        for _ in range(2):
            plan.apply_host(v_host, out=phi_host, stream=stream)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.apply_host(v_host, out=phi_host, stream=stream)
        return world * BATCH * n / ((time.perf_counter() - t0) / args.e2e_steps)

    staged = e2e_rate(False)
    e2e = {"value": e2e_rate(True), "unit": "coalitions/s",
           "h2d_bytes_per_step": BATCH * n * elem, "d2h_bytes_per_step": BATCH * plan.n_scores * elem,
           "route": "tt_fsi_apply_host on page-locked buffers: the tile kernel reads the input in place "
                    "over the host link (zero copy)",
           "staged_copies_value": staged}

    # the other arithmetics on the same inputs: float64 throughout (the
    # literal reading of the exact path, bound by the float64 pipe) and
    # float32 (with its measured error against the exact path, whose own
    # parity with the oracle the tests establish)
    variants, alu = None, None
    if not args.no_variants and args.arith == "exact":
        alu = measure_alu_peaks(dev)
        ref = phi.double().clone()
        vmax = v.abs().amax(dim=1)
        variants = {}
        for arith in ("f64", "f32"):
            vp = fsi.Plan(D, ELL, arith, max_batch=BATCH)
            cps = [c.float() for c in copies] if arith == "f32" else copies
            out = torch.empty((BATCH, vp.n_scores), dtype=cps[0].dtype, device=dev)
            steps = max(5, min(args.steps, 50))
            with ClockSampler(local_rank) as vclocks:
                ms_v, t_tile, t_comb = time_plan(vp, cps, out, steps, stream)
            vp.apply(copies[0].float() if arith == "f32" else copies[0], out=out)
            torch.cuda.synchronize()
            err = ((out.double() - ref).abs().amax(dim=1) / vmax).max().item()
            el = 4 if arith == "f32" else 8
            ach = BATCH * n * el / (t_tile * 1e-3) / 1e9
            entry = {"value": whole_job_rate(BATCH * n, world, ms_v), "unit": "coalitions/s",
                     "ms_per_step": ms_v, "dtype": arith, "steps": steps,
                     "tile_kernel_ms": t_tile, "combine_kernel_ms": t_comb,
                     "max_err_vs_exact_rel_maxv": err,
                     "roofline_hbm": {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                      "peak_kind": peak_kind},
                     "clocks": vclocks.summary()}
            if arith == "f64":
                rec = committed_record("fp64_ops.json")
                if rec is not None:
                    # the float64 pipe's time for this launch's instruction mix
                    # at the measured rates, over the measured kernel time
                    n_add = float(rec["dadd_thread_inst_per_launch"] + rec["dmul_thread_inst_per_launch"])
                    n_fma = float(rec["dfma_thread_inst_per_launch"])
                    ops = n_add + n_fma
                    pk = ops / (n_add / alu["f64_add_per_s"] + n_fma / alu["f64_fma_per_s"])
                    entry["roofline_fp64"] = {
                        "bound": "fp64_alu", "kernel": rec["kernel"], "achieved": ops / (t_tile * 1e-3),
                        "peak": pk, "unit": "float64 instructions/s", "frac": ops / (t_tile * 1e-3) / pk,
                        "peak_kind": "measured live (tt_fsi_peak_launch: add and multiply-add rates, "
                                     "weighted by the kernel's instruction mix)",
                        "fp64_thread_inst_per_launch": ops,
                        "fp64_inst_per_coalition": ops / (BATCH * n),
                        "ops_source": "profiles/fp64_ops.json (ncu, same sources)"}
                else:
                    entry["roofline_fp64"] = None
            variants[arith] = entry
            vp.close()

    student = None
    if not args.no_student and world == 1:
        student = student_run(dev, args.student_epochs, full=False, lr=args.student_lr,
                              schedule=args.student_schedule)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "coalitions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"exact": "int64", "f64": "f64", "f32": "f32"}[args.arith],
        "data": "synthetic",
        "config": {"workload": "mlp_d20_l3_b16", "d": D, "ell": ELL, "global_batch": BATCH * world,
                   "per_gpu_batch": BATCH, "model": "masked-value MLP 20-128-128-1 GELU (random init)",
                   "arith": args.arith, "tile_bits": plan.tile_bits,
                   "l2": "inputs rotate over 3 copies (384 MiB > L2)", "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "kernel": "fsi_tile_fast_kernel", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": kernel_traffic(), "kernel_ms": tile_ms,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "other_kernels_ms": {("fsi_combine_split_kernel" if args.arith == "exact"
                                           else "fsi_combine_fast_kernel"): comb_ms,
                                          "fsi_apply_fast_kernel (fused schedule, outside the timed steps)":
                                              fused_ms}},
        "clocks": clocks.summary(),
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
    }
    if variants is not None:
        line["variants"] = variants
        line["alu_peaks"] = alu
    if student is not None:
        line["student"] = student
    if not args.no_cpu_baseline and world == 1:
        vh = copies[0].cpu().numpy() if args.arith != "f32" else copies[0].double().cpu().numpy()
        line["cpu_baseline"] = cpu_baseline(vh[:4])
        line["cpu_baseline_fast"] = cpu_baseline_fast(vh)
    print(json.dumps(line), flush=True)


def run_configs(args, rank, world, local_rank):
    """Device time per call of tt_fsi_apply for each configuration of the
    build target (inputs resident in HBM, CUDA events on the launching
    stream, 3 rotating input copies where one copy fits in L2)."""
    import numpy as np
    import torch
    import paper_2601_01903_gb300 as fsi
    from paper_2601_01903_gb300 import synthetic

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    gens = {}

    def masked(w):
        v = torch.empty((w.x.shape[0], 1 << w.d), dtype=torch.float64, device=dev)
        fsi.masked_game_into(w.mlp, torch.as_tensor(w.x, device=dev), torch.as_tensor(w.baseline, device=dev), v)
        return v

    def inputs(name):
        if name not in gens:
            if name == "d8":
                w = synthetic.workload_mobius_d8()
                gens[name] = torch.as_tensor(w["v"], device=dev).reshape(1, -1)
            elif name == "d14":
                gens[name] = masked(synthetic.workload_mlp_d14())
            elif name == "d20":
                gens[name] = masked(synthetic.workload_mlp_d20())
            elif name == "d24":
                gens[name] = masked(synthetic.workload_mlp_d24())
            elif name == "n20":
                # white noise at the headline size: the float32 arithmetic's
                # worst case (cancellation in the alternating-sign sums)
                g = torch.Generator(device=dev)
                g.manual_seed(20)
                gens[name] = torch.randn((16, 1 << 20), dtype=torch.float64, device=dev, generator=g)
            elif name == "d28":
                # device time does not depend on the values: seeded noise,
                # one game of 2^28 coalitions (2 GiB)
                g = torch.Generator(device=dev)
                g.manual_seed(28)
                gens[name] = torch.randn((1, 1 << 28), dtype=torch.float64, device=dev, generator=g)
        return gens[name]

    rows = []
    exact_out = {}
    specs = [("cfg1 Moebius game d=8 l=2 B=1", "d8", 8, 2),
             ("cfg2 masked MLP d=14 l=2 B=64", "d14", 14, 2),
             ("cfg3a masked MLP d=20 l=3 B=16", "d20", 20, 3),
             ("cfg3b masked MLP d=24 l=2 B=1", "d24", 24, 2),
             ("order 4, masked MLP d=20 B=16", "d20", 20, 4),
             ("white noise d=20 l=3 B=16", "n20", 20, 3),
             ("large d: noise game d=28 l=3 B=1", "d28", 28, 3)]
    for label, key, d, ell in specs:
        v64 = inputs(key)
        B = v64.shape[0]
        for arith in ("exact", "f64", "f32"):
            for index in (("fsi", "sii", "bii", "stii", "ksii") if key == "d20" and ell == 3 else ("fsi",)):
                if index != "fsi" and arith == "f64":
                    continue
                v = v64.float() if arith == "f32" else v64
                copies = [v] + ([v.clone(), v.clone()] if v.numel() * v.element_size() < (256 << 20) else [])
                plan = fsi.Plan(d, ell, arith, max_batch=B, index=index)
                out = torch.empty((B, plan.n_scores), dtype=v.dtype, device=dev)
                reps = max(5, min(200, int(2e8 // (B << d))))
                for i in range(3):
                    plan.apply(copies[i % len(copies)], out=out)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for i in range(reps):
                    plan.apply(copies[i % len(copies)], out=out)
                e1.record()
                torch.cuda.synchronize()
                plan.check()
                ms = e0.elapsed_time(e1) / reps
                elem = 4 if arith == "f32" else 8
                row = {"config": label, "index": index, "arith": arith, "d": d, "ell": ell, "B": B,
                       "ms_per_call": ms, "coalitions_per_s": B * (1 << d) / (ms * 1e-3),
                       "hbm_frac_of_measured": B * (1 << d) * elem / (ms * 1e-3) / 1e9 / peaks()[0],
                       "calls_timed": reps, "variant": "default"}
                # error against the exact arithmetic on the same input (the
                # exact path's own parity with the oracle is a test), per
                # game as max |difference| / max |v|, the worst game reported
                plan.apply(v, out=out)
                torch.cuda.synchronize()
                if arith == "exact":
                    exact_out[(key, ell, index)] = out.clone()
                else:
                    ref = exact_out[(key, ell, index)]
                    vmax = v64.abs().amax(dim=1)
                    row["max_err_vs_exact_rel_maxv"] = ((out.double() - ref).abs().amax(dim=1) / vmax).max().item()
                rows.append(row)
                plan.close()
    # the comparison variants: the same scores by the site-by-site sweep, and
    # by the sweep of the precontracted operator on v
    for (label, key, d, ell), variant in [(sp, vr) for vr in ("site", "precontract") for sp in specs[2:4]]:
        v64 = inputs(key)
        B = v64.shape[0]
        for arith in ("exact", "f32"):
            v = v64.float() if arith == "f32" else v64
            plan = fsi.Plan(d, ell, arith, max_batch=B, site_sweep=variant == "site",
                            precontract=variant == "precontract")
            out = torch.empty((B, plan.n_scores), dtype=v.dtype, device=dev)
            for i in range(2):
                plan.apply(v, out=out)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(5):
                plan.apply(v, out=out)
            e1.record()
            torch.cuda.synchronize()
            plan.check()
            ms = e0.elapsed_time(e1) / 5
            elem = 4 if arith == "f32" else 8
            rows.append({"config": label, "index": "fsi", "arith": arith, "d": d, "ell": ell, "B": B,
                         "ms_per_call": ms, "coalitions_per_s": B * (1 << d) / (ms * 1e-3),
                         "hbm_frac_of_measured": B * (1 << d) * elem / (ms * 1e-3) / 1e9 / peaks()[0],
                         "calls_timed": 5,
                         "variant": ("site-by-site sweep (Algorithm 1 form)" if variant == "site" else
                                     "precontracted sweep (Section 3.5, no Moebius pass)"),
                         "tile_bits": plan.tile_bits})
            plan.close()
    if rank == 0:
        print(json.dumps({"metric": "device time of tt_fsi_apply per configuration", "unit": "coalitions/s",
                          "n_gpus": 1, "data": "synthetic", "rows": rows}), flush=True)


def run_student_step(args, rank, world, local_rank):
    """The amortised explainer's training step alone: student 16-1024-1024-137,
    batch 4096, synthetic inputs and labels (the step's arithmetic does not
    depend on the values), --steps timed steps after --warmup."""
    import torch
    from paper_2601_01903_gb300 import student as st, synthetic
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    d, H, n_out, B = 16, 1024, 137, 4096
    s = st.Student(d, H, n_out, B, st.init_params(d, H, n_out, 4))
    g = synthetic.Stream(4, 77)
    x = torch.as_tensor(g.normal(B * d).reshape(B, d), dtype=torch.float32, device=dev)
    lab = torch.as_tensor(g.normal(B * n_out).reshape(B, n_out) * 0.01, dtype=torch.float32, device=dev)
    tgt = torch.as_tensor(g.normal(B), dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        s.train_step(x, lab, tgt, 0.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clocks:
        e0.record()
        for _ in range(args.steps):
            s.train_step(x, lab, tgt, 0.0)
        e1.record()
        torch.cuda.synchronize()
    s.check()
    ms = e0.elapsed_time(e1) / args.steps
    flop = 3 * 2 * B * (d * H + H * H + H * n_out)
    mb = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops_sustained": 1700.0}
    peak = float(mb.get("bf16_tflops_sustained", 1700.0))
    if rank == 0:
        print(json.dumps({"metric": "student training step (forward, backward, Adam) on tcgen05", "value": ms,
                          "unit": "ms/step", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
                          "data": "synthetic", "config": {"workload": "student_step", "d": d, "hidden": H,
                                                          "n_out": n_out, "batch": B},
                          "tflops": flop / (ms * 1e-3) / 1e12, "frac_of_sustained_bf16": flop / (ms * 1e-3) / 1e12 / peak,
                          "clocks": clocks.summary()}), flush=True)


def run_value_function(args, rank, world, local_rank):
    """Device time of the value function v_x(S) for every coalition: float64
    and float32 CUDA-core kernels, the tensor-core kernel, and the
    interventional value function with 100 background rows (Section 4.1) on
    the tensor cores.  Models 16-128-128-1 (64 instances) and 20-128-128-1
    (16 instances), random init; the value function is input generation for
    the FSI path and is not part of its timed step."""
    import torch
    import paper_2601_01903_gb300 as fsi
    from paper_2601_01903_gb300 import synthetic
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rows = []
    for d, B in ((16, 64), (20, 16)):
        mlp = fsi.DeviceMLP(synthetic.random_mlp(d, 128, 128, seed=2), dev)
        x = torch.as_tensor(synthetic.gaussian_instances(B, d, seed=2), device=dev)
        base = torch.zeros(d, dtype=torch.float64, device=dev)
        bg = torch.as_tensor(synthetic.gaussian_instances(100, d, seed=7), device=dev)
        o64 = torch.empty((B, 1 << d), dtype=torch.float64, device=dev)
        o32 = torch.empty((B, 1 << d), dtype=torch.float32, device=dev)

        def timed(fn, reps):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        paths = [("float64 CUDA cores (parity path)", lambda: fsi.masked_game_into(mlp, x, base, o64), 1, 1),
                 ("float32 CUDA cores", lambda: fsi.masked_game_into(mlp, x, base, o32), 1, 2),
                 ("tcgen05 BF16 layer 2", lambda: fsi.masked_game_tc(mlp, x, base, out=o32), 1, 5),
                 ("tcgen05, interventional, 100 background rows",
                  lambda: fsi.masked_game_tc(mlp, x, bg, out=o32), 100, 2)]
        for name, fn, n_bg, reps in paths:
            ms = timed(fn, reps)
            rows.append({"d": d, "instances": B, "path": name, "background_rows": n_bg, "ms_per_call": ms,
                         "model_evaluations_per_s": B * (1 << d) * n_bg / (ms * 1e-3),
                         "instances_per_s": B / (ms * 1e-3)})
    if rank == 0:
        print(json.dumps({"metric": "masked-model value function (all 2^d coalitions) per path",
                          "unit": "model evaluations/s", "n_gpus": 1, "data": "synthetic", "rows": rows}),
              flush=True)


def run_uneven(args, rank, world, local_rank):
    """1024 uneven games: the persistent batched launch (autotuned schedule)
    timed against one tt_fsi_apply per game and against a CUDA graph of
    those launches."""
    import torch
    import paper_2601_01903_gb300 as fsi
    from paper_2601_01903_gb300 import synthetic
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    g = synthetic.workload_uneven()
    v = torch.as_tensor(g.v, device=dev)
    phi = torch.zeros(g.n_phi, dtype=torch.float64, device=dev)
    b = fsi.Batch.from_ragged(g, arith=args.arith if args.arith != "f32" else "exact")
    tpi, spi = b.autotune(v, phi)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn(v, phi)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn(v, phi)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local_rank) as clocks:
        ms_p = max_over_ranks(timed(b.apply, args.steps), dev)
    b.check()
    ref_steps = max(3, min(args.steps, 10))
    ms_g = timed(b.apply_per_game, ref_steps)
    ms_c = timed(b.apply_graph, ref_steps)
    b.check()
    coal = float(sum(1 << int(x) for x in g.d))
    peak, peak_kind = peaks()
    achieved = g.v.nbytes / (ms_p * 1e-3) / 1e9
    if rank != 0:
        return
    line = {
        "metric": "batched uneven FSI coalitions/s (one persistent launch)", "value": whole_job_rate(coal, world, ms_p),
        "unit": "coalitions/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_p, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"exact": "int64", "f64": "f64", "f32": "int64"}[args.arith], "data": "synthetic",
        "config": {"workload": "uneven_1024", "games": len(g.d), "d": "U{10..20}", "ell": "U{1,2,3}",
                   "coalitions": coal, "scores": g.n_phi, "tiles_per_item": tpi, "scores_per_item": spi},
        "per_game_launches_ms": ms_g, "cuda_graph_of_per_game_ms": ms_c,
        "speedup_vs_per_game": ms_g / ms_p, "speedup_vs_graph": ms_c / ms_p,
        "roofline": {"bound": "hbm", "kernel": "fsi_batch_kernel", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": kernel_traffic("batch") if args.arith != "f64" else None},
        "clocks": clocks.summary(),
        "gpu_launches": args.steps,
    }
    print(json.dumps(line), flush=True)


def student_run(dev, epochs, full=True, lr=1e-3, schedule="cosine"):
    """Amortised explainer: d=16, l=2 (137 scores), teacher 16-128-128-1,
    x ~ N(0, Sigma) with Sigma_ij = 0.5^|i-j|; 200k training / 10k held-out
    pairs labelled by the exact path; student 16-1024-1024-137, batch 4096,
    cosine learning-rate decay.  Returns training throughput (GEMM
    TFLOP/s), inference instances/s with and without the residual check,
    the exact path's instances/s, and the student's error against exact FSI
    on the held-out set."""
    import numpy as np
    import torch
    from paper_2601_01903_gb300 import student as st, synthetic
    H, BATCH_S, N_TRAIN, N_HELD = 1024, 4096, 200_000, 10_000
    epochs = max(1, epochs)
    ex = st.Explainer(synthetic.workload_student_teacher(), ell=2, hidden=H, batch=BATCH_S)
    t0 = time.perf_counter()
    train = ex.dataset(N_TRAIN, first=0)
    held = ex.dataset(N_HELD, first=N_TRAIN)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    # training (all GEMMs on tcgen05)
    nb = N_TRAIN // BATCH_S
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    with ClockSampler(dev.index or 0) as clocks:
        e0.record(stream)
        losses = ex.train(train, epochs=epochs, lr=lr, schedule=schedule)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_train = e0.elapsed_time(e1)
    steps = epochs * nb
    d, n_out = 16, ex.n_out
    flop_fwd = 2 * BATCH_S * (d * H + H * H + H * n_out)
    flop_step = 3 * flop_fwd  # forward, input gradients, weight gradients
    tflops = flop_step * steps / (ms_train * 1e-3) / 1e12
    # held-out error against exact FSI
    tau = ex.calibrate(held)
    phi = ex.predict_raw(held.x, held.target).double()
    # the accurate reference: exact FSI of FP32 (CUDA-core) value vectors; the
    # training labels came from the tensor-core value function
    lab = ex.exact(held.x.double(), tc=False)
    label_rel_diff = (torch.linalg.norm(held.labels.double() - lab) / torch.linalg.norm(lab)).item()
    rmse = torch.sqrt(((phi - lab) ** 2).mean()).item()
    rel = (torch.linalg.norm(phi - lab) / torch.linalg.norm(lab)).item()
    out, fb = ex.explain(held.x, held.target, first=N_TRAIN)
    rel_fb = (torch.linalg.norm(out - lab) / torch.linalg.norm(lab)).item()
    # baselines the student must beat: the training mean, and least squares on [x, 1]
    mean_rel = (torch.linalg.norm(train.labels.double().mean(0) - lab) / torch.linalg.norm(lab)).item()
    Xtr = torch.cat([train.x.double(), torch.ones(train.x.shape[0], 1, device=dev, dtype=torch.float64)], 1)
    Xh = torch.cat([held.x.double(), torch.ones(held.x.shape[0], 1, device=dev, dtype=torch.float64)], 1)
    coef = torch.linalg.lstsq(Xtr, train.labels.double()).solution
    lin_rel = (torch.linalg.norm(Xh @ coef - lab) / torch.linalg.norm(lab)).item()

    def rate(fn, n, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return n * reps / (a.elapsed_time(b) * 1e-3)

    xb, tb = held.x[:BATCH_S].contiguous(), held.target[:BATCH_S].contiguous()
    ips_student = rate(lambda: ex.student.predict(xb, tb, ex.v_empty), BATCH_S, reps=20)
    ips_checked = rate(lambda: ex.explain(xb, tb, first=N_TRAIN), BATCH_S)
    x64 = held.x[:1024].double()
    ips_exact = rate(lambda: ex.exact(x64), 1024, reps=2)
    res = {
        "student_inst_per_s": ips_checked, "student_only_inst_per_s": ips_student,
        "exact_path_inst_per_s": ips_exact, "speedup_vs_exact": ips_checked / ips_exact,
        "heldout_rel_error": rel, "heldout_rel_error_after_fallback": rel_fb, "heldout_rmse": rmse,
        "baseline_rel_error_mean": mean_rel, "baseline_rel_error_linear": lin_rel,
        "fallback_fraction": fb.float().mean().item(), "epochs": epochs, "train_step_ms": ms_train / steps,
        "train_tflops": tflops, "final_train_loss": losses[-1], "data_generation_s": t_data,
        "threshold": tau, "label_rel_diff_tc_vs_fp32_values": label_rel_diff,
        "config": {"workload": "student_d16_l2", "hidden": H, "batch": BATCH_S, "train": N_TRAIN,
                   "held_out": N_HELD, "residual_samples": ex.K, "lr": lr, "schedule": schedule},
        "clocks": clocks.summary(),
    }
    if full:
        res["exact_path_fp32_values_inst_per_s"] = rate(lambda: ex.exact(x64, tc=False), 1024, reps=2)
        res["value_path"] = "tcgen05 BF16 layer 2" if ex.tc else "FP32 CUDA cores"
        res["steps"] = steps
    return res


def run_student(args, rank, world, local_rank):
    """The amortised explainer on its own line (see student_run)."""
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    r = student_run(dev, args.epochs, full=True, lr=args.student_lr, schedule=args.student_schedule)
    mb = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops_sustained": 1700.0}
    if rank != 0:
        return
    pk = float(mb.get("bf16_tflops_sustained", 1700.0))
    line = {
        "metric": "student inst/s (amortised explainer, d=16 l=2, 137 scores)", "value": r["student_inst_per_s"],
        "unit": "instances/s", "n_gpus": world, "steps": r["epochs"], "warmup": 0,
        "ms_per_step": r["train_step_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic", "config": r["config"],
        "roofline": {"bound": "tensor", "kernel": "gemm_bf16_tcgen05 (training step)", "achieved": r["train_tflops"],
                     "peak": pk, "unit": "TFLOP/s", "frac": r["train_tflops"] / pk, "traffic": None},
        "clocks": r["clocks"], "gpu_launches": r["steps"] * 16,
    }
    line.update({k: v for k, v in r.items() if k not in ("config", "clocks")})
    print(json.dumps(line), flush=True)


def run_peaks(args, rank, world, local_rank):
    """Arithmetic throughput of this GPU: float64 add and multiply-add, 32-
    and 64-bit integer add (the ALU rooflines of the float64 and the exact
    arithmetic)."""
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    r = measure_alu_peaks(dev, reps=max(3, args.steps if args.steps < 50 else 5))
    if rank == 0:
        print(json.dumps({"metric": "arithmetic throughput per GPU", "unit": "operations/s", "n_gpus": 1,
                          "data": "synthetic", **r}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "uneven_1024":
            run_uneven(args, rank, world, local_rank)
        elif args.workload == "student":
            run_student(args, rank, world, local_rank)
        elif args.workload == "configs":
            run_configs(args, rank, world, local_rank)
        elif args.workload == "value_function":
            run_value_function(args, rank, world, local_rank)
        elif args.workload == "student_step":
            run_student_step(args, rank, world, local_rank)
        elif args.workload == "peaks":
            run_peaks(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
