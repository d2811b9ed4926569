#!/usr/bin/env python
"""Benchmark of the contracted-ERI path on GB300.

Workload: the per-class FP64 sweep -- (pp|pp), (dd|dd), (ff|ff), (gg|gg),
each a batch of random shell quartets with fresh centres uniform in a
10 Angstrom box, exponents log-uniform in [0.05, 500], coefficients uniform
in [0.1, 1] and the contraction depth of every shell drawn from {1, 3, 6};
spherical output in FP64.  One step evaluates every quartet of every class
once (one eri_compute per class plan).

Prints one JSON line (rank 0).  value = quartets/s of the whole step with
inputs resident on the device; e2e = the same through the public API with
host buffers (plan upload, compute, copy of the results to pinned host
memory every step).  --impl reference times the CPU oracle instead.
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

import numpy as np  # noqa: E402

from paper_2605_10312_gb300 import synth  # noqa: E402

METRIC = "contracted ERI shell-quartets/s (per-class FP64 sweep)"
UNIT = "quartets/s"
# (class, quartets per step): 10^6 (pp|pp) and (dd|dd), 10^5 (ff|ff) and (gg|gg)
SWEEP = [((1, 1, 1, 1), 1_000_000), ((2, 2, 2, 2), 1_000_000), ((3, 3, 3, 3), 100_000), ((4, 4, 4, 4), 100_000)]
# batch latency: quartets per batch and repeats per class
LATENCY = {(1, 1, 1, 1): 10_000, (2, 2, 2, 2): 10_000, (3, 3, 3, 3): 10_000, (4, 4, 4, 4): 1_000}
LATENCY_REPEATS = 100
KSET = (1, 3, 6)
SEED = 2000
ONLY = None     # --classes: subset of the sweep (profiling runs)
E2E_CHUNK = 250_000  # quartets per plan in the end-to-end leg (planned in parallel)
SCALE = 1.0     # --scale: quartet counts multiplied by this (profiling runs)
# FP64 fused multiply-add lanes per SM per clock, measured on GB300 with the
# fp_peak microbenchmark (independent FMA chains on every SM)
FP64_LANES_PER_SM_CLK = 1.683
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def fp64_peak_tflops(mhz=SM_MAX_MHZ):
    return FP64_LANES_PER_SM_CLK * 2 * SM_COUNT * mhz * 1e6 / 1e12


def workload(rank=0):
    parts = []
    for ls, n in SWEEP:
        if ONLY and "".join("spdfg"[x] for x in ls) not in ONLY:
            continue
        n = max(1, int(n * SCALE))
        basis, q = synth.class_sweep(ls, n, kset=KSET, seed=SEED + 10 * ls[0] + 1000 * rank)
        parts.append((ls, basis, q))
    return parts


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (also the --impl reference arm)
# ---------------------------------------------------------------------------
def oracle_rates(parts, budget_s=15.0, nthreads=None, sizes=None):
    """Oracle quartets/s per class on a bounded sample of each class's
    quartets (a prefix: same geometry and contraction mix), all host cores.

    The oracle's thread pool hands out one quartet per task, so a batch ends
    with threads idle while the slowest quartets finish; a rate taken from
    batches of a few quartets per thread understates the oracle.  Each class
    therefore gets a short calibration (batches growing from 16 quartets, a
    fifth of its budget) and then one batch sized to fill the rest of its
    budget with at least eight quartets per thread; the rate is that batch's.
    ``sizes`` (the second return value of an earlier call) skips the
    calibration.  Returns (rates, sizes, threads)."""
    import oracle
    oracle.build()
    nthreads = nthreads or os.cpu_count() or 1
    rates, out_sizes = {}, {}
    per_class = budget_s / len(parts)
    for ls, basis, q in parts:
        if sizes is None:
            n, done, t_used = 16, 0, 0.0
            while t_used < 0.2 * per_class and done < q.shape[0]:
                sel = q[done:done + n]
                t0 = time.perf_counter()
                oracle.eri(basis, sel, nthreads=nthreads)
                t_used += time.perf_counter() - t0
                done += sel.shape[0]
                n *= 2
            size = int(max(8 * nthreads, done / t_used * 0.8 * per_class))
        else:
            size = sizes[ls]
        sel = q[:min(size, q.shape[0])]
        t0 = time.perf_counter()
        oracle.eri(basis, sel, nthreads=nthreads)
        rates[ls] = sel.shape[0] / (time.perf_counter() - t0)
        out_sizes[ls] = sel.shape[0]
    return rates, out_sizes, nthreads


def tuned_summary(tuned):
    """The autotuner's choices per class: tier, and per kind of contraction
    the cooperative shape (T x nodes per lane, steps per wave of each phase)
    and vote form."""
    if tuned is None:
        return None
    out = {}
    for c, v in tuned.items():
        e = {"tier": v["tier"]}
        for kind, sh in (v.get("shapes") or {}).items():
            e[kind] = "T{}x{} w{}/{} votes {}".format(sh["T"], sh["ilp"], sh["k1"], sh["k2"], sh["votes"])
        out["".join(map(str, c))] = e
    return out


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, else the Arm
    implementer and part codes), else the machine type."""
    import platform
    info = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    if "model name" in info:
        return info["model name"]
    if "cpu part" in info:
        return "{} (CPU implementer {}, part {})".format(platform.machine(), info.get("cpu implementer", "?"),
                                                       info["cpu part"])
    return platform.machine()


def single_core_baseline(parts, budget_s=4.0):
    """The oracle on one host core: per-class rates on a bounded sample and
    the rate of the step's class mix."""
    r, samples, _ = oracle_rates(parts, budget_s=budget_s, nthreads=1)
    return {"value": mix_rate(r), "unit": UNIT, "cores": 1,
            "per_class": {"".join("spdfg"[x] for x in ls): r[ls] for ls in r},
            "sample": "prefix of each class's quartets: " + ", ".join(
                "{} {}".format("".join("spdfg"[x] for x in ls), samples[ls]) for ls in samples) +
            " ({:.0f} s of CPU work)".format(budget_s)}


def sweep():
    return [(ls, max(1, int(n * SCALE))) for ls, n in SWEEP
            if not ONLY or "".join("spdfg"[x] for x in ls) in ONLY]


def mix_rate(rates):
    """Quartets/s of the whole step's class mix given per-class rates."""
    tot = sum(n for _, n in sweep())
    t = sum(n / rates[ls] for ls, n in sweep())
    return tot / t


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    parts = workload()
    times = []
    # one calibration sizes each class's sample for about 6 s of CPU work per
    # step (the same measurement as the cpu_baseline leg, on a smaller
    # budget); every step then evaluates those samples
    per_step = 6.0
    _, sizes, _ = oracle_rates(parts, budget_s=per_step)
    rates = None
    for s in range(args.warmup + args.steps):
        r, samples, cores = oracle_rates(parts, budget_s=per_step, sizes=sizes)
        if s >= args.warmup:
            times.append(mix_rate(r))
            rates = (r, samples, cores)
    value = statistics.median(times)
    r, samples, cores = rates
    tot = sum(n for _, n in sweep())
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(),
        "per_class": {"".join("spdfg"[x] for x in ls): {"quartets_per_s": r[ls], "sample": samples[ls]}
                      for ls in r},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step, a prefix of each class's quartets: " + ", ".join(
                             "{} {}".format("".join("spdfg"[x] for x in ls), samples[ls]) for ls in samples) +
                         " (about {:.0f} s of CPU work, sized by one calibration run)".format(per_step),
                         "cpu_model": cpu_model(), "single_core": single_core_baseline(parts)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_dict():
    return {"workload": "per-class FP64 sweep: " + ", ".join(
        "({0}{0}|{0}{0}) x {1}".format("spdfg"[ls[0]], n) for ls, n in sweep()),
        "K_per_shell": list(KSET), "box_angstrom": 10.0, "exponents": [0.05, 500.0], "output": "spherical",
        "quartets_per_step": sum(n for _, n in sweep()), "l2": "flushed between steps (512 MiB write)"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_2605_10312_gb300 import eri, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.distributed.is_nccl_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    parts = workload(rank)
    tuned = None
    if args.autotune:
        # tier, cooperative shape and vote form per class and kind of
        # contraction, timed on a sample of each class's quartets
        from paper_2605_10312_gb300 import tune
        tuned = {}
        for ls, basis, q in parts:
            tuned.update(tune.autotune(basis, q, sample=args.tune_sample, shapes=True))
    plans, outs = [], []
    for ls, basis, q in parts:
        p = eri.Plan(basis, q, votes=args.votes, persistent=args.persistent)
        p.set_timing(True)
        plans.append((ls, p))
        outs.append(torch.empty(p.output_count, dtype=torch.float64, device=dev))
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        for (ls, p), o in zip(plans, outs):
            p.compute(o, stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ms, launch_ms = [], {}
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush, outside the timed region
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for ls, p in plans:
            for i, rec in enumerate(p.launches()):
                key = (ls, i)
                launch_ms.setdefault(key, []).append((rec, rec["ms"]))
    clk = clocks.stop()
    total_ms = shard.max_over_ranks(sum(step_ms), dev)
    quartets = shard.sum_over_ranks(sum(p.nq for _, p in plans), dev)
    value = quartets * args.steps / (total_ms * 1e-3)

    # dominant kernel: the launch with the largest time share
    dom_key = max(launch_ms, key=lambda k: sum(ms for _, ms in launch_ms[k]))
    recs = launch_ms[dom_key]
    dom_rec = recs[0][0]
    dom_ms = statistics.mean(ms for _, ms in recs)
    achieved = dom_rec["flops"] / (dom_ms * 1e-3) / 1e12
    peak = fp64_peak_tflops()
    per_class = {}
    for ls, p in plans:
        ms = [statistics.mean(m for _, m in launch_ms[(ls, i)]) for i in range(len(p.launches()))]
        fl = sum(r["flops"] for r in p.launches())
        n = p.nq
        per_class["".join("spdfg"[x] for x in ls)] = {
            "quartets": n, "ms": sum(ms), "quartets_per_s": n / (sum(ms) * 1e-3),
            "fp64_tflops": fl / (sum(ms) * 1e-3) / 1e12, "fp64_frac_of_peak": fl / (sum(ms) * 1e-3) / 1e12 / peak,
            "tier": [eri.TIERS_INV.get(r["tier"], r["tier"]) for r in p.launches()[1:]]}
    nlaunch = sum(len(p.launches()) for _, p in plans)
    measured = _traffic_for(dom_rec)
    traffic, executed = measured if measured else (None, None)

    # end to end through the public API with host buffers
    e2e_ms, h2d, d2h = [], 0, 0
    e2e_warmup = 1
    if args.no_e2e:
        args_e2e_steps = 0
    else:
        args_e2e_steps = e2e_warmup + args.steps
    host_outs = [torch.empty(p.output_count, dtype=torch.float64).pin_memory() for _, p in plans]
    # A plan is built on one host thread (about 1.7 us per quartet when every
    # quartet brings new shell pairs), so a class's list is planned in
    # contiguous chunks of about E2E_CHUNK quartets on several threads; the
    # chunks' blocks, in order, are the class's blocks.
    chunks = []
    for k, (ls, basis, q) in enumerate(parts):
        nch = max(1, int(round(q.shape[0] / E2E_CHUNK)))
        edges = np.linspace(0, q.shape[0], nch + 1).astype(np.int64)
        for c in range(nch):
            chunks.append((k, basis, q[edges[c]:edges[c + 1]]))
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max_workers=max(1, min(len(chunks), (os.cpu_count() or 2) - 1)))
    e2e_streams = [stream, torch.cuda.Stream()]
    for it in range(args_e2e_steps):
        barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        # the plans are independent: build them concurrently (the native
        # planner releases the interpreter lock), then evaluate each and copy
        # its blocks to its stretch of the class's pinned host buffer
        built = list(pool.map(lambda ch: eri.Plan(ch[1], ch[2]), chunks))
        at = [0] * len(parts)
        for i, ((k, _, _), p) in enumerate(zip(chunks, built)):
            n = p.output_count
            # two streams in turn: a plan's copy to the host overlaps the
            # next plan's evaluation
            p.compute_host(host_outs[k][at[k]:at[k] + n], e2e_streams[i % 2])
            at[k] += n
            h2d += p.stats()["h2d_bytes"]
            d2h += n * 8
        for st in e2e_streams:
            st.synchronize()
        for p in built:
            p.close()
        barrier()
        if it >= e2e_warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    pool.shutdown()
    e2e_total = shard.max_over_ranks(sum(e2e_ms) if e2e_ms else float("nan"), dev)
    e2e_value = quartets * args.steps / (e2e_total * 1e-3)

    latency = None if args.no_latency else batch_latency(plans, parts, flush, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rates, samples, cores = oracle_rates(parts, budget_s=args.cpu_seconds)
        cpu = {"value": mix_rate(rates), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "prefix of each class's quartets: " + ", ".join(
                   "{} {}".format("".join("spdfg"[x] for x in ls), samples[ls]) for ls in samples) +
               " ({:.0f} s of CPU work)".format(args.cpu_seconds),
               "per_class": {"".join("spdfg"[x] for x in ls): rates[ls] for ls in rates},
               "cpu_model": cpu_model(), "single_core": single_core_baseline(parts)}
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(),
        "per_class": per_class,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     # executed FP64 flops (ncu) over the algorithmic count on
                     # the dominant launch type; null when its counters are stale
                     "fp64_executed_over_algorithmic": executed,
                     "kernel": "{} tier {} ({} quartets)".format(
                         "".join("spdfg"[x] for x in dom_rec["cls"]) if dom_rec["cls"][0] >= 0 else "pair set-up",
                         eri.TIERS_INV.get(dom_rec["tier"], dom_rec["tier"]), dom_rec["quartets"]),
                     "peak_basis": "FP64 FMA issue rate measured by fp_peak ({} lanes/SM/clk) x 2 x 152 SMs x "
                                   "2070 MHz".format(FP64_LANES_PER_SM_CLK)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "plans_per_step": len(chunks), "plan_threads": pool._max_workers},
        "latency": latency,
        "gpu_launches": nlaunch * args.steps,
        "clocks": clk,
        "autotuned": tuned_summary(tuned),
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def batch_latency(plans, parts, flush, stream):
    """p50/p99 device latency of one batch per class (the first LATENCY[class]
    quartets of the sweep), LATENCY_REPEATS repeats after 3 warm-ups, L2
    flushed before each, CUDA events on the launching stream."""
    import torch
    from paper_2605_10312_gb300 import eri
    out = {}
    for (ls, basis, q) in parts:
        n = min(LATENCY.get(ls, 10_000), q.shape[0])
        p = eri.Plan(basis, q[:n])
        o = torch.empty(p.output_count, dtype=torch.float64, device=flush.device)
        ms = []
        for it in range(3 + LATENCY_REPEATS):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.compute(o, stream)
            e1.record(stream)
            e1.synchronize()
            if it >= 3:
                ms.append(e0.elapsed_time(e1))
        p.close()
        out["".join("spdfg"[x] for x in ls)] = {
            "batch_quartets": n, "repeats": LATENCY_REPEATS, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "mean_ms": float(np.mean(ms))}
    return out


def _traffic_for(rec):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    summary, when it was taken on the current kernel source; else null."""
    path = os.path.join(ROOT, "profiles", "dominant_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    import hashlib
    from paper_2605_10312_gb300 import eri
    key = "".join("spdfg"[x] for x in rec["cls"]) if rec["cls"][0] >= 0 else "setup"
    ent = d.get(key)
    if not ent or ent.get("tier") != eri.TIERS_INV.get(rec["tier"]):
        return None
    h = hashlib.sha256()
    for f in ent.get("source_files", []):
        # paths relative to the package (bare names: its csrc folder)
        rel = f if "/" in f else os.path.join("csrc", f)
        h.update(open(os.path.join(ROOT, "paper_2605_10312_gb300", rel), "rb").read())
    if ent.get("source_sha256") != h.hexdigest():
        return None
    return ent["bytes_per_quartet"] * rec["quartets"], ent.get("fp64_executed_over_algorithmic")


# ---------------------------------------------------------------------------
# ablations of the paper's Sec. V-B on this generator and this GPU
# ---------------------------------------------------------------------------
ABLATION_N = {(1, 1, 1, 1): 100_000, (2, 1, 2, 1): 40_000, (2, 2, 2, 1): 20_000, (2, 2, 2, 2): 10_000,
              (3, 3, 2, 2): 2_000, (3, 3, 3, 3): 1_000}


def run_ablation(args):
    """Axis rule, DSA, spherical fusion and tier ablations: one JSON line per
    (class, variant) with throughput and the generator's graph metrics."""
    import torch
    from paper_2605_10312_gb300 import eri
    from paper_2605_10312_gb300.build import ABLATION_CLASSES, ABLATION_OPTS
    from paper_2605_10312_gb300.gen import hrr, program
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    default = ("prose", "dsa", "stepwise")

    def timed(plan, out, reps=3):
        for _ in range(2):
            plan.compute(out, stream)
        stream.synchronize()
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.compute(out, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    for ls in ABLATION_CLASSES:
        n = max(1, int(ABLATION_N[ls] * SCALE))
        basis, q = synth.class_sweep(ls, n, kset=(1, 3), seed=4000 + sum(ls))
        rows = [(o, "coop") for o in [default] + ABLATION_OPTS]
        rows += [(default, t) for t in ("reg", "shared", "global")]
        for opts, tier in rows:
            try:
                # whole pairs, higher l first: every quartet stays in the
                # generated class (la >= lb, lc >= ld)
                plan = eri.Plan(basis, q, axis_rule=opts[0], schedule=opts[1], sph_mode=opts[2], tier=tier,
                                orientation="l")
            except eri.EriError as e:
                print(json.dumps({"ablation": "".join(map(str, ls)), "opts": opts, "tier": tier,
                                  "unavailable": str(e)}))
                continue
            out = torch.empty(max(1, plan.output_count), dtype=torch.float64, device="cuda")
            ms = timed(plan, out)
            prog = program.make(*ls, *opts)
            c = prog.counts()
            st = plan.stats()
            print(json.dumps({"ablation": "".join(map(str, ls)), "opts": opts, "tier": tier, "quartets": n,
                              "ms": ms, "quartets_per_s": n / (ms * 1e-3),
                              "fp64_tflops": st["flops"] / (ms * 1e-3) / 1e12,
                              "vrr_nodes": c["vrr_nodes"], "peak_live": c["peak_live"],
                              "p2_ops": hrr.op_counts(prog.p2)[0], "flops_per_prim": c["per_prim_flops"]}),
                  flush=True)
            plan.close()
            del out
    return 0


# ---------------------------------------------------------------------------
# batched mixed-class workload: Schwarz-screened water cluster
# ---------------------------------------------------------------------------
def run_water(args):
    """All surviving classes of a Schwarz-screened water cluster (dz shell
    layout) in one plan, replayed as one CUDA graph; optional autotuning."""
    import torch
    from paper_2605_10312_gb300 import eri, screen, tune
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    basis = synth.water_cluster(args.waters, seed=3, layout=args.layout)
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        pairs, qd = screen.pair_bounds_device(basis, stream=stream)
        torch.cuda.synchronize()
        t_bounds = time.perf_counter() - t0
        # the survivor list built on the device (count, prefix sum,
        # compaction), then copied to the host for the planner
        dp = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
        t1 = time.perf_counter()
        qs, ps = screen.sort_pairs(qd, dp)
        dq = eri.screen_quartets(qs, ps, args.threshold, stream)
        torch.cuda.synchronize()
        t_screen_dev = time.perf_counter() - t1
        quartets = dq.cpu().numpy()
        t_screen = time.perf_counter() - t0
        qb = qd.cpu().numpy()
        npairs = pairs.shape[0]
        total = npairs * (npairs + 1) // 2
        tuned = None
        if args.autotune:
            tuned = tune.autotune(basis, quartets, sample=args.tune_sample, shapes=True)
        t1 = time.perf_counter()
        plan = eri.Plan(basis, quartets, digest=args.jk, persistent=args.persistent)
        t_plan = time.perf_counter() - t1
        out = torch.empty(max(1, plan.output_count), dtype=torch.float64, device="cuda")
        plan.set_timing(True)
        plan.compute(out, stream)
        stream.synchronize()
        per_class = {}
        for rec in plan.launches()[1:]:
            key = "".join("spdfg"[x] for x in rec["cls"])
            e = per_class.setdefault(key, {"quartet_parts": 0, "ms": 0.0, "flops": 0.0, "tier": eri.TIERS_INV[rec["tier"]]})
            e["quartet_parts"] += rec["quartets"]
            e["ms"] += rec["ms"]
            e["flops"] += rec["flops"]
        plan.set_timing(False)
        plan.capture(out, stream)
        for _ in range(args.warmup):
            plan.replay(stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.replay(stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
    jk = run_water_jk(args, basis, plan, out, stream) if args.jk else None
    st = plan.stats()
    line = {"workload": "water cluster: {} waters ({} atoms), {} layout, Schwarz {:g}".format(
                args.waters, 3 * args.waters, args.layout, args.threshold),
            "nshell": int(basis.nshell), "pairs": int(npairs), "quartets_total": int(total),
            "quartets_survived": int(quartets.shape[0]), "survived_frac": quartets.shape[0] / total,
            "bounds_s": t_bounds, "screen_s": t_screen, "screen_device_s": t_screen_dev, "plan_s": t_plan,
            "ms_per_step": ms,
            "output_gb": plan.output_count * 8 / 1e9,
            "value": quartets.shape[0] / (ms * 1e-3), "unit": "quartets/s",
            "fp64_tflops": st["flops"] / (ms * 1e-3) / 1e12,
            "fp64_frac_of_peak": st["flops"] / (ms * 1e-3) / 1e12 / fp64_peak_tflops(),
            "launches_per_step": st["launches"] + 1, "graph": True, "persistent": bool(args.persistent), "jk": jk,
            "autotuned": tuned_summary(tuned),
            "per_class": {k: {"parts": v["quartet_parts"], "ms": v["ms"], "tier": v["tier"],
                              "fp64_frac": v["flops"] / max(1e-9, v["ms"] * 1e-3) / 1e12 / fp64_peak_tflops()}
                          for k, v in sorted(per_class.items(), key=lambda kv: -kv[1]["ms"])}}
    print(json.dumps(line))
    return 0


def run_water_jk(args, basis, plan, out, stream):
    """Coulomb and exchange matrices of a random positive semidefinite
    density from the screened list.  Two forms, each a graph replay per step
    after J and K are zeroed: (a) the ERI graph and then the separate
    digestion pass (its HBM roofline counts one read of every block plus
    24 B of quartet data per quartet); (b) eri_compute_jk captured as one
    graph, evaluation and digestion (a persistent plan digests inside its
    launch).  The step time reported is that of (b)."""
    import torch
    nbf = int(sum(2 * l + 1 for l in basis.shell_l))
    rng = np.random.default_rng(11)
    C = rng.standard_normal((nbf, nbf // 4))
    D = torch.from_numpy(C @ C.T / nbf).cuda()
    J = torch.zeros_like(D)
    K = torch.zeros_like(D)
    fused = bool(getattr(args, "persistent", False))

    def timed(body):
        ms, part = [], []
        for it in range(args.warmup + args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            body(e1)
            e2.record(stream)
            e2.synchronize()
            if it >= args.warmup:
                ms.append(e0.elapsed_time(e2))
                part.append(e1.elapsed_time(e2))
        return statistics.mean(ms), statistics.mean(part)

    def separate(e1):
        plan.replay(stream)
        J.zero_()
        K.zero_()
        e1.record(stream)
        plan.digest_jk(out, D, J, K, stream)

    def combined(e1):
        J.zero_()
        K.zero_()
        e1.record(stream)
        plan.replay(stream)

    def energies():
        return {"coulomb": float(torch.sum(D * J).item()), "exchange": float(torch.sum(D * K).item())}

    nq = plan.nq
    res = {"nbf": nbf, "fused": fused, "unit": "quartets/s (ERI + J/K digestion)"}
    with torch.cuda.stream(stream):
        if not fused:
            sep_ms, dig = timed(separate)
            nbytes = 8.0 * plan.output_count + 24.0 * nq
            peak = hbm_peak_gbs()
            res["separate_pass"] = {
                "ms_per_step": sep_ms, "digest_ms": dig, "energies": energies(),
                "digest_roofline": {"bound": "hbm", "achieved": nbytes / (dig * 1e-3) / 1e9, "peak": peak,
                                    "unit": "GB/s", "frac": nbytes / (dig * 1e-3) / 1e9 / peak,
                                    "algorithmic_bytes": nbytes}}
        plan.capture_jk(D, J, K, stream)
        ms, _ = timed(combined)
        res.update({"ms_per_step": ms, "value": nq / (ms * 1e-3), "energies": energies()})
        # leave the plan's graph as the ERI-only one
        plan.capture(out, stream)
    return res


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300 (MEASURED_PEAKS.json), else
    6.8 TB/s, an earlier copy measurement on a GB300."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def _class_labels(basis, quartets):
    """Canonical class label of each quartet (pairs ordered high l first,
    bra pair not below the ket pair) and the list of labels."""
    l = basis.shell_l[np.asarray(quartets)]
    bra = np.sort(l[:, :2], axis=1)[:, ::-1]
    ket = np.sort(l[:, 2:], axis=1)[:, ::-1]
    swap = bra[:, 0] * 5 + bra[:, 1] < ket[:, 0] * 5 + ket[:, 1]
    hi = np.where(swap[:, None], ket, bra)
    lo = np.where(swap[:, None], bra, ket)
    code = ((hi[:, 0] * 5 + hi[:, 1]) * 5 + lo[:, 0]) * 5 + lo[:, 1]
    uniq, inv = np.unique(code, return_inverse=True)
    labels = ["".join("spdfg"[(c // 5 ** k) % 5] for k in (3, 2, 1, 0)) for c in uniq]
    return inv, labels


def run_water_mixed(args):
    """Mixed precision on a screened water cluster: quartets with Schwarz
    bound below --fp32-below run FP32 recurrences.  Times the mixed plan and
    the all-FP64 plan on the same quartets (CUDA graphs) and reports the
    per-class max and RMS difference between them."""
    import torch
    from paper_2605_10312_gb300 import eri, screen
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    basis = synth.water_cluster(args.waters, seed=3, layout=args.layout)
    with torch.cuda.stream(stream):
        pairs, qp = screen.pair_bounds(basis, stream=stream)
        total = synth.count_screened(qp, args.threshold)
        if args.sample and args.sample < total:
            quartets = synth.sample_screened_quartets(qp, pairs, args.threshold, args.sample, seed=7)
        else:
            quartets = synth.screened_quartets(qp, pairs, args.threshold)
        qb = screen.quartet_bounds(qp, quartets)
        plans = {"fp64": eri.Plan(basis, quartets),
                 "mixed": eri.Plan(basis, quartets, qbound=qb, fp32_below=args.fp32_below)}
        outs, ms, launch_ms = {}, {}, {}
        for name, p in plans.items():
            o = torch.empty(max(1, p.output_count), dtype=torch.float64, device="cuda")
            # one timed pass for the per-class, per-precision split
            p.set_timing(True)
            p.compute(o, stream)
            stream.synchronize()
            for rec in p.launches()[1:]:
                key = "{}/{}".format("".join("spdfg"[x] for x in rec["cls"]), rec["precision"])
                launch_ms[(name, key)] = launch_ms.get((name, key), 0.0) + rec["ms"]
            p.set_timing(False)
            p.capture(o, stream)
            for _ in range(args.warmup):
                p.replay(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                p.replay(stream)
            e1.record(stream)
            e1.synchronize()
            ms[name] = e0.elapsed_time(e1) / args.steps
            outs[name] = o
        off = plans["fp64"].offsets()
        cls, labels = _class_labels(basis, quartets)
        fp32q = qb < args.fp32_below
        sizes = torch.from_numpy(np.diff(off)).to("cuda")
        cid = torch.repeat_interleave(torch.from_numpy(cls.astype(np.int64)).to("cuda"), sizes)
        d = (outs["mixed"][: off[-1]] - outs["fp64"][: off[-1]]).abs()
        nc = len(labels)
        mx = torch.zeros(nc, dtype=torch.float64, device="cuda").scatter_reduce_(0, cid, d, reduce="amax")
        ss = torch.zeros(nc, dtype=torch.float64, device="cuda").index_add_(0, cid, d * d)
        cnt = torch.zeros(nc, dtype=torch.float64, device="cuda").index_add_(0, cid, torch.ones_like(d))
        mx, rms = mx.cpu().numpy(), torch.sqrt(ss / cnt.clamp(min=1)).cpu().numpy()
        stream.synchronize()
    st = plans["mixed"].stats()
    per_class = {}
    for k, lab in enumerate(labels):
        sel = cls == k
        per_class[lab] = {"quartets": int(sel.sum()), "fp32_quartets": int((sel & fp32q).sum()),
                          "max_abs_diff_vs_fp64": float(mx[k]), "rms_diff_vs_fp64": float(rms[k])}
    line = {"workload": "water cluster: {} waters ({} atoms), {} layout, Schwarz {:g}, FP32 below {:g}".format(
                args.waters, 3 * args.waters, args.layout, args.threshold, args.fp32_below),
            "nshell": int(basis.nshell), "pairs": int(pairs.shape[0]), "quartets_screened": int(total),
            "quartets": int(quartets.shape[0]),
            "sample": None if quartets.shape[0] == total else "uniform seeded sample of the screened list",
            "fp32_quartets": int(fp32q.sum()), "fp32_parts": st["fp32_parts"],
            "ms_fp64": ms["fp64"], "ms_mixed": ms["mixed"], "speedup": ms["fp64"] / ms["mixed"],
            "value_mixed": quartets.shape[0] / (ms["mixed"] * 1e-3),
            "value_fp64": quartets.shape[0] / (ms["fp64"] * 1e-3), "unit": "quartets/s",
            "max_abs_diff_vs_fp64": float(mx.max()), "per_class": per_class,
            "launch_ms": {n: {k: v for (nn, k), v in sorted(launch_ms.items(), key=lambda kv: -kv[1]) if nn == n}
                          for n in plans}}
    print(json.dumps(line))
    return 0


def run_per_k(args):
    """Per class and fixed contraction depth K in {1, 3, 6} (all four shells
    the same K): quartets/s and FP64 fraction, L2 flushed between repeats."""
    import torch
    from paper_2605_10312_gb300 import eri
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # quartets per run: about half a second of work at the measured rates
    counts = {1: {1: 2_000_000, 3: 400_000, 6: 40_000}, 2: {1: 1_000_000, 3: 200_000, 6: 20_000},
              3: {1: 200_000, 3: 20_000, 6: 2_000}, 4: {1: 40_000, 3: 4_000, 6: 400}}
    rows = {}
    for ls, _ in SWEEP:
        for K in (1, 3, 6):
            n = max(1, int(counts[ls[0]][K] * SCALE))
            basis, q = synth.class_sweep(ls, n, kset=(K,), seed=SEED + 10 * ls[0] + K)
            tuned = None
            if args.autotune:
                from paper_2605_10312_gb300 import tune
                tuned = tune.autotune(basis, q, sample=args.tune_sample, shapes=True)
            p = eri.Plan(basis, q, votes=args.votes, persistent=args.persistent)
            if tuned:
                # this (class, K) only: the next one starts from the static choices
                for c in tuned:
                    eri.set_class_tier(c, 0)
                    for kind in eri.KINDS:
                        eri.set_class_shape(c, kind, -1)
            out = torch.empty(p.output_count, dtype=torch.float64, device="cuda")
            ms = []
            for it in range(args.warmup + args.steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                p.compute(out, stream)
                e1.record(stream)
                e1.synchronize()
                if it >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            t = statistics.mean(ms)
            fl = p.stats()["flops"]
            rows["{}_K{}".format("".join("spdfg"[x] for x in ls), K)] = {
                "quartets": n, "ms": t, "quartets_per_s": n / (t * 1e-3),
                "fp64_frac_of_peak": fl / (t * 1e-3) / 1e12 / fp64_peak_tflops(),
                "flops_per_quartet": fl / n, "autotuned": tuned_summary(tuned)}
            p.close()
            del out
    print(json.dumps({"workload": "per-class sweep at fixed K (all four shells), 10 Angstrom box",
                      "l2": "flushed between repeats", "steps": args.steps, "per_class_k": rows}))
    return 0


def run_serve(args):
    """Serving loop with continuous batching: a pool of seeded water clusters
    (dz layout, 4-66 waters) registered on the device, requests of a seeded
    slice of a molecule's Schwarz-screened quartet list (log-uniform in
    [1e3, 1e6] quartets), mixed FP32/FP64 policy.  Phases: a burst (all
    requests at t = 0: the capacity), Poisson arrivals at --rate, at 70% of
    the capacity and at 150% of it."""
    import torch
    from paper_2605_10312_gb300 import eri, serve
    torch.cuda.set_device(0)
    eri.library()
    rng = np.random.default_rng(5)
    # host planner threads: all cores but two (the request loop and the CUDA
    # driver's own threads), at most 16
    planners = args.planners or max(1, min(16, (os.cpu_count() or 3) - 2))
    srv = serve.Server(budget_bytes=args.serve_budget_gb << 30, slots=args.slots, planners=planners,
                       fp32_below=args.fp32_below if args.fp32_below is not None else 1e-6, timeout_s=30.0,
                       chunk_quartets=args.chunk or None)
    t0 = time.perf_counter()
    pools = {}
    sizes = sorted(int(x) for x in rng.integers(4, 67, size=args.molecules))
    for k, nw in enumerate(sizes):
        mol = srv.register(k, synth.water_cluster(nw, seed=500 + k, layout="dz"))
        pools[k] = serve.screened_pool(mol, args.threshold, 2_000_000, seed=k)
    setup_s = time.perf_counter() - t0
    # warm-up: compile-free, but first plans of each class upload programs
    srv.serve(serve.poisson_requests(pools, 1.0, 8, seed=99, burst=True))
    phases = {}
    burst = serve.poisson_requests(pools, 1.0, args.requests, seed=1, burst=True)
    phases["burst"] = serve.summary(srv.serve(burst), offered_span=0.0)
    cap = phases["burst"]["served_requests_per_s"]
    for name, rate, seed in (("rate_{:g}".format(args.rate), args.rate, 2), ("capacity_70pct", 0.7 * cap, 3),
                             ("capacity_150pct", 1.5 * cap, 4)):
        reqs = serve.poisson_requests(pools, rate, args.requests, seed=seed)
        phases[name] = dict(serve.summary(srv.serve(reqs)), rate=rate)
    srv.close()
    line = {"workload": "serving: Poisson ERI requests over {} water clusters ({} waters), dz layout, "
                        "Schwarz {:g}, requests of 1e3-1e6 quartets, FP32 below {:g}".format(
                            len(sizes), sizes, args.threshold, srv.fp32_below),
            "slots": args.slots, "planners": planners, "budget_gb": args.serve_budget_gb,
            "chunk_quartets": args.chunk or None,
            "requests_per_phase": args.requests, "setup_s": setup_s, "capacity_requests_per_s": cap,
            "phases": phases}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--classes", default="", help="comma-separated subset, e.g. gggg (profiling runs)")
    ap.add_argument("--scale", type=float, default=1.0, help="multiply the quartet counts (profiling runs)")
    ap.add_argument("--ablation", action="store_true", help="axis / DSA / spherical / tier ablations instead")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "water", "serve", "per-k"])
    ap.add_argument("--rate", type=float, default=50.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests per phase")
    ap.add_argument("--molecules", type=int, default=8, help="serve: molecules in the pool")
    ap.add_argument("--slots", type=int, default=16, help="serve: concurrent requests (streams)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="serve: requests above this many quartets run as parallel chunk plans while few "
                         "requests are in flight (0: never)")
    ap.add_argument("--planners", type=int, default=0, help="serve: host planner threads (0: cores - 2)")
    ap.add_argument("--serve-budget-gb", type=int, default=16, help="serve: device-memory budget")
    ap.add_argument("--waters", type=int, default=20)
    ap.add_argument("--layout", default="dz", choices=["dz", "tz"])
    ap.add_argument("--threshold", type=float, default=1e-10)
    ap.add_argument("--autotune", action="store_true",
                    help="tune tiers, cooperative shapes and vote forms on a sample before planning")
    ap.add_argument("--tune-sample", type=int, default=1024, help="quartets per class group the autotuner times")
    ap.add_argument("--votes", default="auto", choices=["auto", "off", "on"],
                    help="team-cooperative programs: warp votes around optional FP64 terms")
    ap.add_argument("--persistent", action="store_true",
                    help="persistent plans: every class in one launch per precision over a device work list")
    ap.add_argument("--jk", action="store_true", help="water workload: also digest into J and K")
    ap.add_argument("--fp32-below", type=float, default=None,
                    help="water workload in mixed precision: FP32 recurrences below this Schwarz bound")
    ap.add_argument("--sample", type=int, default=0, help="water workload: sample this many screened quartets")
    args = ap.parse_args()
    global ONLY, SCALE
    ONLY = set(c for c in args.classes.split(",") if c) or None
    SCALE = args.scale
    if args.impl == "reference":
        return run_reference(args)
    if args.ablation:
        return run_ablation(args)
    if args.workload == "water":
        return run_water_mixed(args) if args.fp32_below is not None else run_water(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "per-k":
        return run_per_k(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
