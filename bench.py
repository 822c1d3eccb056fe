#!/usr/bin/env python
"""FCIQMC configurations updated per second on GB300.

Headline workload (default): c5 in the paper's FP64 arithmetic -- 2D periodic
8 x 8 real-space Bose-Hubbard model, N = 64, t = 1, U = 8 (127-bit addresses),
FP64 amplitudes, threshold 1, target N_t = 5e8 walkers, dt = 2e-4, started
from N_w = 10 on uniform filling.  The first 25 % of the configuration's 2000
steps are equilibration (untimed, as the paper discards equilibration); then
the autotuner, W warm-up steps and K timed steps.

value   = sum over timed steps of len (occupied configurations updated) /
          device time of the K steps (CUDA events on the run's stream,
          graph-replayed steps), summed over ranks / max time over ranks.
e2e     = the same metric through the public API as a user drives it: per
          step one parameter write from pinned host memory, one step, and
          one read of the step's statistics row back to the host.
roofline= the dominant kernel's algorithmic bytes per launch / its mean
          CUDA-event duration (steps launched kernel by kernel right after
          the timed region), against the measured HBM copy bandwidth.
cpu_baseline = the CPU oracle, single thread, on a bounded sample of the
          equilibrated vector (rank 0, N = 1 only).

At N = 1 the same JSON line also carries, under "more", the other measured
forms: c5 as configured (FP32 amplitudes), c2 (1D, FP64), and the c4
equal-error comparison (64 runs as one FP32 batch, as one FP64 batch, and
one after another in FP64).  --config/--mode pick another workload alone.

--impl reference runs the CPU oracle instead (the paper ships no GPU code):
each step is one oracle step on a bounded sample of the same workload.
With --gpus N > 1 under torchrun every rank steps an independent replica
(run_id = rank): the step has no data-path exchange to shard.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "FCIQMC configs updated/s"
UNIT = "configs/s"
MODE_CODE = {"INT": 0, "REAL64": 1, "REAL32": 2, "DETERMINISTIC": 3}
DTYPE = {"INT": "int64", "REAL64": "f64", "REAL32": "f32", "DETERMINISTIC": "f64"}
ANN_CODE = {"auto": 0, "sort": 1, "hash": 2}
# bytes fq_run_stats copies back per call: the error word and the run state
STATS_D2H_BYTES = 4 + 192  # the error word, then the 192-byte run state
# the sources a committed ncu summary depends on: the kernels, and the host
# code that sizes the buffers, tables and launch shapes they run with
KERNEL_FILES = ["fq_kernels.cuh", "fq_device.cuh", "fq_shared.h", "fq_launch.cuh", "fq_api.cu"]


def describe(cfg, name):
    kind = {1: "1D periodic real-space", 2: "2D periodic real-space", 3: "1D momentum-space"}
    lat = "%dx%d" % (cfg["Lx"], cfg["Ly"]) if cfg["kind"] == 2 else "M=%d" % cfg["Lx"]
    return ("%s: %s Bose-Hubbard %s, N=%d, t=%g, U=%g, %s, N_t=%.0e, dt=%g, seed %d, start 10 "
            "walkers on the starting address" % (name, kind[cfg["kind"]], lat, cfg["N"], cfg["t"],
                                                 cfg["u"], cfg["mode"], cfg["target"], cfg["dt"],
                                                 cfg["seed"]))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    """Barrier and max/sum over ranks (a no-op for one process)."""

    def __init__(self, world, backend):
        self.world = world
        self.dist = None
        if world > 1:
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def reduce(self, value: float, op: str) -> float:
        if not self.dist:
            return value
        import torch

        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX if op == "max" else self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


def aggregate(dist: Dist, elapsed_s: float, units: float):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    t = dist.reduce(elapsed_s, "max")
    u = dist.reduce(units, "sum")
    return u / t, t


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_digest():
    """Digest of the kernel sources with comments and blank space removed, so
    that only a change of the code itself makes a committed ncu summary stale."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_2601_19505_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_per_alg_byte(kernel: str, workload: str):
    """DRAM bytes per algorithmic byte of `kernel` from a committed ncu summary
    (profiles/<kernel>_<workload>.md), if its kernel digest is current."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    try:
        if vals.get("kernel_digest") != kernel_digest():
            return None
        return float(vals["dram_bytes_per_launch"]) / float(vals["algorithmic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def sizes(cfg):
    kb = 8 if cfg["N"] + cfg["Lx"] * cfg["Ly"] - 1 <= 64 else 16
    ab = {"INT": 8, "REAL64": 8, "REAL32": 4, "DETERMINISTIC": 8}[cfg["mode"]]
    sb = {"INT": 4, "REAL64": 8, "REAL32": 4, "DETERMINISTIC": 8}[cfg["mode"]]
    return kb, ab, sb


# ---------------------------------------------------------------------------
# CPU oracle timings (baseline only)

def oracle_rate(cfg, keys_int, amps, shift, step, budget_s=12.0, seed=0):
    """Oracle configs/s on a bounded sample: one step on n entries, n grown
    until one step takes about budget_s / 3, then timed once more."""
    import oracle as O

    m = O.Model(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], cfg["t"], cfg["u"])
    p = O.default_params(mode=MODE_CODE[cfg["mode"]], dt=cfg["dt"], target=cfg["target"],
                         seed=cfg["seed"])
    rng = np.random.default_rng(seed)
    n = min(len(keys_int), 20000)
    rate = None
    while True:
        idx = np.sort(rng.choice(len(keys_int), n, replace=False))
        run = O.Run(m, p)
        run.seed([keys_int[i] for i in idx], amps[idx], shift, step)
        t0 = time.perf_counter()
        run.step(1)
        dt = time.perf_counter() - t0
        rate = n / dt
        if dt > budget_s / 3 or n >= len(keys_int):
            return rate, n, dt
        n = int(min(len(keys_int), n * max(2.0, (budget_s / 3) / dt)))


def synthetic_vector(cfg, n, seed):
    import oracle as O

    m = O.Model(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], cfg["t"], cfg["u"])
    rng = np.random.default_rng(seed)
    occ = W.random_occupations(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], n, rng, max_moves=30)
    keys = [m.encode(o) for o in occ]
    amps = W.random_amplitudes(len(keys), rng, mode=cfg["mode"])
    return keys, amps, m


def reference_arm(args, cfg, name):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O

    O.build()
    budget = 150.0
    pool_n = 60000
    keys, amps, m = synthetic_vector(cfg, pool_n, 1)
    p = O.default_params(mode=MODE_CODE[cfg["mode"]], dt=cfg["dt"], target=cfg["target"],
                         seed=cfg["seed"])
    # calibrate the per-entry cost, then size each step's sample
    run = O.Run(m, p)
    run.seed(keys[:5000], amps[:5000], -2.0, 1000)
    t0 = time.perf_counter()
    run.step(1)
    per = (time.perf_counter() - t0) / 5000
    n = int(max(200, min(pool_n, budget / max(1, args.steps + args.warmup) / per)))
    rng = np.random.default_rng(2)
    tot_t, tot_n = 0.0, 0
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(len(keys), n, replace=False))
        run = O.Run(m, p)
        run.seed([keys[i] for i in idx], amps[idx], -2.0, 1000 + s)
        t0 = time.perf_counter()
        run.step(1)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            tot_t += dt
            tot_n += n
    value = tot_n / tot_t
    sample = ("each step: one oracle step on %d entries drawn from a seeded synthetic %d-entry "
              "vector of the %s workload (random hop walks from uniform filling, "
              "threshold-shaped amplitudes)" % (n, pool_n, name))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[cfg["mode"]], "data": "synthetic",
            "config": {"workload": describe(cfg, name), "sample_entries_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm

def release_device_memory():
    import gc

    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def gpu_arm(args, cfg, name, dist, with_cpu=True):
    """Measure one workload; the JSON object of the line (rank 0) or None."""
    import torch

    import paper_2601_19505_gb300 as fq

    rank, world, local = dist_env()
    h = fq.Hamiltonian(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], cfg["t"], cfg["u"])
    p = fq.default_params(mode=MODE_CODE[cfg["mode"]], dt=cfg["dt"], target=cfg["target"],
                          seed=cfg["seed"], run_id=rank, annihilation=ANN_CODE[args.annihilation],
                          capacity_vec=int(args.capacity_vec), capacity_spawn=int(args.capacity_spawn))
    run = fq.Run(h, p)
    run.seed_default(W.START_WEIGHT)
    equil = args.equil if args.equil is not None else cfg["steps"] // 4
    done = 0
    while done < equil:
        k = min(250, equil - done)
        run.advance(k, chunk=k)  # grows the capacities if a step overflows them
        done += k
    tune_steps = 0
    if not args.no_autotune:
        s_before = run.stats()["step"]
        run.autotune(2)
        tune_steps = run.stats()["step"] - s_before
    run.step(args.warmup)
    run.stats()
    run.history()  # drain
    stream = torch.cuda.ExternalStream(run.stream) if run.stream else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    run.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    dist.barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    hist = run.history()
    assert len(hist) == args.steps, (len(hist), args.steps)
    units = float(hist["len"].sum())
    value, tmax = aggregate(dist, elapsed, units)

    # per-kernel durations right after the timed region (kernel-by-kernel launch)
    nprof = min(200, max(20, args.steps // 10))
    before = run.stats()
    ms = run.profile(nprof)
    prof = run.history()
    kb, ab, sb = sizes(cfg)
    L_in = np.r_[before["len"], prof["len"][:-1]].astype(float)
    L_out = prof["len"].astype(float)
    S = prof["n_spawns"].astype(float)
    alg = {"spawn": float(np.mean(L_in * (kb + ab) + S * (kb + sb))),
           "merge": float(np.mean(L_in * (kb + ab) + S * (kb + sb) + L_out * (kb + ab)))}
    kms = {"spawn": ms[0], "merge": ms[1], "shift": ms[2]}
    dom = "merge" if ms[1] >= ms[0] else "spawn"
    peak, peak_kind = measured_peak()
    achieved = alg[dom] / (kms[dom] * 1e-3) / 1e9
    ratio = traffic_per_alg_byte("k_" + dom, name)
    traffic = alg[dom] * ratio if ratio else None

    # end to end through the public API, host buffers in the loop
    ne2e = min(args.steps, 1000)
    t0 = time.perf_counter()
    e2e_units = 0
    for _ in range(ne2e):
        run.set_target(cfg["target"])
        run.step(1)
        e2e_units += run.stats()["len"]
    e2e_t = time.perf_counter() - t0
    e2e_value, _ = aggregate(dist, e2e_t, float(e2e_units))
    paths = run.merge_paths()
    shape = run.shape()
    arms = run.arm_times()

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and with_cpu and not args.no_cpu_baseline:
            # a bounded random sample of whole segments of the equilibrated
            # vector (exporting the whole vector would take minutes at 5e8)
            keys, amps = run.sample(400000, seed=1)
            kint = [int(k["lo"]) | (int(k["hi"]) << 64) for k in keys] if kb == 16 else \
                keys["lo"].astype(object).tolist()
            st = run.stats()
            rate, n, tsec = oracle_rate(cfg, kint, amps, st["shift"], st["step"])
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "one single-threaded oracle step on %d entries drawn at random from "
                             "whole segments of the equilibrated GPU vector (len %d), %.1f s"
                             % (n, st["len"], tsec)}
        L_mean = float(hist["len"].mean())
        S_mean = float(hist["n_spawns"].mean())
        ws = 2 * L_mean * (kb + ab) + 2 * S_mean * (kb + sb)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[cfg["mode"]], "data": "synthetic",
            "config": {"workload": describe(cfg, name), "equilibration_steps": equil,
                       "autotune_steps": tune_steps, "len_mean": L_mean,
                       "spawns_mean": S_mean,
                       "exact_columns_mean": float(hist["exact_steps"].mean()),
                       "graph_replay": True,
                       "l2": "working set per step %.2f GB > 129 MB L2; no flush" % (ws / 1e9),
                       "parallelism": "replicas x%d" % world,
                       "launch_shape": shape,
                       "annihilation": shape["annihilation"],
                       "autotuner_merge_ms_per_arm": arms,
                       "merge_buckets_onchip_scratch": list(paths)},
            "roofline": {"bound": "hbm", "kernel": "k_" + dom, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                         if peak_kind == "measured" else "fallback 6800 GB/s",
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": alg[dom],
                         "kernel_ms": kms,
                         "kernel_gbs": {k: alg[k] / (kms[k] * 1e-3) / 1e9 for k in alg},
                         "kernel_frac": {k: alg[k] / (kms[k] * 1e-3) / 1e9 / peak for k in alg}},
            "cpu_baseline": cpu,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8,
                    "d2h_bytes_per_step": STATS_D2H_BYTES, "steps": ne2e},
            "gpu_launches": 3 * args.steps,
        }
    run.close()
    del run
    release_device_memory()
    return out


def brief(line):
    """The figures of a measured workload that the headline line nests."""
    r = line["roofline"]
    return {"workload": line["config"]["workload"], "value": line["value"], "unit": line["unit"],
            "dtype": line["dtype"], "ms_per_step": line["ms_per_step"],
            "len_mean": line["config"]["len_mean"], "spawns_mean": line["config"]["spawns_mean"],
            "kernel_ms": r["kernel_ms"], "kernel_gbs": r["kernel_gbs"],
            "kernel_frac": r["kernel_frac"], "dominant": r["kernel"], "frac": r["frac"],
            "annihilation": line["config"]["annihilation"],
            "autotuner_merge_ms_per_arm": line["config"]["autotuner_merge_ms_per_arm"],
            "clocks": line.get("clocks")}


# ---------------------------------------------------------------------------
# Equal-error comparison: the 64 runs of c4 stepped as one FP32 batch, as one
# FP64 batch, and one after another in plain FP64

def equal_error_arm(args):
    import torch

    import paper_2601_19505_gb300 as fq
    from paper_2601_19505_gb300 import analysis as A

    cfgs = W.batch_configs(64, seed=1)
    steps = cfgs[0]["steps"]
    equil = steps // 4
    timed = steps - equil

    def make(c, mode):
        h = fq.Hamiltonian(c["kind"], c["Lx"], c["Ly"], c["N"], c["t"], c["u"])
        p = fq.default_params(mode=MODE_CODE[mode], dt=c["dt"], target=c["target"],
                              seed=c["seed"], run_id=c["run_id"])
        r = fq.Run(h, p)
        r.seed_default(W.START_WEIGHT)
        return h, r

    def timed_steps(step_fn, stream_handle, n):
        stream = torch.cuda.ExternalStream(stream_handle) if stream_handle \
            else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step_fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def estimates(hist):
        e = A.ratio_estimate(hist["hproj"], hist["vproj"])
        sh = A.blocked_mean(hist["shift"])
        return (e["ratio"], e["err"], float(hist["len"].sum()), sh["mean"], sh["err"],
                float(np.mean(hist["vproj"])), float(np.mean(hist["len"])))

    def batched(mode):
        made = [make(c, mode) for c in cfgs]
        runs = [r for _, r in made]
        batch = fq.Batch(runs)
        batch.step(equil)
        try:
            batch.sync()
        except fq.FqError:
            bad = [(c["run_id"], c["Lx"], c["target"], r.error_bits(), r.capacity())
                   for c, r in zip(cfgs, runs) if r.error_bits()]
            raise RuntimeError("batched %s runs failed: %s" % (mode, bad))
        if not args.no_autotune:
            batch.autotune(2)
        batch.sync()
        for r in runs:
            r.history()
        t = timed_steps(batch.step, runs[0].stream, timed)
        batch.sync()
        est = [estimates(r.history()) for r in runs]
        batch.close()
        for r in runs:
            r.close()
        release_device_memory()
        return t, est

    t32, est32 = batched("REAL32")
    t64b, est64b = batched("REAL64")
    # plain FP64, one run after another
    t64, est64 = 0.0, []
    for c in cfgs:
        h, r = make(c, "REAL64")
        r.step(equil)
        r.sync()
        r.history()
        t64 += timed_steps(r.step, r.stream, timed)
        if r.sync():
            raise RuntimeError("FP64 run %d failed" % c["run_id"])
        est64.append(estimates(r.history()))
        r.close()
    release_device_memory()

    def pick(a, b):
        # the projected energy where both forms give a finite estimate with an
        # error bar, else the shift estimator
        fin = all(np.isfinite(v) and v != 0.0 for v in (a[0], a[1], b[0], b[1]))
        return (a[0], a[1], b[0], b[1], "projected") if fin else (a[3], a[4], b[3], b[4], "shift")

    def compare(ta, ea, tb, eb):
        """a against b at equal error: b's time over the time a needs for b's error bars."""
        use = [pick(x, y) for x, y in zip(ea, eb)]
        vr = np.array([(u[1] / u[3]) ** 2 for u in use])
        agree = sum(1 for u in use if abs(u[0] - u[2]) <= 2.0 * math.hypot(u[1], u[3]))
        return use, {"median_var_ratio": float(np.median(vr)), "max_var_ratio": float(vr.max()),
                     "speedup_to_equal_error_median": tb / (ta * float(np.median(vr))),
                     "speedup_to_equal_error_worst": tb / (ta * float(vr.max())),
                     "energies_agree_2sigma": agree, "runs": len(use)}

    u32 = sum(e[2] for e in est32)
    u64b = sum(e[2] for e in est64b)
    u64 = sum(e[2] for e in est64)
    use, total = compare(t32, est32, t64, est64)
    _, batching = compare(t64b, est64b, t64, est64)
    _, precision = compare(t32, est32, t64b, est64b)
    return {
        "workload": "c4: 64 periodic 1D real-space Bose-Hubbard runs, M = N ~ U{10..30}, "
                    "U/t ~ U[1, 10], N_t log-uniform in [1e4, 1e6] (default_rng(1)), dt = 1e-3, "
                    "5000 steps (first 25 % untimed), 10 walkers on uniform filling",
        "timed_steps": timed,
        "fp32_batch": {"seconds": t32, "configs_per_s": u32 / t32},
        "fp64_batch": {"seconds": t64b, "configs_per_s": u64b / t64b},
        "fp64_sequential": {"seconds": t64, "configs_per_s": u64 / t64},
        "fp32_batch_vs_fp64_sequential": total,
        "batching_alone_fp64_batch_vs_fp64_sequential": batching,
        "precision_alone_fp32_batch_vs_fp64_batch": precision,
        "estimator_shift_runs": sum(1 for u in use if u[4] == "shift"),
        "median_err_fp64": float(np.median([u[3] for u in use])),
        "per_run": [{"M": c["Lx"], "U": round(c["u"], 4), "N_t": round(c["target"]),
                     "E32": u[0], "err32": u[1], "E64": u[2], "err64": u[3], "est": u[4]}
                    for c, u in zip(cfgs, use)],
    }


# ---------------------------------------------------------------------------
# c3 (momentum space, sign problem): FP32 against FP64 amplitudes at the step
# where the population first reaches N_t.  The overshoot that follows (about
# ten times N_t) leaves no equilibrated window, so this compares throughput
# on the same state size, not error bars.

def c3_precision_arm(args):
    import torch

    import paper_2601_19505_gb300 as fq

    torch.cuda.set_device(0)
    cfg = W.CONFIGS["c3"]
    out = {}
    n = min(args.steps, 3)
    for mode in ("REAL32", "REAL64"):
        # each annihilation arm on its own run: the autotuner's trial steps
        # would outgrow any capacity while the population grows ~25 % a step
        arms = {}
        for ann in ("hash", "sort"):
            h = fq.Hamiltonian(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], cfg["t"], cfg["u"])
            p = fq.default_params(mode=MODE_CODE[mode], dt=cfg["dt"], target=cfg["target"],
                                  seed=cfg["seed"], annihilation=ANN_CODE[ann])
            run = fq.Run(h, p)
            run.seed_default(W.START_WEIGHT)
            st = run.stats()
            while st["norm"] < cfg["target"] and st["step"] < 1000:
                run.advance(2, chunk=2)
                st = run.stats()
            run.reserve(int(5e8), int(1e9))  # the timed steps keep growing ~25 % each
            before = run.stats()
            ms = run.profile(n)
            hist = run.history()
            units = float(hist["len"][-n:].sum())
            t = (ms[0] + ms[1] + ms[2]) * 1e-3 * n
            arms[ann] = {"configs_per_s": units / t, "ms_per_step": 1e3 * t / n,
                         "kernel_ms": {"spawn": ms[0], "merge": ms[1], "shift": ms[2]},
                         "step": before["step"], "len": before["len"], "norm": before["norm"]}
            run.close()
            del run
            release_device_memory()
        best = max(arms, key=lambda a: arms[a]["configs_per_s"])
        out[mode] = dict(arms[best], annihilation=best, arms=arms)
    line = {"metric": METRIC + " (c3, FP32 vs FP64 amplitudes at N = N_t)",
            "value": out["REAL32"]["configs_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": min(args.steps, 3), "warmup": 0, "ms_per_step": out["REAL32"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": describe(cfg, "c3") + "; timed once the one-norm first "
                                   "reaches N_t, kernel by kernel (CUDA events)"},
            "precision": out}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# c3 trajectories: FP32 against FP64 amplitudes over the configuration's 5000
# steps at reduced targets, blocked energies where the population holds at
# its target, and the full target's population over its first steps

def c3_trajectory_arm(args):
    import paper_2601_19505_gb300 as fq
    from paper_2601_19505_gb300 import analysis as A

    cfg = dict(W.CONFIGS["c3"])
    out = {"workload": describe(cfg, "c3"), "runs": []}

    def one(mode, target, steps, zeta=None):
        h = fq.Hamiltonian(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], cfg["t"], cfg["u"])
        kw = {} if zeta is None else {"zeta": zeta}
        p = fq.default_params(mode=MODE_CODE[mode], dt=cfg["dt"], target=target, seed=cfg["seed"],
                              **kw)
        run = fq.Run(h, p)
        run.seed_default(W.START_WEIGHT)
        rows = []
        t0 = time.perf_counter()
        done = 0
        stopped = None
        while done < steps:
            k = min(50, steps - done)
            try:
                run.advance(k, chunk=50, grow=2.0, max_grows=12)
            except fq.FqError as e:  # the population outgrew the device memory
                stopped = "%s (capacity %s)" % (e, list(run.capacity()))
                rows.append(run.history())
                break
            rows.append(run.history())
            done += k
        hist = np.concatenate(rows)
        wall = time.perf_counter() - t0
        run.close()
        release_device_memory()
        half = hist[len(hist) // 2:]
        rec = {"mode": mode, "target": target, "zeta": p.zeta, "xi": p.xi,
               "steps": int(len(hist)), "wall_s": wall, "stopped": stopped,
               "norm_over_target_last_half": float(np.mean(half["norm"]) / target),
               "len_max": int(hist["len"].max()), "step_of_len_max": int(hist["step"][np.argmax(hist["len"])]),
               "trajectory_every_10": [[int(r["step"]), int(r["len"]), float(r["norm"]),
                                        float(r["shift"]), int(r["n_spawns"]),
                                        int(r["exact_steps"])] for r in hist[::10]]}
        sh = A.blocked_mean(half["shift"])
        e = A.ratio_estimate(half["hproj"], half["vproj"])
        rec["shift_last_half"] = [sh["mean"], sh["err"]]
        rec["projected_last_half"] = [e["ratio"], e["err"]]
        out["runs"].append(rec)
        return rec

    for target in (1e5, 1e6):
        for mode in ("REAL32", "REAL64"):
            one(mode, target, cfg["steps"])
    one("REAL32", cfg["target"], args.steps)
    # the damping scaled with the time step: zeta / dt = 8, as the defaults
    # have at dt = 0.01 (and xi = zeta^2 / 4)
    for mode in ("REAL32", "REAL64"):
        one(mode, 1e6, cfg["steps"], zeta=0.08 * cfg["dt"] / 0.01)
    print(json.dumps({"metric": METRIC + " (c3 trajectories)", "c3_trajectory": out}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Late against early compression and the semistochastic threshold t_rel
# (Sec. 7, Eq. early-comp): the statistical efficiency of the shift,
# f = 1 / (sigma_S^2 Omega t~) with the blocked error sigma_S of its mean,
# Omega timed steps and t~ the median time of a step (here CUDA-event time
# on the GPU), on the model families of the paper's two comparisons: real
# space M = N = 12, u = 6 (t_rel and the compression style), and momentum
# space M = N = 10, u = 6 (the compression style against N_t, where the
# sign problem shows).  The exact-column rule is |c| t_rel >= m (reading of
# Sec. 7.1), so a smaller t_rel takes fewer exact columns.

def compression_sweep_arm(args):
    import torch

    import paper_2601_19505_gb300 as fq
    from paper_2601_19505_gb300 import analysis as A

    steps = max(1000, int(args.sweep_steps))
    chunk = 1000
    equil = steps // 10
    out = {"steps": steps, "equilibration_steps": equil, "chunk": chunk, "dt": 1e-3,
           "real_space": [], "momentum_space": []}

    def one(kind, M, N, u, target, compression, t_rel, seed=1):
        h = fq.Hamiltonian(kind, M, 1, N, 1.0, u)
        p = fq.default_params(mode=MODE_CODE["REAL64"], dt=1e-3, target=float(target), seed=seed,
                              compression=compression, t_rel=float(t_rel))
        run = fq.Run(h, p)
        run.seed_default(W.START_WEIGHT)
        run.advance(equil, chunk=min(equil, 5000))
        run.history()  # drain the equilibration rows
        stream = torch.cuda.ExternalStream(run.stream) if run.stream else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times, rows = [], []
        for _ in range(steps // chunk):
            torch.cuda.synchronize()
            e0.record(stream)
            run.advance(chunk, chunk=chunk)  # grows the capacities if a step overflows them
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3 / chunk)
            rows.append(run.history())
        hist = np.concatenate(rows)
        run.close()
        sh = A.blocked_mean(hist["shift"])
        e = A.ratio_estimate(hist["hproj"], hist["vproj"])
        t_med = float(np.median(times))
        ex = hist["exact_steps"].astype(float)
        tot = ex + hist["inexact_steps"].astype(float)
        return {"compression": "early" if compression else "late", "t_rel": t_rel,
                "target": target, "steps": int(len(hist)),
                "shift_mean": sh["mean"], "shift_err": sh["err"],
                "projected": e["ratio"], "projected_err": e["err"],
                "t_step_us": 1e6 * t_med,
                "f_shift": 1.0 / (sh["err"] ** 2 * len(hist) * t_med) if sh["err"] > 0 else None,
                "len_mean": float(hist["len"].mean()), "spawns_mean": float(hist["n_spawns"].mean()),
                "exact_fraction": float(np.mean(ex / np.maximum(tot, 1.0)))}

    def safe(*a):
        try:
            return one(*a)
        except fq.FqError as e:  # a population that dies or outgrows the device
            return {"compression": "early" if a[5] else "late", "t_rel": a[6], "target": a[4],
                    "error": str(e)}

    for comp in (0, 1):
        for t_rel in (1e-9, 1.0 / 16, 0.25, 1.0, 4.0, 16.0, 64.0, 256.0):
            out["real_space"].append(safe(1, 12, 12, 6.0, 1e4, comp, t_rel))
        for target in (30, 100, 300, 1000, 3000, 10000):
            out["momentum_space"].append(safe(3, 10, 10, 6.0, target, comp, 1.0))
    print(json.dumps({"metric": "statistical efficiency of the shift (compression styles, t_rel)",
                      "compression_sweep": out}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# The step's variants at c2 size (1D M = N = 20, u = 2, FP64, N_t = 1e7 per
# run): what replica overlaps (Sec. 4.3), Gram-Schmidt excited states (Sec.
# 2.2) and early compression (Sec. 7.1) cost per step, with the added
# kernels' algorithmic bytes over their added time against the HBM peak

def variants_arm(args):
    import torch

    import paper_2601_19505_gb300 as fq

    cfg = dict(W.CONFIGS["c2"])
    equil, n = 2500, max(50, min(int(args.steps), 1000))
    peak, peak_kind = measured_peak()
    kb, ab, _ = sizes(cfg)
    out = {"workload": describe(cfg, "c2") + " per run", "timed_steps": n,
           "equilibration_steps": equil, "peak_gbs": peak, "peak_source": peak_kind}

    def make(run_id, compression=0, keys=None):
        h = fq.Hamiltonian(cfg["kind"], cfg["Lx"], cfg["Ly"], cfg["N"], cfg["t"], cfg["u"])
        p = fq.default_params(mode=MODE_CODE["REAL64"], dt=cfg["dt"], target=cfg["target"],
                              seed=cfg["seed"], run_id=run_id, compression=compression)
        r = fq.Run(h, p)
        if keys is None:
            r.seed_default(W.START_WEIGHT)
        else:
            r.seed(fq.keys_from_ints(keys), [W.START_WEIGHT] * len(keys), h.column(keys[0])[0], 0)
        return h, r

    def per_step(step, stream_handle):
        stream = torch.cuda.ExternalStream(stream_handle) if stream_handle \
            else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    # replicas: two runs of one seed (run ids 0 and 1), overlaps off, dot
    # products only, and dot products with G2(d), d = 0..3
    (h0, r0), (h1, r1) = make(0), make(1)
    b = fq.Batch([r0, r1])
    b.step(equil)
    b.sync()
    b.autotune(2)
    t_base = per_step(b.step, r0.stream)
    b.set_overlaps([])
    t_dot = per_step(b.step, r0.stream)
    b.set_overlaps([0, 1, 2, 3])
    t_g2 = per_step(b.step, r0.stream)
    b.sync()
    L = float(r0.stats()["len"] + r1.stats()["len"])
    byt = L * (kb + ab)  # both vectors read once per step
    out["replicas"] = {
        "ms_per_step_two_runs": t_base, "ms_per_step_with_dots": t_dot,
        "ms_per_step_with_dots_and_g2_d0_3": t_g2, "len_both_runs": L,
        "overlap_bytes_per_step": byt,
        "overlap_gbs_dots": byt / ((t_dot - t_base) * 1e-3) / 1e9 if t_dot > t_base else None,
        "overlap_gbs_g2": byt / ((t_g2 - t_base) * 1e-3) / 1e9 if t_g2 > t_base else None}
    b.close()
    for r in (r0, r1):
        r.close()
    release_device_memory()

    # excited states: state 1 also starts on a neighbour of the start address
    h0, r0 = make(0)
    start = int(fq.keys_to_ints(r0.export()[0])[0])
    nb = h0.column(start)[1][0]
    _, r1 = make(0, keys=[start, nb])
    b = fq.Batch([r0, r1])
    b.set_spectral(2)
    b.step(equil)
    b.sync()
    t_gs = per_step(b.step, r0.stream)
    b.sync()
    L0, L1 = float(r0.stats()["len"]), float(r1.stats()["len"])
    b.set_spectral(0)
    t_plain = per_step(b.step, r0.stream)
    b.sync()
    # dots read both vectors, the update reads both and writes state 1 again
    gbyt = (2.0 * (L0 + L1) + L1) * (kb + ab)
    out["spectral_K2"] = {
        "ms_per_step_two_runs": t_plain, "ms_per_step_with_gram_schmidt": t_gs,
        "len_states": [L0, L1], "gram_schmidt_bytes_per_step": gbyt,
        "gram_schmidt_gbs": gbyt / ((t_gs - t_plain) * 1e-3) / 1e9 if t_gs > t_plain else None}
    b.close()
    for r in (r0, r1):
        r.close()
    release_device_memory()

    # early against late compression: one run each, kernel by kernel
    for comp, name in ((0, "late"), (1, "early")):
        _, r = make(0, compression=comp)
        r.advance(equil, chunk=equil)
        r.history()
        ms = r.profile(n)
        hist = r.history()
        out["compression_" + name] = {
            "kernel_ms": {"spawn": ms[0], "merge": ms[1], "shift": ms[2]},
            "ms_per_step": sum(ms), "len_mean": float(hist["len"].mean()),
            "spawns_mean": float(hist["n_spawns"].mean()),
            "configs_per_s": float(hist["len"].mean()) / (sum(ms) * 1e-3)}
        r.close()
        release_device_memory()
    print(json.dumps({"metric": METRIC + " (step variants at c2 size)", "variants": out}),
          flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--config", choices=sorted(W.CONFIGS), default="c5")
    ap.add_argument("--equil", type=int, default=None)
    ap.add_argument("--target", type=float, default=None,
                    help="override the workload's N_t (reduced cases for profiling)")
    ap.add_argument("--capacity-vec", type=float, default=0,
                    help="vector capacity in entries (0: derived from N_t)")
    ap.add_argument("--capacity-spawn", type=float, default=0,
                    help="spawn capacity per step in entries (0: derived from N_t)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--annihilation", choices=sorted(ANN_CODE), default="auto",
                    help="annihilation arm (auto: the autotuner times hash and sort)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-more", action="store_true",
                    help="measure only the chosen workload (no nested c5-FP32, c2 and c4 lines)")
    ap.add_argument("--equal-error", action="store_true",
                    help="only the c4 comparison: 64 runs as one FP32 batch, as one FP64 batch "
                         "and one after another in FP64, at equal projected-energy error")
    ap.add_argument("--c3-precision", action="store_true",
                    help="c3: FP32 against FP64 amplitudes where the population first "
                         "reaches its target")
    ap.add_argument("--c3-trajectory", action="store_true",
                    help="c3: FP32 against FP64 trajectories over 5000 steps at N_t = 1e6 and "
                         "1e7, and the first --steps steps at the configuration's N_t")
    ap.add_argument("--compression-sweep", action="store_true",
                    help="late against early compression and the semistochastic threshold: "
                         "statistical efficiency of the shift on 12/12 real space and 10/10 "
                         "momentum space")
    ap.add_argument("--variants", action="store_true",
                    help="cost per step of replica overlaps, Gram-Schmidt excited states and "
                         "early compression at c2 size")
    ap.add_argument("--sweep-steps", type=int, default=100000,
                    help="timed steps per run of --compression-sweep")
    ap.add_argument("--mode", choices=sorted(MODE_CODE), default=None,
                    help="the amplitude mode (default: FP64 for the c5 headline, else the "
                         "workload's own)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    cfg = dict(W.CONFIGS[args.config])
    headline = args.config == "c5" and args.mode is None
    if headline:
        cfg["mode"] = "REAL64"  # the paper's arithmetic; c5 as configured is nested below
    elif args.mode:
        cfg["mode"] = args.mode
    if args.target or args.capacity_vec or args.capacity_spawn:
        headline = False
    if args.target:
        cfg["target"] = args.target
    if args.impl == "reference":
        return reference_arm(args, cfg, args.config)
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.equal_error:
        line = {"metric": METRIC + " (batched FP32 vs sequential FP64 at equal error)",
                "equal_error": equal_error_arm(args)}
        print(json.dumps(line), flush=True)
        return 0
    if args.c3_precision:
        return c3_precision_arm(args)
    if args.c3_trajectory:
        return c3_trajectory_arm(args)
    if args.compression_sweep:
        return compression_sweep_arm(args)
    if args.variants:
        return variants_arm(args)
    dist = Dist(world, "nccl")
    out = gpu_arm(args, cfg, args.config, dist)
    if out is not None and world == 1 and headline and not args.no_more:
        more = {}
        c5 = dict(W.CONFIGS["c5"])
        more["c5_as_configured_fp32"] = brief(gpu_arm(args, c5, "c5", dist, with_cpu=False))
        more["c2"] = brief(gpu_arm(args, dict(W.CONFIGS["c2"]), "c2", dist, with_cpu=False))
        more["c4_equal_error"] = equal_error_arm(args)
        out["more"] = more
    if out is not None:
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
