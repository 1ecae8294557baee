#!/usr/bin/env python3
"""Benchmark of one Blahut-Arimoto iteration on BDC_d at n = 24.

Metric: W(y|x) pair-evaluations per second (effective: the 2*3^n - 2^n
(input, distinct output) pairs an iteration covers, divided by the time of
one iteration) and milliseconds per BA iteration.  A step is one full BA
iteration (output marginal, log, divergence, bounds, update) of the n=24,
d=0.5 instance in FP32 on the factorised sweep, with every input resident in
HBM; the FP64 sweep, the FP64 literal enumeration (the plain FP64 GPU form),
the FP64 certificate and the d-free precompute are timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs its own instance
(instances are independent: weak scaling, no data-path collective); the
reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "W(y|x) pair-evals/s and s/BA-iteration at n=24, FP32+FP64-certify vs FP64"
UNIT = "pair-evals/s"
N_BITS = int(os.environ.get("BDC_BENCH_N", "24"))
D_VALUE = 0.5


def pairs_per_iteration(n: int) -> int:
    """(input, distinct output) pairs one BA iteration covers: sum_x N_x = 2*3^n - 2^n."""
    return 2 * 3 ** n - 2 ** n


def stage_bytes(n: int, n1: int, n2: int, elem: int, half: bool) -> dict:
    """Algorithmic HBM bytes of each sweep stage (unique values each launch must
    read or write once, all instances of the step).  In the complement half mode
    every sweep launch touches half of the values (the other half are their
    complements), so its bytes are halved."""
    N = (1 << n) // (2 if half else 1)
    split = n2 > 0
    return {
        # p and Dbar in, updated p and F1 (rows below 2^n1) out
        "cols_fwd": (4 if split else 3) * N * elem + (0 if split else 4 * N * elem),
        # every row (F1 or p) in, bottom half of every row out
        "rows_fwd": 4 * N * elem,
        # every (u1, u2) pair in once, the F1/p terms, log2 q of the H1 codes out
        # (an iteration does not store q)
        "combine": 5 * N * elem,
        # log2 q in (its re-reads are L2 hits), Gb out
        "rows_adj": 4 * N * elem,
        # Gb, Hb, p in, D out (single pass: L, Hb, p in, D out)
        "cols_adj": 5 * N * elem,
        # the iteration boundary in one pass: Gb (every row), Hb, p in; updated p
        # and the next iteration's F1 out (D is not stored)
        "cols_step": 6 * N * elem,
        "symmetrize": 2 * N * elem,  # reads and writes the stored half
        "finalize": 0,
    }


# ncu counters of the FP32 iteration kernels (DRAM bytes read + written and
# shared-memory wavefronts per launch), one capture of this bench's own
# workload, summarised in a JSON file beside the text summaries of the same
# captures.  The file records a hash of the kernel source it was taken from;
# once that source changes the counters no longer describe the kernels and
# are reported as null.
COUNTERS = os.path.join(ROOT, "profiles", "ncu_counters_n24.json")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2604_05867_b300", "csrc", "sweep.cu")


def kernel_source_hash() -> str:
    import hashlib
    with open(KERNEL_SOURCE, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_counters(stage: str, n: int, sched: dict):
    """(counters, source) of one launch of `stage`: the capture's record
    (dram_bytes, smem_wavefronts, lsu_wavefronts, ...), or ({}, why) when no
    capture of the current kernels exists."""
    try:
        with open(COUNTERS) as f:
            j = json.load(f)
    except Exception:
        return {}, "no counter file"
    if j.get("source_sha") != kernel_source_hash():
        return {}, "kernels changed since the capture"
    for r in j.get("launches", []):
        if (r["stage"], r["n"], r["n1"], r["n2"], r["width"]) == (stage, n, sched["n1"], sched["n2"], sched["width"]):
            return r, j.get("command", "")
    return {}, "no capture of this schedule"


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--id=" + self.gpu_id, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [s.strip() for s in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return {"hbm_gbs": float(j["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "source": "fallback"}


# ----------------------------------------------------------------------------
# oracle timing (host cores) -- the CPU baseline and the reference arm
# ----------------------------------------------------------------------------
def oracle_rate(n: int, d: float, seconds: float, seed: int = 0, threads: int = 0):
    """Time the FP64 oracle's divergence walk (the definition: every (x,
    distinct y) pair) on random inputs of length n until about `seconds` of
    work; returns (pair-evals/s for a full iteration, threads, sample
    description, seconds).  A BA iteration of the oracle walks every pair
    twice (output marginal, then divergence) at the same cost per pair, so
    the full-iteration rate is half the walk rate.  The pairs are counted
    outside the timed calls."""
    import oracle
    from paper_2604_05867_b300 import inputs

    used = oracle.set_threads(threads if threads > 0 else (len(os.sched_getaffinity(0))
                                                            if hasattr(os, "sched_getaffinity") else os.cpu_count()))
    q = np.ones(2 << n)  # any positive q: the walk's cost does not depend on its values
    q[0] = 0.0
    size, total_pairs, total_t, total_x = 32, 0, 0.0, 0
    it = 0
    while total_t < seconds:
        xs = inputs.random_inputs(n, size, seed=seed + it).astype(np.uint64)
        t0 = time.perf_counter()
        oracle.D_list(n, d, q, xs)
        dt = time.perf_counter() - t0
        total_pairs += oracle.pairs_list(n, xs)
        total_t += dt
        total_x += size
        it += 1
        if dt < seconds / 8:
            size *= 2
    rate = total_pairs / total_t / 2.0
    sample = ("divergence walk of the FP64 oracle on %d thread(s) over %d random inputs of length %d, %d pairs in "
              "%.1f s, extrapolated to a full iteration (2 (2*3^n - 2^n) pairs: marginal + divergence passes)"
              % (used, total_x, n, total_pairs, total_t))
    return rate, used, sample, total_t


def oracle_sweep_rate(n: int, d: float, iters: int = 1):
    """The oracle's factorised sweep (O2, same algorithm as the GPU path, plain
    FP64 C with OpenMP) timed over `iters` full BA iterations at length n on
    all host cores: output marginal, log2, transposed sweep, D, bounds, update.
    The d-free entropy table S it reads is zero-filled here (its values do not
    change the time; computing it is the once-per-n precompute, timed apart on
    the GPU).  Returns (effective pair-evals/s, ms per iteration, threads)."""
    import oracle
    used = oracle.set_threads(len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    S = np.zeros((1 << n, n + 1))
    p = np.full(1 << n, 1.0 / (1 << n))
    t0 = time.perf_counter()
    oracle.ba_sweep(n, d, iters, p0=p, S=S)
    dt = (time.perf_counter() - t0) / iters
    return pairs_per_iteration(n) / dt, 1000.0 * dt, used


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    n = N_BITS
    per_step = []
    rates = []
    cores = None
    for s in range(args.warmup + args.steps):
        budget = 0.5 if s < args.warmup else max(0.5, min(3.0, 150.0 / max(1, args.steps)))
        r, cores, sample, t = oracle_rate(n, D_VALUE, budget, seed=1000 * s)
        if s >= args.warmup:
            rates.append(r)
            per_step.append(pairs_per_iteration(n) / r)
    value = float(statistics.median(rates))
    ms = 1000.0 * pairs_per_iteration(n) / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "BA iteration on BDC_d, n=24, d=0.5 (all 2^24 inputs); each step times the FP64 "
                               "oracle's divergence walk on a random sample of inputs and extrapolates it to the "
                               "full iteration", "n": n, "d": [D_VALUE], "extrapolated": True,
                   "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: " + sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, rank: int, world: int):
    import torch
    import torch.distributed as dist

    import paper_2604_05867_b300 as bdc
    from paper_2604_05867_b300 import shard

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    n = N_BITS
    # weak scaling: one n = 24 instance per rank (the instances are independent)
    (d,) = shard.shard([D_VALUE] * world, rank, world)

    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        # iterations per graph replay: the largest divisor of the timed step
        # count up to 64, so the timed region is whole graph replays
        chunk = max(c for c in range(1, 65) if args.steps % c == 0)
        eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=1, chunk=chunk), stream=stream)
        a0_s = time.perf_counter() - t0
        # pick the sweep schedules for this GPU (part of the setup, not of a step)
        if args.sched_fp32:
            n2s, ws = (int(v) for v in args.sched_fp32.split(","))
            sched32 = dict(eng.set_schedule("fp32", n2s, ws), forced=True)
        else:
            sched32 = eng.autotune("fp32", reps=3, cache=args.sched_cache)
        sched64 = eng.autotune("fp64", reps=2, cache=args.sched_cache)

        # warm-up: W untimed FP32 iterations; the CUDA graph the timed call
        # replays is captured and instantiated here too (setup, not a step)
        eng.iterate(args.warmup, -1.0, "fp32", "sweep")
        eng.prepare("fp32", "sweep")
        torch.cuda.synchronize()

        props = torch.cuda.get_device_properties(dev)
        gpu_id = getattr(props, "pci_bus_id", None)
        gpu_id = str(gpu_id) if gpu_id else str(local)
        clocks = ClockSampler(gpu_id)
        clocks.start()
        # keep the GPU under load (untimed iterations) while the sampler starts:
        # after half a second idle the first kernels run measurably slower (the
        # forward rows pass by up to 20% for a while), and on a GPU fresh to this
        # process half a second of load still left the timed steps 2% slower
        # than two seconds do, so the timed steps follow two seconds of load;
        # then the W warm-up steps again
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 2.0:
            eng.iterate(chunk, -1.0, "fp32", "sweep")
            torch.cuda.synchronize()
        eng.iterate(args.warmup, -1.0, "fp32", "sweep")
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = eng.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lo, up, it = eng.iterate(args.steps, -1.0, "fp32", "sweep")
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms_total = ev0.elapsed_time(ev1)
        launches = eng.launch_count() - launches0
        # per-stage times (events after every kernel, no graph), same workload,
        # taken straight after the timed steps while the GPU is still under load
        stages = eng.profile("fp32", "sweep", reps=5) if rank == 0 else None
        clk = clocks.stop()
        ms = shard.max_over_ranks(ms_total / args.steps, device=dev)  # slowest rank's time per step
        # every rank iterates its own instance: the job covers `world` instances per step
        value = pairs_per_iteration(n) * world / (ms / 1000.0)

        extra = {}
        if rank == 0:
            half = sched32["n2"] > 0 and sched32["width"] < (1 << sched32["n2"])
            sb = stage_bytes(n, sched32["n1"], sched32["n2"], 4, half)
            peaks = measured_peaks()
            dev_peaks = bdc.measure_peaks(stream)
            top = max((k for k in stages if k in sb and sb[k] > 0), key=lambda k: stages[k])
            achieved = sb[top] / (stages[top] / 1000.0) / 1e9
            cnt, csrc = measured_counters(top, n, sched32)
            dram, wf, lsu = cnt.get("dram_bytes"), cnt.get("smem_wavefronts"), cnt.get("lsu_wavefronts")
            roof = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": dram,
                    "peak_source": peaks["source"], "algorithmic_bytes": sb[top],
                    "traffic_source": csrc, "note": "complement half mode: %s" % half}
            if wf is not None:
                # the kernel's binding on-chip resource: shared-memory bandwidth,
                # against the peak measured in this run (bdc_measure_peaks)
                smem_tb = wf * 128 / (stages[top] / 1000.0) / 1e12
                roof["shared_memory"] = {"bytes_per_launch": wf * 128, "achieved": smem_tb,
                                         "peak": dev_peaks["smem_tbs"], "unit": "TB/s",
                                         "frac": smem_tb / dev_peaks["smem_tbs"],
                                         "source": "ncu shared-memory wavefronts of one launch x 128 B / this run's "
                                                   "event time; peak measured in this run"}
            if lsu is not None and clk.get("sm_mhz"):
                # the L1 data pipe that serves both the shared-memory steps and
                # the 16-byte global accesses of 4-column tile rows: one
                # wavefront per cycle per SM at the SM clock sampled in this run
                lsu_rate = lsu / (stages[top] / 1000.0) / 1e9
                lsu_peak = dev_peaks["sms"] * clk["sm_mhz"] / 1e3
                roof["l1_data_pipe"] = {"wavefronts_per_launch": lsu, "shared_wavefronts": wf,
                                        "achieved": lsu_rate, "peak": lsu_peak, "unit": "G wavefronts/s",
                                        "frac": lsu_rate / lsu_peak,
                                        "source": "ncu l1tex__data_pipe_lsu_wavefronts.sum of one launch / this "
                                                  "run's event time; peak 1 wavefront/cycle/SM x SMs x sampled SM clock"}
            stage_total = sum(stages.values())

            # FP64 sweep iteration (same-algorithm precision baseline)
            eng.iterate(2, -1.0, "fp64", "sweep")
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eng.iterate(5, -1.0, "fp64", "sweep")
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1) / 5
            # its additions against the FP64 pipe measured in this run: one
            # forward step adds two terms and one adjoint step one, per element,
            # over the columns (2^(n1+1) x 2^n2 elements, n1 steps) and rows
            # (2^(n1+1) x 2^(n2+1), n2 steps) passes; halved in half mode
            half64 = sched64["n2"] > 0 and sched64["width"] < (1 << sched64["n2"])
            el_steps = (2 << n) * sched64["n1"] + (4 << n) * sched64["n2"]
            adds64 = 3 * el_steps // (2 if half64 else 1)
            fp64_rate = adds64 / (ms64 / 1000.0) / 1e12

            # FP64 certificate of the current p
            e0.record(stream)
            cert = eng.certify()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_cert = e0.elapsed_time(e1)

            # plain FP64 GPU form: literal enumeration (orbit representatives)
            ms_lit = None
            if not args.skip_literal:
                e0.record(stream)
                eng.iterate(1, -1.0, "fp64", "literal")
                e1.record(stream)
                torch.cuda.synchronize()
                ms_lit = e0.elapsed_time(e1)
            eng.iterate(1, -1.0, "fp32", "sweep")  # back to the FP32 representation

            # batched form at the same n: four d values in one engine (every launch
            # covers all instances; the d-free precompute is shared)
            ms_batch = None
            if not args.skip_batched:
                beng = bdc.Engine(n, [0.2, 0.4, 0.6, 0.8], options=bdc.default_options(enable_literal=0, chunk=8),
                                  stream=stream)
                beng.autotune("fp32", reps=3, cache=args.sched_cache)
                beng.iterate(args.warmup, -1.0, "fp32", "sweep")
                beng.prepare("fp32", "sweep")
                torch.cuda.synchronize()
                e0.record(stream)
                beng.iterate(40, -1.0, "fp32", "sweep")
                e1.record(stream)
                torch.cuda.synchronize()
                ms_batch = e0.elapsed_time(e1) / 40
                beng.close()
                del beng
                torch.cuda.empty_cache()

            # end to end through the public API, as a user job: the input
            # distribution comes from pinned host memory (bdc_set_p: host->device
            # copy and the device checks), K FP32 BA iterations (bdc_ba_iterate),
            # the per-iteration bounds back to the host (bdc_get_history) and the
            # FP64 certificate of the result (bdc_certify_upper, host outputs);
            # per step = the job's wall time / K, bytes per step likewise
            K = args.steps
            p0 = torch.full((1, 1 << n), 1.0 / (1 << n), dtype=torch.float64).pin_memory().numpy()
            eng.set_p(p0)
            eng.prepare("fp32", "sweep")  # (setup: the replayed graphs exist before the job)
            eng.iterate(K, -1.0, "fp32", "sweep")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            eng.set_p(p0)
            eng.iterate(K, -1.0, "fp32", "sweep")
            hist = eng.history(0, K)
            cert_e2e = eng.certify()
            e2e_s = (time.perf_counter() - t0) / K
            assert len(hist[0]) == K and np.isfinite(cert_e2e["upper"][0])
            extra = {
                "roofline": roof,
                "stages_ms": stages,
                "stage_sum_ms": stage_total,
                "forms": {
                    "fp32_sweep_ms_per_iter": ms,
                    "fp64_sweep_ms_per_iter": ms64,
                    "fp64_literal_ms_per_iter": ms_lit,
                    "fp64_certify_ms": ms_cert,
                    "precompute_a0_s": a0_s,
                    "batched_4d_ms_per_iter_all": ms_batch,
                    "batched_4d_pair_evals_per_s": (4 * pairs_per_iteration(n) / (ms_batch / 1000.0)) if ms_batch else None,
                    "fp64_sweep_adds_per_s_1e12": fp64_rate,
                    "fp64_sweep_frac_of_measured_fp64_pipe": fp64_rate / dev_peaks["fp64_tops"],
                    "speedup_fp32_vs_fp64_sweep": ms64 / ms,
                    "speedup_fp32_sweep_vs_fp64_literal": (ms_lit / ms) if ms_lit else None,
                    "speedup_fp64_sweep_vs_fp64_literal": (ms_lit / ms64) if ms_lit else None,
                    "certified_upper_over_n": float(cert["upper"][0]) / n,
                    "certify_margin_bits": float(cert["margin"][0]),
                    "lower_after_run": float(lo[0]), "upper_after_run": float(up[0]),
                },
                "e2e": {"value": pairs_per_iteration(n) / e2e_s, "unit": UNIT,
                        "h2d_bytes_per_step": (8 << n) / K, "d2h_bytes_per_step": 16.0 + 24.0 / K,
                        "ms_per_step": e2e_s * 1000.0, "steps": K,
                        "call": "one job per K steps: Engine.set_p(pinned host p0) -> bdc_set_p; "
                                "Engine.iterate(K) -> bdc_ba_iterate; Engine.history -> bdc_get_history; "
                                "Engine.certify -> bdc_certify_upper; wall time / K"},
                "device_peaks": dict(dev_peaks, source="bdc_measure_peaks in this run"),
            }
            if world == 1 and not args.skip_cpu:
                rate, cores, sample, _ = oracle_rate(n, d, args.cpu_seconds)
                extra["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                         "sample": sample}
                r1, _, sample1, _ = oracle_rate(n, d, args.cpu_seconds / 3, threads=1)
                extra["cpu_baseline_single_thread"] = {"value": r1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                                       "sample": sample1}
                r2, ms2, c2 = oracle_sweep_rate(n, d, 1)
                extra["cpu_baseline_same_algorithm"] = {
                    "value": r2, "unit": UNIT, "cores": c2, "kind": "oracle (factorised sweep, O2)",
                    "ms_per_iteration": ms2,
                    "sample": "one full FP64 BA iteration at n=%d on the oracle's factorised sweep; effective "
                              "pair-evals/s = (2*3^n - 2^n) / its time" % n}
        eng.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "BA iteration on BDC_d, n=24, d=0.5 (all 2^24 inputs), FP32 factorised sweep",
                       "n": n, "d": [d], "instances_per_gpu": 1, "parallelism": "instance-parallel",
                       "l2": "inputs larger than L2 (per-iteration working set ~0.8 GB vs 126 MB L2)",
                       "step": "one BA iteration: q sweep, log2, adjoint sweep, D, bounds, orbit mean, p update",
                       "schedule_fp32": sched32, "schedule_fp64": sched64},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the configurations of the workload, each run end to end (one JSON line each)
# ----------------------------------------------------------------------------
def _sync_time(fn, stream):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def run_config(args):
    import torch

    import paper_2604_05867_b300 as bdc
    from paper_2604_05867_b300 import dual, inputs, shard

    # under torchrun the instance grids of the batched and large configurations
    # are split over the ranks (one GPU each; instances are independent, so no
    # data-path collective), results gathered on rank 0, time = max over ranks
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rank, world = shard.init_from_env("nccl")
    stream = torch.cuda.Stream()
    res = {"config_run": args.config, "ranks": world}
    with torch.cuda.stream(stream):
        if rank != 0 and args.config not in ("batched", "large"):
            pass  # single-GPU configurations run on rank 0 alone
        elif args.config == "ba10":
            # plain FP64 BA at n=10, d=0.5: gap < 1e-9 or 2000 iterations; against the
            # oracle's BA on the channel built from all 2^10 deletion patterns
            import oracle
            n, d, T, tol = 10, 0.5, 2000, 1e-9
            t0 = time.perf_counter()
            ref = oracle.ba_bdc(n, d, T, tol=tol)
            t_or = time.perf_counter() - t0
            for impl in ("sweep", "literal"):
                eng = bdc.Engine(n, [d], stream=stream)
                (lo, up, it), t = _sync_time(lambda: eng.iterate(T, tol, "fp64", impl), stream)
                hlo, hup = eng.history(0)
                m = min(len(hlo), len(ref["lower"]))
                c = eng.certify()
                res["gpu_" + impl] = {"iters": int(it[0]), "lower": float(lo[0]), "upper": float(up[0]),
                                      "ms_per_iter": 1000 * t / max(1, it[0]),
                                      "max_abs_diff_lower_vs_oracle": float(np.max(np.abs(hlo[:m] - ref["lower"][:m]))),
                                      "max_abs_diff_upper_vs_oracle": float(np.max(np.abs(hup[:m] - ref["upper"][:m]))),
                                      "certified_upper": float(c["upper"][0]), "margin": float(c["margin"][0])}
                eng.close()
            res["oracle"] = {"iters": int(ref["iters"]), "lower": float(ref["lower"][-1]),
                             "upper": float(ref["upper"][-1]), "ms_per_iter": 1000 * t_or / ref["iters"]}
        elif args.config == "n20":
            # n=20, d=0.7: 500 FP32 iterations, FP64 certificate of C_20/20
            import oracle
            n, d, T = 20, 0.7, 500
            eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0), stream=stream)
            eng.autotune("fp32")
            (lo, up, it), t = _sync_time(lambda: eng.iterate(T, -1.0, "fp32", "sweep"), stream)
            c, tc = _sync_time(lambda: eng.certify(), stream)
            res.update({"n": n, "d": d, "iters": T, "ms_per_iter": 1000 * t / T, "lower": float(lo[0]),
                        "upper": float(up[0]), "certified_upper": float(c["upper"][0]),
                        "certified_upper_over_n": float(c["upper"][0]) / n, "margin": float(c["margin"][0]),
                        "certify_ms": 1000 * tc, "pairs_per_s_effective": pairs_per_iteration(n) * T / t})
            if args.oracle_check:
                # the oracle's dual value of the same certified input: q by the
                # oracle's factorised sweep (pinned against its q_full), then
                # max_x D_x from the definition (certify)
                p = eng.get_p()[0]
                eps = 2.0 ** -30
                t0 = time.perf_counter()
                q = oracle.sweep_q(n, d, (1 - eps) * p + eps / (1 << n))
                U, _ = oracle.certify(n, d, q)
                res["oracle_certify"] = {"U": U, "diff": float(c["upper"][0]) - U, "seconds": time.perf_counter() - t0}
            eng.close()
        elif args.config == "batched":
            # n=22 with 32 d in [0.05, 0.95] and n in {14,16,18,20} with 8 d each, one graph per rank
            grid = shard.shard_grid(inputs.batched_d_grid(), rank, world)
            T = args.iters or 500
            opts = bdc.default_options(enable_literal=0, chunk=10)
            engs = [bdc.Engine(n, ds, options=opts, stream=stream) for n, ds in grid.items()]
            for e in engs:
                e.autotune("fp32")
            batch = bdc.Batch(engs, chunk=10)
            batch.iterate(10, -1.0, "fp32")
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            ran, t = _sync_time(lambda: batch.iterate(T, -1.0, "fp32"), stream)
            t = shard.max_over_ranks(t, device=torch.device("cuda", local))
            pairs = sum(pairs_per_iteration(e.n) * e.nd for e in engs)
            certs, tc = _sync_time(lambda: [e.certify() for e in engs], stream)
            mine = {"pairs": pairs, "instances": sum(e.nd for e in engs), "iters": ran,
                    "certified_upper_over_n": {str(e.n): [round(float(u) / e.n, 8) for u in c["upper"]]
                                               for e, c in zip(engs, certs)},
                    "d": {str(e.n): e.ds for e in engs},
                    "max_margin": max(float(np.max(c["margin"])) for c in certs), "certify_seconds": tc}
            parts = shard.gather_to_rank0(mine)
            if rank == 0:
                tot_pairs = sum(m["pairs"] for m in parts)
                res.update({"instances": sum(m["instances"] for m in parts), "iters": ran, "seconds": t,
                            "ms_per_iter_all_instances": 1000 * t / ran,
                            "pairs_per_s_effective": tot_pairs * ran / t,
                            "certify_seconds_max_rank": max(m["certify_seconds"] for m in parts),
                            "per_rank": [{"d": m["d"], "certified_upper_over_n": m["certified_upper_over_n"]}
                                         for m in parts],
                            "max_margin": max(m["max_margin"] for m in parts)})
            batch.close()
            for e in engs:
                e.close()
        elif args.config == "dual":
            # n=22, d=0.8: 50 BA iterations -> theta; tau=1e-3; FD (h=1e-6, FP64) on 64
            # random coordinates; 200 Adam steps; FP64 certified max_x D_x
            n, d, tau, h = 22, 0.8, 1e-3, 1e-6
            eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0), stream=stream)
            eng.iterate(50, -1.0, "fp32", "sweep")
            theta0 = dual.theta_from_q(eng, eng.get_q("fp64")[0])
            th = torch.tensor(theta0, dtype=torch.float64, device="cuda")
            (F, mD, g, gd), tg = _sync_time(lambda: eng.dual_bound(0, th, tau, "fp64", grad=True), stream)
            g = g.cpu().numpy()
            errs, aerrs, top_errs = [], [], []
            gscale = float(np.max(np.abs(g)))

            def fd_at(i):
                tp, tm = th.clone(), th.clone()
                tp[i] += h
                tm[i] -= h
                return (eng.dual_bound(0, tp, tau, "fp64", grad=False)[0] -
                        eng.dual_bound(0, tm, tau, "fp64", grad=False)[0]) / (2 * h)

            # 64 seeded random coordinates: absolute error (most of them carry
            # gradients far below the central difference's rounding noise,
            # ~eps |F| / h = 1e-9)
            for i in inputs.fd_coordinates(len(theta0), 64, seed=0):
                aerrs.append(abs(fd_at(int(i)) - g[i]))
            # relative error on 64 seeded coordinates drawn from the significant
            # ones (|g| >= 1e-3 of the largest), and on the 8 largest
            sig = np.flatnonzero(np.abs(g) >= 1e-3 * gscale)
            for i in sig[inputs.fd_coordinates(len(sig), 64, seed=1)]:
                errs.append(abs(fd_at(int(i)) - g[i]) / abs(g[i]))
            for i in np.argsort(-np.abs(g))[:8]:
                top_errs.append(abs(fd_at(int(i)) - g[i]) / abs(g[i]))
            # dF/dd at fixed theta by central differences over two more engines
            fdd = []
            for dd in (d + h, d - h):
                e2 = bdc.Engine(n, [dd], options=bdc.default_options(enable_literal=0), stream=stream)
                fdd.append(e2.dual_bound(0, th, tau, "fp64", grad=False)[0])
                e2.close()
            fd_d = (fdd[0] - fdd[1]) / (2 * h)
            out, t = _sync_time(lambda: dual.optimize_dual(eng, 0, tau=tau, steps=200, lr=1e-2, ba_iters=0,
                                                           precision="fp32", theta0=theta0), stream)
            res.update({"n": n, "d": d, "tau": tau, "F": F, "max_D": mD, "dF_dd": gd,
                        "value_and_grad_ms_fp64": 1000 * tg, "fd_coords": len(aerrs), "fd_rel_coords": len(errs),
                        "fd_significant_coords": int(len(sig)), "dF_dd_central_difference": fd_d,
                        "dF_dd_rel_err": abs(fd_d - gd) / max(abs(gd), 1e-300),
                        "fd_max_rel_err": float(np.max(errs)) if errs else None,
                        "fd_max_abs_err": float(np.max(aerrs)), "grad_max_abs": gscale,
                        "fd_top8_max_rel_err": float(np.max(top_errs)),
                        "ba_lower_after_50": float(eng.history(0)[0][-1]),
                        "adam_steps": 200, "adam_seconds": t,
                        "certified_initial": out["certified_initial"], "certified_final": out["certified_final"],
                        "certified_final_over_n": out["certified_final"] / n, "margin": out["margin"]})
            eng.close()
        elif args.config == "large":
            # n=26, 7 values of d, 300 FP32 iterations each, FP64 certificate of C_26(d)/(26(1-d))
            from paper_2604_05867_b300.inputs import LARGE_SWEEP_D
            n, T = args.n or 26, args.iters or 300
            dlist = list(LARGE_SWEEP_D)[:args.nd] if args.nd else list(LARGE_SWEEP_D)
            ds = shard.shard_grid({n: dlist}, rank, world).get(n, [])
            mine = {"d": ds}
            if ds:
                t0 = time.perf_counter()
                eng = bdc.Engine(n, ds, options=bdc.default_options(enable_literal=0), stream=stream)
                t_bind = time.perf_counter() - t0
                eng.autotune("fp32")
                torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            if ds:
                (lo, up, it), t = _sync_time(lambda: eng.iterate(T, -1.0, "fp32", "sweep"), stream)
                c, tc = _sync_time(lambda: eng.certify(), stream)
                mine.update({"bind_precompute_s": t_bind, "seconds": t, "certify_seconds": tc,
                             "workspace_gb": eng.ws_bytes / 1e9,
                             "certified_upper": [float(u) for u in c["upper"]],
                             "certified_over_n_1_minus_d": [float(u) / (n * (1 - dv)) for u, dv in zip(c["upper"], ds)],
                             "margin_max": float(np.max(c["margin"])),
                             "lower_last": [float(v) for v in lo], "upper_last": [float(v) for v in up]})
                eng.close()
            else:
                mine["seconds"] = 0.0
            t = shard.max_over_ranks(mine["seconds"], device=torch.device("cuda", local))
            parts = shard.gather_to_rank0(mine)
            if rank == 0:
                alld = [d_ for m in parts for d_ in m["d"]]
                res.update({"n": n, "d": alld, "iters": T, "seconds": t, "ms_per_iter_all_instances": 1000 * t / T,
                            "pairs_per_s_effective": pairs_per_iteration(n) * len(alld) * T / t,
                            "per_rank": parts})
        elif args.config == "literal":
            # the plain FP64 GPU form on its own: literal enumeration iterations
            # (supersequence walk for q, subsequence walk for D, on orbit
            # representatives); a small case for profiling its kernels
            n, d, T = args.n or 20, 0.5, args.iters or 2
            eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=1), stream=stream)
            eng.iterate(1, -1.0, "fp64", "literal")
            (lo, up, it), t = _sync_time(lambda: eng.iterate(T, -1.0, "fp64", "literal"), stream)
            from math import comb
            # leaves of the supersequence walk: every output class of length k
            # has sum_{i <= n-k} C(n, i) supersequences (Lemma num_superseq)
            rk = [1] + [((1 << k) + (1 << ((k + 1) // 2)) + ((1 << (k // 2)) if k % 2 == 0 else 0)) // 4
                        for k in range(1, n + 1)]
            q_leaves = sum(rk[k] * sum(comb(n, i) for i in range(n - k + 1)) for k in range(n + 1))
            d_nodes = pairs_per_iteration(n) / 4.0  # distinct (rep x, y) pairs, orbit-reduced (up to fixed points)
            res.update({"n": n, "d": d, "iters": T, "ms_per_iter": 1000 * t / T, "lower": float(lo[0]),
                        "upper": float(up[0]), "q_walk_leaves_per_iter": q_leaves,
                        "d_walk_pairs_per_iter_approx": d_nodes,
                        "enumerated_pairs_per_s": (q_leaves + d_nodes) * T / t,
                        "stages_ms": eng.profile("fp64", "literal", reps=1)})
            eng.close()
        elif args.config == "exact":
            # exact deletion channels BDC_{n,k} for every k in one engine of
            # length-mixture instances, certified; then C(d) bounds by Lemma
            # prob-vs-exact on the grid of the paper's C(d) table, the
            # high-noise constant by Lemma convex, and Lemma worse-UB (s = 2)
            # from C_{n-2,k}
            from paper_2604_05867_b300 import bounds
            n, T, tol = args.n or 24, args.iters or 3000, 1e-4
            t0 = time.perf_counter()
            res_k = bounds.exact_capacities(n, list(range(0, n + 1)), iters=T, tol=tol, precision="fp32",
                                            options=bdc.default_options(enable_literal=0), stream=stream)
            t_exact = time.perf_counter() - t0
            Cnk = [res_k[k]["upper"] for k in range(n + 1)]
            grid = [0.01, 0.02, 0.03, 0.04, 0.05, 0.10, 0.15, 0.20, 0.25, 0.30, 0.35, 0.40, 0.45, 0.50, 0.55,
                    0.60, 0.64, 0.65, 0.68]
            cd = bounds.cd_table(grid, {n: Cnk})
            _, ratio = bounds.high_noise(0.64, [v for d_, v, _ in cd if d_ == 0.64][0])
            # Lemma worse-UB from the exact channels of length n - 2 (certified
            # the same way) and C_{2,0..2} = 0, 1, 2
            res_m = bounds.exact_capacities(n - 2, list(range(0, n - 1)), iters=T, tol=tol, precision="fp32",
                                            options=bdc.default_options(enable_literal=0), stream=stream)
            Cm = [res_m[k]["upper"] for k in range(n - 1)]
            split = {k: bounds.split_bound(n, k, 2, [0.0, 1.0, 2.0], Cm) for k in range(n + 1)}
            # the direct BDC_d engine at three d: the lemma's bound is never below
            # its certified lower bound
            direct = {}
            for dv in (0.1, 0.5, 0.64):
                e = bdc.Engine(n, [dv], options=bdc.default_options(enable_literal=0), stream=stream)
                lo, up, it = e.iterate(T, tol, "fp32", "sweep")
                c = e.certify()
                direct[str(dv)] = {"certified_upper_over_n": float(c["upper"][0]) / n,
                                   "lower_over_n": float(c["lower"][0]) / n, "iters": int(it[0]),
                                   "prob_vs_exact_over_n": bounds.prob_vs_exact(n, dv, Cnk) / n}
                e.close()
            res.update({"n": n, "tol_bits": tol, "seconds_all_k": t_exact,
                        "Cnk_certified": {str(k): res_k[k]["upper"] for k in res_k},
                        "Cnk_iters": {str(k): res_k[k]["iters"] for k in res_k},
                        "Cnk_gap": {str(k): res_k[k]["ba_upper"] - res_k[k]["ba_lower"] for k in res_k},
                        "Cnk_table": bounds.ck_table(n, {k: res_k[k]["upper"] for k in range(1, n + 1)}),
                        "worse_ub_from_n_minus_2": {str(k): v for k, v in split.items()},
                        "Cd_table": [{"d": d_, "bound": bounds.ceil4(v), "n": nb} for d_, v, nb in cd],
                        "high_noise_ratio_at_0.64": bounds.ceil4(ratio), "direct_bdc": direct})
        elif args.config == "fp64sweep":
            # FP64 sweep iterations at n = 24 (the same-algorithm precision
            # baseline); a case for profiling the FP64 sweep kernels
            n, d, T = args.n or 24, 0.5, args.iters or 5
            eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0), stream=stream)
            sched = eng.autotune("fp64", reps=2)
            eng.iterate(2, -1.0, "fp64", "sweep")
            (lo, up, it), t = _sync_time(lambda: eng.iterate(T, -1.0, "fp64", "sweep"), stream)
            res.update({"n": n, "d": d, "iters": T, "ms_per_iter": 1000 * t / T, "schedule_fp64": sched,
                        "stages_ms": eng.profile("fp64", "sweep", reps=2),
                        "device_peaks": bdc.measure_peaks(stream)})
            eng.close()
        else:
            raise SystemExit("unknown config " + args.config)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-literal", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--config", default=None,
                    choices=["ba10", "n20", "batched", "dual", "large", "literal", "fp64sweep", "exact"],
                    help="run one workload configuration end to end instead of the headline bench")
    ap.add_argument("--iters", type=int, default=0)
    ap.add_argument("--n", type=int, default=0, help="input length of the literal / fp64sweep / exact / large configs")
    ap.add_argument("--nd", type=int, default=0, help="large config: use the first ND values of its d list")
    ap.add_argument("--sched-fp32", default=None, metavar="N2,W",
                    help="use this FP32 sweep schedule (n2, column width) instead of the autotuner's")
    ap.add_argument("--sched-cache", default=None,
                    help="JSON file of tuned sweep schedules (read if present, written after a search)")
    ap.add_argument("--oracle-check", action="store_true")
    args = ap.parse_args()
    if args.config:
        run_config(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
