#!/usr/bin/env python3
"""Benchmark of the event-based SISe3 simulation on one GB300 (or N, as replicas).

Main line (one "step"): the national-scale SISe3 instance, 37,000 herds x 1,460
days, 3,000,000 scheduled events (exit / enter / aging / external transfer), one
replicate per GPU; the whole horizon is the step (stochastic step, events and phi
update of every day).  Inputs are resident in HBM when the timed region starts; the
L2 cache (129 MB; the state and event schedule fit in it) is flushed between timed
steps by writing a 512 MB buffer.

Legs, each with its correctness check: the plain SISe instance (1,000 nodes x 365
days; bit-exact against the oracle over the whole horizon), the batched national
network (256 replicates x 365 days; a seeded subset of replicates bit-exact against
the oracle), the score-function gradient (10,000 nodes x 4,096 replicates x 365
days; central differences under common random numbers on 1,024 replicates), the
uneven batch (512 instances in one persistent launch against running them one after
another; a seeded subset bit-exact against the oracle), the synthetic benchmark of
Sec. 4.2, the parameter fit of Sec. 4.3 and the general model.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
specification the CUDA path matches bit for bit) on a bounded sample instead.
Multi-GPU (torchrun): replicas only; rank k runs replicate k (its own Philox
stream), no collective on the data path; value = all ranks' node-days / max time.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
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

METRIC = "node-days/sec and SSA events/sec (batched vs plain, bit-exact to oracle)"
# algorithmic HBM bytes of the stochastic step per node-day (counts read and written,
# SISe3 24 + 24 B, SISe 8 + 8 B; phi read and written 8 + 8 B)
SSA_BYTES_PER_NODE_DAY = {3: 64, 1: 32}
# Algorithmic binary64 work of the direct method, counted two ways (FP64 lane-ops):
#  - per draw (Gillespie step, including the one draw per node-day that ends the
#    day): about 40 -- -log(u) 20-25, one IEEE divide 8-10, rates, sums and compares
#    about 6 -- the figure the kernel's roofline uses;
#  - the specification's own operations (R4-R6, R8 of the design record), add/mul = 1
#    and divide = 7 (its measured throughput is 1/7 of DFMA's), the -log counted as 0
#    because the specification computes it in integer fixed point.  SISe3:
#      per fired transition: 2 (P sums) + 7 (tau) + 1 (t + tau) + 1 (r) + 1 (threshold)
#                            + 2 (two rates) + 1 (A_j) = 15
#      per node-day: closing draw 2 + 7 + 1 = 10; rates 3 x 4 = 12; phi update 12 = 34
FP64_PER_DRAW = 40
FP64_PER_TRANSITION = {3: 15, 1: 12}
FP64_PER_NODE_DAY = {3: 34, 1: 24}
# event step: a 16-B record per event, and read + write of the Nc int32 counts of
# each herd it touches (two for a transfer)
EVENT_RECORD_BYTES = 16
# ncu summary of the stochastic-step kernel: its DRAM bytes per launch count as the
# roofline's traffic only while the kernel sources still hash to the captured ones
SSA_PROFILE = os.path.join(ROOT, "profiles", "k_node_day_dealt_national_day300.md")
# the device sources the stochastic-step kernel is compiled from
SSA_SOURCES = ("ssa.cu", "ssa_device.cuh", "devmath.cuh", "softdiv.cuh", "neglog_table.h", "internal.h")
# days whose prevalence the gradient leg differentiates: the last day and the 52
# week ends (days 7, 14, ..., 364 of the year, as indices 6, 13, ..., 363)
GRADIENT_DAYS = np.array([364] + [7 * k - 1 for k in range(1, 53)], np.int32)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def kernel_sources_digest():
    import hashlib
    d = os.path.join(ROOT, "paper_1502_02908_gb300", "csrc")
    h = hashlib.sha256()
    for f in SSA_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(path):
    """DRAM bytes per launch from an ncu summary (lines `dram_bytes_per_launch: N`
    and `sources_sha256: H`), or None when absent or taken on other sources."""
    try:
        with open(path) as fh:
            kv = dict(line.strip("- `\n").split(": ", 1) for line in fh if ": " in line and line.startswith("- `"))
        if kv.get("sources_sha256") != kernel_sources_digest():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--days", type=int, default=1460)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-gradient", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--uneven-instances", type=int, default=512)
    ap.add_argument("--no-synthetic", action="store_true")
    ap.add_argument("--no-fitting", action="store_true")
    ap.add_argument("--no-general", action="store_true")
    ap.add_argument("--no-sharded", action="store_true")
    return ap.parse_args()


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_baseline(w, days, note):
    """Times the CPU oracle (single thread) on the first `days` days of `w`."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.run(w, ndays=days, replicates=[0])
    dt = time.perf_counter() - t0
    nd = w.N * days
    ev = int(r.counters[0, 0] + r.counters[0, 1])
    return {"value": nd / dt, "unit": "node-days/s", "cores": 1, "kind": "oracle",
            "sample": f"{note}: first {days} of {w.T} days, 1 replicate, single thread",
            "seconds": dt, "events_per_s": ev / dt}, r


def oracle_many(jobs, threads=None):
    """Runs the CPU oracle on every (workload, replicate, days) of `jobs`, one job per
    host thread on all cores (each oracle call is single-threaded C that releases
    the interpreter lock).  Returns (results, wall seconds, threads used)."""
    import oracle
    oracle.build()
    L = oracle.lib()
    n = max(1, min(threads or os.cpu_count() or 1, len(jobs)))
    # largest jobs first, so that the pool's tail is short
    by_size = sorted(range(len(jobs)), key=lambda i: -jobs[i][0].N * jobs[i][2])
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        futs = {i: ex.submit(oracle.run, jobs[i][0], ndays=jobs[i][2], replicates=[jobs[i][1]], lib_handle=L)
                for i in by_size}
        res = [futs[i].result() for i in range(len(jobs))]
    return res, time.perf_counter() - t0, n


def traced_kernels(sim, reset, run):
    """Per-kernel device time over one untimed run: the day loop captured as a CUDA
    graph with a pair of CUDA events around every kernel (no host launch gaps in
    the spans) and without programmatic dependent launch, so that each span holds
    that kernel's own execution only (under programmatic dependent launch a kernel
    starts early and its span includes waiting for the previous one).  Returns
    {"ssa" | "events" | "finalize": (ms, launches)}."""
    sim.set_launch("graph")
    sim.set_overlap(False)
    reset()
    sim.profile(True)
    run()
    prof = sim.profile_read()
    sim.profile(False)
    sim.set_overlap(True)
    return prof


def event_bytes(w, days):
    """Algorithmic bytes of the event step over days [0, days): each event's 16-B
    record plus a read and a write of the Nc counts of every herd it touches."""
    from paper_1502_02908_gb300 import workloads as W
    m = w.events.day < days
    n = int(m.sum())
    n_transfer = int((w.events.kind[m] == W.EXTERNAL).sum())
    return n * EVENT_RECORD_BYTES + (n + n_transfer) * w.nc * 4 * 2


def fp64_peak(B):
    """Measured FP64 instruction-lane throughput (sim_fp64_peak): FMA and add."""
    fma, fma_ms = B.fp64_peak(0, 1 << 14)
    add, _ = B.fp64_peak(1, 1 << 14)
    return {"fma_lane_ops_per_s": fma, "add_lane_ops_per_s": add, "fma_launch_ms": fma_ms,
            "how": "sim_fp64_peak: 8 independent chains per thread, whole waves, best of 3 launches"}


def ssa_alone(B, torch, w, R, tuned, steps=2):
    """The stochastic-step kernel timed alone: the same instance and replicates
    without their events, so that every launch of the day loop is a stochastic
    step (plus one phi/statistics launch at the end), captured as a CUDA graph
    without programmatic dependent launch and timed with one pair of CUDA events
    around the whole run.  Returns {"ms_per_launch", "launches", "transitions",
    "node_days"} of one run (its own transitions)."""
    sim = B.Sim(w.model, w.u0, w.phi0, w.params, w.T, seed=w.seed)
    sim.set_group_threshold(tuned["group_threshold"])
    sim.tune(tuned["warp_threshold"])
    sim.set_launch("graph")
    sim.set_overlap(False)
    u0 = np.repeat(w.u0[None], R, 0)
    phi0 = np.repeat(w.phi0[None], R, 0)
    times = []
    _, _, c0 = sim.stats()
    for i in range(1 + steps):
        sim.set_state(u0, phi0, 0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(); sim.run(w.T); e1.record()
        torch.cuda.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
    _, _, c1 = sim.stats()
    sim.close()
    ms = statistics.median(times)
    return {"ms_per_launch": ms / w.T, "launches": w.T, "run_ms": ms,
            "transitions": int((c1[:, 0] - c0[:, 0]).sum()) // (1 + steps), "node_days": w.N * R * w.T}


def ssa_roofline(w, R, alone, peak, ms_per_step, hbm_peak):
    """Roofline of the stochastic-step kernel from its launches timed alone."""
    avg_s = alone["ms_per_launch"] / 1000
    n = alone["launches"]
    # draws: every fired transition plus the one draw per node-day that ends the day
    # (an upper bound: a node-day with no positive rate draws nothing)
    draws = alone["transitions"] + alone["node_days"]
    per_launch = FP64_PER_DRAW * draws / n
    spec_per_launch = (FP64_PER_TRANSITION[w.model] * alone["transitions"] +
                       FP64_PER_NODE_DAY[w.model] * alone["node_days"]) / n
    achieved = per_launch / avg_s
    bytes_per_launch = SSA_BYTES_PER_NODE_DAY[w.model] * w.N * R
    hbm = bytes_per_launch / avg_s / 1e9
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G FP64 lane-ops/s",
            "frac": achieved / peak,
            "ops_per_launch": per_launch, "ops_count": f"{FP64_PER_DRAW} per draw (draws = transitions + node-days)",
            "frac_spec_count": spec_per_launch / avg_s / peak,
            "avg_launch_us": 1e6 * avg_s, "launches": n,
            "timing": "the stochastic step alone (the instance without its events, graph-launched back to back, "
                      "no programmatic dependent launch), one pair of CUDA events around the run; its own "
                      f"transitions ({alone['transitions']}) counted",
            "avg_launch_x_day_loop_ms": 1e3 * avg_s * w.T, "fits_in_ms_per_step": 1e3 * avg_s * w.T <= ms_per_step,
            "peak_source": "measured: sim_fp64_peak (FP64 FMA lane-ops/s on this GPU)",
            "hbm": {"achieved": hbm, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm / hbm_peak if hbm_peak else None, "bytes_per_launch": bytes_per_launch}}


def events_roofline(w, T, prof, hbm_peak):
    ev_ms, ev_n = prof["events"]
    if not ev_n:
        return None
    avg_s = ev_ms / 1000 / ev_n
    b = event_bytes(w, T) / ev_n
    return {"kernel": "k_events_day_df (event step)", "bound": "latency", "achieved": b / avg_s / 1e9,
            "peak": hbm_peak, "unit": "GB/s", "frac": (b / avg_s / 1e9) / hbm_peak if hbm_peak else None,
            "bytes_per_launch": b, "avg_launch_us": 1e6 * avg_s, "launches": ev_n,
            "timing": "CUDA events around every launch of a graph-captured day loop without programmatic "
                      "dependent launch; each span also holds the event records' own cost (a few us)",
            "note": "HBM view of algorithmic bytes; the launch is bound by the day's longest "
                    "transfer-graph component, applied serially by one thread"}


def plain_sise_leg(args, B, W, torch, oracle_check, fp64=None, hbm_peak=None):
    """The plain SISe instance: 1,000 nodes x 365 days, 20,000 events; bit-exact
    against the oracle over the whole horizon."""
    from paper_1502_02908_gb300 import autotune
    w = W.sise_plain()
    best, _ = autotune.autotune(w, days=73, thresholds=(1 << 30, 200), modes=("stream", "graph"), repeats=1,
                                groups=(1 << 30, 100))
    sim = B.Sim.from_workload(w)
    sim.set_group_threshold(best["group_threshold"]); sim.tune(best["warp_threshold"]); sim.set_launch(best["launch"])
    u0 = w.u0[None]; phi0 = w.phi0[None]
    steps, warm = 10, 3
    times = []
    _, _, c0 = sim.stats()
    for i in range(warm + steps):
        sim.set_state(u0, phi0, 0)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(); sim.run(w.T); e1.record()
        torch.cuda.synchronize()
        if i >= warm:
            times.append(e0.elapsed_time(e1))
    c, p, _ = sim.state()
    pi, pn, c1 = sim.stats()
    sim.close()
    ms = statistics.median(times)
    per = (c1[0] - c0[0]) // (warm + steps)
    line = {"workload": f"SISe plain: {w.N} nodes x {w.T} days, {len(w.events)} events, 1 replicate",
            "value": w.N * w.T / (ms / 1000), "unit": "node-days/s", "ms_per_step": ms, "steps": steps,
            "warmup": warm, "transitions_per_step": int(per[0]), "events_per_step": int(per[1]),
            "events_per_s": int(per[0] + per[1]) / (ms / 1000), "launch": best}
    if fp64:
        alone = ssa_alone(B, torch, w, 1, best)
        line["roofline"] = dict(kernel="k_node_day_dealt (stochastic step)",
                                **ssa_roofline(w, 1, alone, fp64, ms, hbm_peak))
        line["roofline"]["hbm"]["note"] = "algorithmic bytes; the state stays in L2 within a step"
    if oracle_check:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        ref = oracle.run(w)
        dt = time.perf_counter() - t0
        line["bitexact_vs_oracle"] = {
            "days": w.T, "counts_equal": bool(np.array_equal(c, ref.counts)),
            "phi_equal": bool(np.array_equal(p, ref.phi)),
            "daily_stats_equal": bool(np.array_equal(pi[:, :w.T], ref.prev_i) and np.array_equal(pn[:, :w.T], ref.prev_n)),
            "counters_equal": bool(np.array_equal(c1[0] - c0[0], ref.counters[0] * (warm + steps)))}
        line["cpu_baseline"] = {"value": w.N * w.T / dt, "unit": "node-days/s", "cores": 1, "kind": "oracle",
                                "sample": "the whole instance, 1 replicate, single thread"}
    return line


def batched_leg(args, B, W, torch, plain_value, hbm_peak, fp64, oracle_check):
    """The national network batched: 256 replicates x 365 days, each with its own
    (upsilon, gamma), in one handle; launch mode chosen by a short autotune.  A
    seeded subset of replicates is checked bit for bit against the oracle, which
    also gives the all-core CPU baseline."""
    from paper_1502_02908_gb300 import autotune
    w = W.sise3_batched(R=256, T=365)
    # the daily CUDA-graph loop against the persistent work-stealing kernel in each
    # block shape (256 replicates give it work enough to fill the GPU every day)
    best, table = autotune.autotune(w, days=20, thresholds=(1 << 30,), modes=("graph", "persistent"), repeats=1,
                                    groups=(1 << 30, 800), shapes=B.BATCH_SHAPES)
    sim = B.Sim.from_workload(w)
    autotune.apply(sim, best)
    u0 = np.repeat(w.u0[None], w.R, 0); phi0 = np.repeat(w.phi0[None], w.R, 0)
    steps, warm = 3, 1
    times = []
    _, _, c0 = sim.stats()
    for i in range(warm + steps):
        sim.set_state(u0, phi0, 0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(); sim.run(w.T); e1.record()
        torch.cuda.synchronize()
        if i >= warm:
            times.append(e0.elapsed_time(e1))
    counts, phi, _ = sim.state()
    _, _, c1 = sim.stats()
    ms = statistics.median(times)
    value = w.N * w.R * w.T / (ms / 1000)
    trans = int((c1[:, 0] - c0[:, 0]).sum()) // (warm + steps)
    evs = int((c1[:, 1] - c0[:, 1]).sum()) // (warm + steps)
    sim.close()
    B.batch_shape(*B.BATCH_SHAPES[0])
    line = {"workload": f"SISe3 national network, {w.R} replicates x {w.T} days, own (upsilon, gamma) each",
            "value": value, "unit": "node-days/s", "steps": steps, "warmup": warm, "ms_per_step": ms,
            "events_per_s": (trans + evs) / (ms / 1000), "transitions_per_s": trans / (ms / 1000),
            "scheduled_events_per_s": evs / (ms / 1000), "transitions_per_step": trans, "events_per_step": evs,
            "launch": best, "autotune_ms_20_days": {f"{m} {sh[0]}x{sh[1]}" if sh else m: round(t, 2)
                                                     for _, g, m, sh, t in table if g == best["group_threshold"]},
            "vs_plain": value / plain_value}
    if best["launch"] == "persistent":
        # arithmetic view of the whole persistent launch (event items included, so
        # a lower bound for its stochastic-step chunks)
        achieved = FP64_PER_DRAW * (trans + w.N * w.R * w.T) / (ms / 1000)
        line["roofline"] = {"kernel": "k_batch %dx%d (persistent: stochastic-step chunks and event items)"
                                      % tuple(best["batch_shape"]),
                            "bound": "alu", "achieved": achieved / 1e9, "peak": fp64 / 1e9,
                            "unit": "G FP64 lane-ops/s", "frac": achieved / fp64,
                            "ops_count": f"{FP64_PER_DRAW} per draw (draws = transitions + node-days)",
                            "peak_source": "measured: sim_fp64_peak (FP64 FMA lane-ops/s on this GPU)"}
    else:
        alone = ssa_alone(B, torch, w, w.R, best, steps=1)
        line["roofline"] = dict(kernel="k_node_day_dealt (stochastic step, 256 replicates)",
                                **ssa_roofline(w, w.R, alone, fp64, ms, hbm_peak))
        line["roofline"]["hbm"]["note"] = "the state (counts and phi of 256 replicates, 0.6 GB read and " \
                                          "written per launch) exceeds L2"
    if line["roofline"]["frac"] > 1:
        line["roofline"]["note"] = ("a fraction above 1: the kernel delivers the binary64 specification's "
                                    "decisions faster than the FP64 pipe could compute them, because it takes "
                                    "them in binary32 and fixed point within certified error margins (binary64 "
                                    "only inside them); its own limit is instruction issue")
    if oracle_check:
        rng = np.random.default_rng(3)
        reps = sorted(int(r) for r in rng.choice(w.R, size=16, replace=False))
        res, dt, n = oracle_many([(w, r, w.T) for r in reps])
        ok_c = all(np.array_equal(counts[r], x.counts[0]) for r, x in zip(reps, res))
        ok_p = all(np.array_equal(phi[r], x.phi[0]) for r, x in zip(reps, res))
        line["bitexact_vs_oracle"] = {"replicates": reps, "days": w.T, "counts_equal": bool(ok_c),
                                      "phi_equal": bool(ok_p)}
        line["cpu_baseline"] = {"value": len(reps) * w.N * w.T / dt, "unit": "node-days/s", "cores": n,
                                "kind": "oracle",
                                "sample": f"{len(reps)} seeded replicates of the {w.R}, whole horizon, "
                                          "one replicate per host thread"}
    return line


def gradient_leg(args, B, W, G, torch, oracle_check=False):
    """The score-function gradient on SISe, 10,000 nodes x 4,096 replicates x 365
    days, of the final prevalence and the 52 week-end prevalences with respect to
    (upsilon, gamma, beta, alpha): simulation with score terms, the reverse sweep of
    the phi recursion and the moment sums, in chunks of 1,024 replicates.  Checked
    against central finite differences (h = 1e-3 relative, common random numbers)
    on the first 1,024 replicates at all 53 days (the final day and the 52 week
    ends) and all four parameters: 212 comparisons, passed when none is 4 standard
    errors apart and at most 3 are more than 3 apart (under the normal law 0.57 are
    expected beyond 3)."""
    w = W.sise_gradient()
    spec = G.GradientSpec(w, GRADIENT_DAYS, chunk=1024)
    G.score_gradient(G.GradientSpec(W.sise_gradient(R=64, T=30), np.array([29], np.int32), chunk=64))  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chunks, R, _ = G.run_moments(spec)
    dt = time.perf_counter() - t0
    ratios = spec.class_ratios()
    mean_f, grad, se = G.estimate(chunks, R, ratios)
    line = {"workload": f"score-function gradient, SISe {w.N} nodes x {w.R} replicates x {w.T} days, "
                        f"{len(w.events)} events; f = final and 52 week-end prevalences; theta = "
                        "(upsilon, gamma, beta, alpha)",
            "seconds": dt, "value": w.N * w.R * w.T / dt, "unit": "node-days/s (with score terms)",
            "chunks": int(chunks.shape[0]), "chunk_replicates": spec.chunk,
            "final_prevalence": float(mean_f[0]), "gradient_final": grad[0].tolist(), "se_final": se[0].tolist()}
    # central differences with common random numbers on the first chunk's
    # replicates, at every differentiated day (the runs cost the same for any
    # number of days)
    w1 = W.sise_gradient(R=spec.chunk)
    s1 = G.GradientSpec(w1, GRADIENT_DAYS, chunk=spec.chunk)
    _, g1, se1 = G.estimate(chunks[:1], spec.chunk, ratios)
    t0 = time.perf_counter()
    fd, fd_se = G.fd_gradient(s1, rel_h=1e-3)
    z = np.abs(g1 - fd) / np.sqrt(se1 ** 2 + fd_se ** 2)
    pick = [0, 26]                                 # final day (364) and week 26 (day index 181)
    line["fd_check"] = {"replicates": spec.chunk, "days": GRADIENT_DAYS.tolist(), "rel_h": 1e-3,
                        "comparisons": int(z.size), "max_z": float(z.max()),
                        "beyond_3_se": int((z >= 3.0).sum()), "expected_beyond_3_se": round(z.size * 0.0027, 2),
                        "passed": bool(z.max() < 4.0 and (z >= 3.0).sum() <= 3),
                        "final_and_week26": {"days": GRADIENT_DAYS[pick].tolist(), "score": g1[pick].tolist(),
                                             "score_se": se1[pick].tolist(), "fd": fd[pick].tolist(),
                                             "fd_se": fd_se[pick].tolist(), "z": z[pick].tolist(),
                                             "within_3_se": bool(np.all(z[pick] < 3.0))},
                        "seconds": time.perf_counter() - t0}
    if oracle_check:
        # the oracle with score terms on 16 replicates, one per host thread, and the
        # 4,096-replicate run extrapolated linearly from it
        import oracle
        oracle.build()
        L = oracle.lib()
        n = min(16, os.cpu_count() or 1)
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            list(ex.map(lambda r: oracle.run(w, replicates=[r], score=True, lib_handle=L), range(n)))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n * w.N * w.T / dt, "unit": "node-days/s (with score terms)", "cores": n,
                                "kind": "oracle",
                                "sample": f"{n} replicates with score terms, whole horizon, one replicate per host "
                                          f"thread; the {w.R}-replicate run extrapolated: "
                                          f"{dt * w.R / n:.0f} s"}
    return line


def uneven_leg(args, B, W, torch, oracle_check, fp64=None):
    """The uneven batch: 512 instances mixing SISe and SISe3 (node counts log-uniform
    in [100, 50,000], horizons 90-1,460 days, 80 events per node-year) advanced in
    one persistent work-stealing launch, against running the instances one after
    another (CUDA-graph day loops); every instance's final counts equal across the
    two, and a seeded subset of instances bit-exact against the oracle."""
    t0 = time.perf_counter()
    ws = W.uneven_batch(n_inst=args.uneven_instances)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    # handles created on host threads, one instance each (their event scheduling is
    # host work; the library keeps no state shared between handles)
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        sims = list(ex.map(B.Sim.from_workload, ws))
    load_s = time.perf_counter() - t0
    node_days = sum(w.N * w.T for w in ws)
    n_events = sum(len(w.events) for w in ws)
    steps, warm = 2, 1
    times = []
    for i in range(warm + steps):
        for s in sims:
            s.reset()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(); B.run_batch(sims); e1.record()
        torch.cuda.synchronize()
        if i >= warm:
            times.append(e0.elapsed_time(e1))
    finals = [s.state()[:2] for s in sims]
    batch_states = [f[0] for f in finals]
    batch_phi = [f[1] for f in finals]
    ctr = np.stack([s.stats()[2][0] for s in sims])
    ms = statistics.median(times)
    # one after another: each instance's own CUDA-graph day loop
    for s in sims:
        s.reset()
        s.set_launch("graph")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for w, s in zip(ws, sims):
        s.run(w.T)
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    same = all(np.array_equal(s.state()[0], c) for s, c in zip(sims, batch_states))
    for s in sims:
        s.close()
    per_run = ctr                                   # sim_reset clears the counters: the last run's
    line = {"workload": f"uneven batch: {len(ws)} instances (SISe / SISe3, N log-uniform 100-50,000, "
                        "T 90-1,460 days, 80 events per node-year), one persistent launch",
            "value": node_days / (ms / 1000), "unit": "node-days/s", "ms_per_step": ms, "steps": steps,
            "warmup": warm, "node_days_per_step": node_days, "events": n_events,
            "events_per_s": float(per_run[:, 0].sum() + per_run[:, 1].sum()) / (ms / 1000),
            "transitions_per_s": float(per_run[:, 0].sum()) / (ms / 1000),
            "scheduled_events_per_s": float(per_run[:, 1].sum()) / (ms / 1000),
            "block_shape": list(B.BATCH_SHAPES[0]),
            "one_after_another_ms": seq_ms, "speedup_vs_one_after_another": seq_ms / ms,
            "batch_equals_one_after_another": bool(same), "generate_s": gen_s, "load_events_s": load_s}
    if fp64:
        # arithmetic view of the whole persistent launch (its event items included,
        # so a lower bound for the stochastic step): 40 FP64 lane-ops per draw
        draws = float(per_run[:, 0].sum()) + node_days
        achieved = FP64_PER_DRAW * draws / (ms / 1000)
        line["roofline"] = {"kernel": "k_batch (persistent: stochastic-step chunks and event items)",
                            "bound": "alu", "achieved": achieved / 1e9, "peak": fp64 / 1e9,
                            "unit": "G FP64 lane-ops/s", "frac": achieved / fp64,
                            "ops_count": f"{FP64_PER_DRAW} per draw (draws = transitions + node-days)",
                            "peak_source": "measured: sim_fp64_peak (FP64 FMA lane-ops/s on this GPU)"}
        if achieved > fp64:
            line["roofline"]["note"] = ("a fraction above 1: the kernel delivers the binary64 specification's "
                                        "decisions faster than the FP64 pipe could compute them, because it "
                                        "takes them in binary32 and fixed point within certified error margins "
                                        "(binary64 only inside them); its own limit is instruction issue")
    if oracle_check:
        rng = np.random.default_rng(5)
        pick = sorted(int(i) for i in rng.choice(len(ws), size=min(16, len(ws)), replace=False))
        res, dt, n = oracle_many([(ws[i], 0, ws[i].T) for i in pick])
        ok_c = all(np.array_equal(batch_states[i][0], r.counts[0]) for i, r in zip(pick, res))
        ok_p = all(np.array_equal(batch_phi[i][0], r.phi[0]) for i, r in zip(pick, res))
        line["bitexact_vs_oracle"] = {"instances": pick, "counts_equal": bool(ok_c), "phi_equal": bool(ok_p)}
        nd = sum(ws[i].N * ws[i].T for i in pick)
        line["cpu_baseline"] = {"value": nd / dt, "unit": "node-days/s", "cores": n, "kind": "oracle",
                                "sample": f"{len(pick)} seeded instances of the {len(ws)}, whole horizons "
                                          f"({nd} node-days), one instance per host thread"}
    return line


def synthetic_leg(args, B, W, torch, oracle_check):
    """The paper's synthetic benchmark (Sec. 4.2): 1,000 nodes with S = I = 1,000,
    unit rates both ways, 1,000 days, rho = 0.1 with k = 16 sub-domains (12 transfers
    a day): about 2,000 transitions per node-day.  Launch shape by a short autotune;
    bit-exactness checked against the oracle over the first days."""
    from paper_1502_02908_gb300 import autotune
    w = W.synthetic_sis()
    best, _ = autotune.autotune(w, days=10, thresholds=(1 << 30, 400), modes=("graph",), repeats=1,
                                groups=(1 << 30, 100))
    sim = B.Sim.from_workload(w)
    sim.set_group_threshold(best["group_threshold"]); sim.tune(best["warp_threshold"]); sim.set_launch(best["launch"])
    u0 = w.u0[None]; phi0 = w.phi0[None]
    steps, warm = 2, 1
    times = []
    _, _, c0 = sim.stats()
    for i in range(warm + steps):
        sim.set_state(u0, phi0, 0)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(); sim.run(w.T); e1.record()
        torch.cuda.synchronize()
        if i >= warm:
            times.append(e0.elapsed_time(e1))
    _, _, c1 = sim.stats()
    sim.close()
    ms = sum(times) / steps
    trans = int(c1[0, 0] - c0[0, 0]) // (warm + steps)
    line = {"workload": f"synthetic SIS (Sec. 4.2): {w.N} nodes, S = I = 1000, unit rates, {w.T} days, "
                        f"rho = 0.1, k = 16 ({len(w.events)} transfers)",
            "value": w.N * w.T / (ms / 1000), "unit": "node-days/s", "transitions_per_s": trans / (ms / 1000),
            "transitions_per_step": trans, "steps": steps, "warmup": warm, "ms_per_step": ms,
            "launch": best}
    if oracle_check:
        import oracle
        oracle.build()
        days = 3
        t0 = time.perf_counter()
        ref = oracle.run(w, ndays=days, replicates=[0])
        dt = time.perf_counter() - t0
        chk = B.Sim.from_workload(w)
        chk.set_group_threshold(best["group_threshold"]); chk.tune(best["warp_threshold"])
        chk.run(days)
        c, p, _ = chk.state()
        chk.close()
        line["bitexact_vs_oracle"] = {"days": days, "counts_equal": bool(np.array_equal(c[0], ref.counts[0])),
                                      "phi_equal": bool(np.array_equal(p[0], ref.phi[0]))}
        line["oracle_transitions_per_s"] = int(ref.counters[0, 0]) / dt
    return line


def general_leg(args, B, W, torch, oracle_check):
    """The general compartment model (product-form propensities, sparse dependency
    graph, event masks and offsets) on national-size networks: SISe3 written in the
    general form on the national network (the same instance as the main line), and
    an SEIRS model with two continuous variables under the midpoint update on 37,000
    nodes.  CUDA-graph day loop; bit-exactness against the general oracle over a
    prefix of each horizon."""
    out = {}
    cases = (("sise3_national_general", W.as_general(W.sise3_national()), 365),
             ("seirs_midpoint", W.seirs_env(N=37_000, T=365, n_events=1_000_000, R=1, y_source=W.Y_MIDPOINT), 60))
    from paper_1502_02908_gb300 import autotune
    for name, w, check_days in cases:
        w.T = min(args.days, w.T)
        thr, gthr = -1, -1
        if not args.no_tune:
            # a third of the horizon: the early days of an epidemic do not rank the thresholds
            (thr, gthr), _ = autotune.autotune_general(w, days=max(10, w.T // 3))
        sim = B.GenSim.from_workload(w)
        sim.set_launch("graph")
        n_warp = sim.set_warp_threshold(thr)
        n_group = sim.set_group_threshold(gthr)
        u0 = w.u0[None]; y0 = w.y0[None]
        steps, warm = 2, 1
        times = []
        c0 = sim.counters()
        for i in range(warm + steps):
            sim.set_state(u0, y0, 0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(); sim.run(w.T); e1.record()
            torch.cuda.synchronize()
            if i >= warm:
                times.append(e0.elapsed_time(e1))
        c1 = sim.counters()
        sim.close()
        ms = sum(times) / steps
        trans = int(c1[0, 0] - c0[0, 0]) // (warm + steps)
        m = w.model
        line = {"workload": f"{name}: {w.N} nodes x {w.T} days, {len(w.events)} events, "
                            f"{m.nc} compartments, {m.nt} transitions, {m.ny} continuous variables",
                "value": w.N * w.T / (ms / 1000), "unit": "node-days/s", "transitions_per_s": trans / (ms / 1000),
                "transitions_per_step": trans, "ms_per_step": ms, "steps": steps, "warmup": warm,
                "gpu_launches_per_step": 2 * w.T + (1 if m.ny and m.y_source != W.Y_PRE_EVENT else 0),
                "warp_threshold": thr, "warp_nodes": n_warp, "group_threshold": gthr, "group_nodes": n_group}
        if oracle_check:
            import oracle
            oracle.build()
            days = min(check_days, w.T)
            t0 = time.perf_counter()
            ref = oracle.run_general(w, ndays=days)
            dt = time.perf_counter() - t0
            chk = B.GenSim.from_workload(w)
            chk.run(days)
            c, y, _ = chk.state()
            chk.close()
            line["bitexact_vs_oracle"] = {"days": days, "counts_equal": bool(np.array_equal(c, ref.counts)),
                                          "y_equal": bool(np.array_equal(y, ref.y))}
            line["oracle_node_days_per_s"] = w.N * days / dt
        out[name] = line
    return out


def fitting_leg(args, B, W, torch):
    """The parameter fit of Sec. 4.3 on the national network: a reference trajectory
    with upsilon* = [8.8, 3.2, 1]e-3, 21 regions, N = 10 trajectories per evaluation of
    G over the whole horizon, Hooke-Jeeves from k0 = 1.6 k* with steps 0.5 k*, 20
    iterations (the paper's setup)."""
    from paper_1502_02908_gb300 import fitting as F
    w = W.sise3_national()
    regions = F.county_regions(w.N, 21)
    ups_star = np.array([8.8e-3, 3.2e-3, 1e-3])
    k_star = F.superparameters(ups_star, w.params.gamma[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = F.reference_totals(w, regions, 21, ups_star)
    goal = F.Goal(w, regions, 21, ref, trajectories=10)
    try:
        goal(1.6 * k_star)                                   # warm-up (graph capture)
        goal.evaluations = 0
        t1 = time.perf_counter()
        res = F.hooke_jeeves(lambda k: goal(k)[0], 1.6 * k_star, 0.5 * k_star, iterations=20)
        t_search = time.perf_counter() - t1
        g_star, vg_star = goal(k_star)
        g_hat, vg_hat = goal(res.x)
    finally:
        goal.close()
    return {"workload": f"parameter fit (Sec. 4.3) on the national network: {w.N} herds x {w.T} days, "
                        "21 regions, 10 trajectories per evaluation, Hooke-Jeeves 20 iterations from 1.6 k*",
            "search_s": t_search, "evaluations": res.evaluations, "s_per_evaluation": t_search / res.evaluations,
            "setup_s": t1 - t0, "k_star": k_star.tolist(), "k_hat": res.x.tolist(),
            "G2_k_star": g_star, "G2_k_hat": g_hat, "VG2_k_star": vg_star,
            "relative_residual": F.relative_residual(np.sqrt(g_hat), np.sqrt(g_star)),
            "paper_context": "Sec. 4.3 Table: 46.6 min on 12 CPU cores for 10 trajectories (register data)",
            "gradient_variant": gradient_fit_leg(F, W, torch)}


def gradient_fit_leg(F, W, torch):
    """The gradient-based variant: the daily national prevalence of 1,000 SISe herds
    over 120 days (512 replicates per evaluation) against a target curve from
    independent streams at (upsilon*, gamma*); normalised descent with the
    score-function gradient in log scale from (1.5 upsilon*, 0.7 gamma*)."""
    w = W.sise_plain(N=1000, T=120, n_events=6000, R=512)
    days = np.arange(3, 120, 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    target = F.prevalence_curve(w, days, seed_offset=1000)
    goal = F.PrevalenceGoal(w, days, target)
    x0 = np.log([1.5, 0.7])
    g0, grad0, se0 = goal(x0)
    t1 = time.perf_counter()
    res = F.gradient_descent(goal, x0, step=0.2, iterations=20)
    t_search = time.perf_counter() - t1
    return {"workload": f"SISe, {w.N} herds x {w.T} days, {w.R} replicates per evaluation, prevalence on "
                        f"{days.size} days; 20 descent steps from (1.5, 0.7) x (upsilon*, gamma*)",
            "search_s": t_search, "setup_s": t1 - t0, "evaluations": res.evaluations + 1,
            "scale_hat": np.exp(res.x).tolist(), "G2_start": g0, "G2_end": res.f,
            "gradient_over_se_at_start": (np.abs(grad0) / se0).tolist()}


def sharded_leg(B, W, torch, dist, rank, ws, w):
    """One national replicate with its nodes split over the ranks: each rank runs
    the stochastic step and phi update of its contiguous node range and the whole
    event list, exchanging the day's touched herds' counts with an all-gather
    (NCCL) between the two halves of each day.  Each rank checks its own nodes
    against a single-handle run of the same replicate."""
    from paper_1502_02908_gb300 import sharded as S
    exchange = S.allgather_exchange()
    times = []
    own = None
    for i in range(2):                             # the first run warms up
        e = S.EngineShard(w, rank, ws)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        S.run_days(e, w.T, exchange)
        e1.record()
        torch.cuda.synchronize()
        if i:
            times.append(e0.elapsed_time(e1))
        own = e.own_state()
        lo, hi = e.lo, e.hi
        e.close()
    ms = torch.tensor([times[0]], device="cuda")
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    single = B.Sim(w.model, w.u0, w.phi0, w.params, w.T, seed=w.seed)
    single.load_events(w.events)
    single.run(w.T)
    c, p, _ = single.state()
    single.close()
    ok = torch.tensor([int(np.array_equal(own[0], c[:, :, lo:hi]) and np.array_equal(own[1], p[:, lo:hi]))],
                      device="cuda")
    dist.all_reduce(ok, op=dist.ReduceOp.MIN)
    ms = float(ms.item())
    return {"workload": f"SISe3 national, one replicate, {w.N} herds x {w.T} days split over {ws} ranks "
                        "(node-sharded; touched herds exchanged daily by all-gather)",
            "value": w.N * w.T / (ms / 1000), "unit": "node-days/s", "ms_per_step": ms, "ranks": ws,
            "scaling": "strong", "bitexact_vs_single_gpu": bool(ok.item())}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


# days of the national horizon that one CPU step covers: the same sample for the
# reference arm's steps and for the main line's cpu_baseline
CPU_SAMPLE_DAYS = 365


def run_reference(args, dist, rank, ws):
    from paper_1502_02908_gb300 import workloads as W
    if rank != 0:
        return
    w = W.sise3_national()
    days = CPU_SAMPLE_DAYS                      # bounded sample per step
    times = []
    for i in range(args.warmup + args.steps):
        base, _ = oracle_baseline(w, days, "national SISe3")
        if i >= args.warmup:
            times.append(base["seconds"])
    total = sum(times)
    value = w.N * days * args.steps / total
    sample = f"national SISe3: first {days} of {w.T} days, 1 replicate, single thread, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "node-days/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+int32", "data": "synthetic",
            "config": {"workload": f"SISe3 national: {w.N} herds x {w.T} days, {len(w.events)} events, "
                                   "1 replicate per GPU (plain)",
                       "replicates_per_gpu": 1, "parallelism": f"replicas x{args.gpus}"},
            "cpu_baseline": {"value": value, "unit": "node-days/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "node-days/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist, rank, ws = dist_setup()
    if args.impl == "reference":
        run_reference(args, dist, rank, ws)
        if dist:
            dist.destroy_process_group()
        return
    import torch
    from paper_1502_02908_gb300 import binding as B
    from paper_1502_02908_gb300 import workloads as W
    from paper_1502_02908_gb300.build import build
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build()
    leg_s = {}
    t_leg = time.perf_counter()
    w = W.sise3_national()
    w.T = min(args.days, w.T)        # a shorter horizon of the same instance
    tuned = {"warp_threshold": -1, "group_threshold": -1, "launch": "graph"}
    if not args.no_tune:
        from paper_1502_02908_gb300 import autotune
        tuned, _ = autotune.autotune(w, days=max(10, w.T // 10), thresholds=(1 << 30, 800, 400, 200),
                                     modes=("stream", "graph"), repeats=1, groups=(1 << 30, 300, 200, 100))
    sim = B.Sim(w.model, w.u0, w.phi0, w.params, w.T, seed=w.seed, replicate_base=rank)
    t0 = time.perf_counter()
    sim.load_events(w.events)
    preprocess_s = time.perf_counter() - t0

    def configure():
        sim.set_group_threshold(tuned["group_threshold"])
        sim.tune(tuned["warp_threshold"])
        sim.set_launch(tuned["launch"])

    configure()
    stream = torch.cuda.current_stream()
    R, N, T = 1, w.N, w.T
    u0_all = np.repeat(w.u0[None], R, 0)
    phi0_all = np.repeat(w.phi0[None], R, 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def reset():
        sim.set_state(u0_all, phi0_all, 0)

    def step():
        sim.run(T)

    for _ in range(args.warmup):
        reset(); step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    _, _, ctr0 = sim.stats()
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            reset()
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream); step(); e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    total_ms = sum(times)
    pi, pn, ctr1 = sim.stats()
    # counters accumulate over every run of the handle: the timed steps' share
    transitions = int(ctr1[0, 0] - ctr0[0, 0]) // args.steps
    events = int(ctr1[0, 1] - ctr0[0, 1]) // args.steps
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    node_days = N * T * R * ws
    value = node_days * args.steps / (total_ms / 1000)
    ev_rate = (transitions + events) * ws * args.steps / (total_ms / 1000)
    ms_per_step = total_ms / args.steps

    # end to end through the C ABI with host buffers: set state from host, run, read
    # the final state and the daily statistics back to host
    e2e_times = []
    for _ in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.set_state(u0_all, phi0_all, 0)
        sim.run(T)
        c, p, _ = sim.state()
        pi, pn, ctr2 = sim.stats()
        e2e_times.append(time.perf_counter() - t0)
    h2d = u0_all.nbytes + phi0_all.nbytes
    d2h = c.nbytes + p.nbytes + pi.nbytes + pn.nbytes + ctr2.nbytes
    e2e = {"value": node_days / statistics.median(e2e_times), "unit": "node-days/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # per-kernel device time over one traced (untimed) step without overlap
    prof = traced_kernels(sim, reset, step)
    configure()
    ssa_ms, ssa_n = prof["ssa"]
    ev_ms, ev_n = prof["events"]
    fin_ms, fin_n = prof["finalize"]
    tot_k = ssa_ms + ev_ms + fin_ms
    peaks = measured_peaks()
    fp64 = fp64_peak(B)
    alone = ssa_alone(B, torch, w, R, tuned)
    roofline = dict(kernel="k_node_day_dealt (stochastic step)",
                    **ssa_roofline(w, R, alone, fp64["fma_lane_ops_per_s"], ms_per_step, peaks.get("hbm_gbs")))
    roofline["traffic"] = profiled_traffic(SSA_PROFILE)
    roofline["hbm"]["note"] = "algorithmic bytes; the state stays in L2 within a step"
    roofline["traced"] = {"share": {"ssa": ssa_ms / tot_k, "events": ev_ms / tot_k, "finalize": fin_ms / tot_k},
                          "step_ms": tot_k, "ssa_avg_launch_us": 1000 * ssa_ms / max(ssa_n, 1),
                          "note": "CUDA events around every launch (each span also holds the event records' "
                                  "own cost)"}

    line = {"metric": METRIC, "value": value, "unit": "node-days/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+int32", "data": "synthetic",
            "config": {"workload": f"SISe3 national: {N} herds x {T} days, {len(w.events)} events, "
                                   "1 replicate per GPU (plain)",
                       "replicates_per_gpu": R, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{ws}"},
            "events_per_s": ev_rate, "ssa_transitions_per_step": transitions, "events_per_step": events,
            "preprocess_s": preprocess_s, "e2e": e2e, "roofline": roofline,
            "roofline_events": events_roofline(w, T, prof, peaks.get("hbm_gbs")),
            "fp64_peak_measured": fp64,
            "gpu_launches": (ssa_n + ev_n + fin_n) * args.steps, "clocks": clk.summary()}
    line["config"]["launch"] = tuned
    oracle_check = not args.no_cpu_baseline
    if rank == 0 and oracle_check:
        days = min(CPU_SAMPLE_DAYS, T)
        base, ref = oracle_baseline(w, days, "national SISe3")
        line["cpu_baseline"] = {k: base[k] for k in ("value", "unit", "cores", "kind")}
        line["cpu_baseline"]["sample"] = (f"national SISe3: first {days} of {w.T} days, 1 replicate, single "
                                          "thread (the reference arm times the same sample per step)")
        # bit-exactness of this configuration at the sampled horizon
        chk = B.Sim(w.model, w.u0, w.phi0, w.params, w.T, seed=w.seed)
        chk.load_events(w.events)
        chk.run(days)
        c, p, _ = chk.state()
        chk.close()
        line["bitexact_vs_oracle"] = {"days": days, "counts_equal": bool(np.array_equal(c[0], ref.counts[0])),
                                      "phi_max_rel": float(np.max(np.abs(p[0] - ref.phi[0]) /
                                                                  np.maximum(np.abs(ref.phi[0]), 1e-300)))}
    sim.close()
    del flush
    leg_s["main"] = time.perf_counter() - t_leg

    def leg(name, fn):
        t = time.perf_counter()
        line[name] = fn()
        torch.cuda.empty_cache()
        leg_s[name] = time.perf_counter() - t

    if dist and not args.no_sharded:
        t = time.perf_counter()
        line["sharded"] = sharded_leg(B, W, torch, dist, rank, ws, w)
        leg_s["sharded"] = time.perf_counter() - t
    if rank == 0:
        if not args.no_plain:
            leg("sise_plain", lambda: plain_sise_leg(args, B, W, torch, oracle_check, fp64["fma_lane_ops_per_s"],
                                                     peaks.get("hbm_gbs")))
        if not args.no_batched:
            leg("batched", lambda: batched_leg(args, B, W, torch, value / ws, peaks.get("hbm_gbs"),
                                               fp64["fma_lane_ops_per_s"], oracle_check))
        if not args.no_gradient:
            from paper_1502_02908_gb300 import gradient as G
            leg("gradient", lambda: gradient_leg(args, B, W, G, torch, oracle_check))
        if not args.no_uneven:
            leg("uneven", lambda: uneven_leg(args, B, W, torch, oracle_check, fp64["fma_lane_ops_per_s"]))
        if not args.no_synthetic:
            leg("synthetic", lambda: synthetic_leg(args, B, W, torch, oracle_check))
        if not args.no_fitting:
            leg("fitting", lambda: fitting_leg(args, B, W, torch))
        if not args.no_general:
            leg("general", lambda: general_leg(args, B, W, torch, oracle_check))
        line["leg_seconds"] = leg_s
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
