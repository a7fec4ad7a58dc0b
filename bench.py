"""Benchmark: Monte Carlo AEB braking rollouts per second on GB300.

Workload: one scenario with the single-scenario distributions (v0~U(15,35),
d0~N(60,5) in [30,90], mu~U(0.4,0.9), grade~N(0,0.02), m~N(1600,100),
Cd~U(0.28,0.35), tau~U(0.1,0.3), delay~U(0.1,0.3), range noise~N(0,0.5);
per-axle caps, lead at d0, dt = 1 ms, 10 s horizon), N = 1e7 samples: the
largest point of the throughput sweep over N = 1e3..1e7.  Parameters are drawn
by the library's seeded host sampler and are resident in HBM when timing starts.

A step = one pass of the hot path: the FP32-compensated rollout of all N
samples plus the deterministic reduction to counts, moments and histograms.
`value` is rollouts/s of that step; the FP64-plain path is timed on the same
samples and reported beside it ("fp64_plain").  `e2e` is the same metric
through aeb_evaluate (pinned host parameters in, host stats out, copies in
the timed region).  The inputs (800 MB of parameters) exceed the 129 MB L2,
so no flush is needed between steps.

Beside the headline the line carries the serving run (Poisson requests,
latency percentiles), the scenario-grid batched run, the TTC-threshold sweep and
a coarse-step study (the same samples at dt = 0.1 .. 20 ms: speed and the error
against the 0.1 ms rollouts), a moving-lead run (a lead braking ahead), a TTC
run with noisy, late and missing readings and a rare-event estimate (plain Monte
Carlo against importance sampling); `--no-extras` skips the last six.

`--impl reference` times the plain CPU oracle on a bounded sample of the same
workload on the host cores (the CPU baseline), with the same metric.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import aeb_inputs as ai  # noqa: E402

METRIC = "rollouts/sec FP32-comp vs FP64 plain on 1 GB300; p99 request latency vs 530 ms"
UNIT = "rollouts/s"
# Algorithmic binary64 operations (add, subtract, multiply) of one RK4 step of
# the per-axle model in the plain definition: actuator 21, four accelerations
# 4 x 8, three stage speeds 6, position and speed updates 7 + 7.  min and
# comparisons are not counted.
FLOPS_PER_STEP = 73
SMS, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 80.5
FP64_PEAK_TFLOPS = 1.25  # GB300 dense FP64, nominal
# DRAM bytes per sample of the FP32 rollout kernel, from one ncu capture at
# N = 2e6 (199.7 MB per launch); traffic grows in proportion to the samples.
FP32_TRAFFIC_BYTES_PER_SAMPLE = 199.657728e6 / 2e6
# thread instructions the FP32 kernel executes per RK4 lane-step on this
# workload (ncu smsp__inst_executed x thread_inst_executed_per_inst_executed at
# N = 2e6, same profile); the issue-slot view of the roofline
FP32_THREAD_INST_PER_STEP = 22.46
FP32_ISSUE_PEAK = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6  # lane-instructions/s


EXTRAS = ("grid", "sweep", "dt", "c1", "lead", "perception", "rare")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--ttc-thr", type=float, default=None,
                    help="brake on the TTC trigger at this threshold (s) instead of "
                         "immediately (same samples; for profiling the TTC kernel)")
    ap.add_argument("--perception", action="store_true",
                    help="with --ttc-thr: per-step readings (1 m noise, 20 %% dropout, 50 ms "
                         "latency), as in the perception line (for profiling its kernel)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--c1-full", action="store_true",
                    help="run the binary64 kernel at every N x dt cell of the N sweep")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra lines (grid, sweep, dt study, N x dt, moving lead, "
                         "perception, rare event)")
    ap.add_argument("--extras", default=",".join(EXTRAS),
                    help="comma-separated extra lines to run (default: all of "
                         + ",".join(EXTRAS) + ")")
    args = ap.parse_args()
    args.extras = set() if args.no_extras else {e for e in args.extras.split(",") if e}
    unknown = args.extras - set(EXTRAS)
    if unknown:
        ap.error(f"unknown --extras {sorted(unknown)}; choose from {','.join(EXTRAS)}")
    return args


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.t.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4)
                          if r[3 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline_configs(cores: int):
    """The oracle on bounded samples of the batched-grid and TTC-sweep workloads
    (all host cores): every 64th grid scenario with its first 500 samples, and 8
    thresholds x 8 sweep scenarios x 500 samples."""
    import oracle
    res = {}
    m = ai.single_model()
    grid = ai.grid_scenarios(seed=2)[::64]
    parts = [oracle.sample(m, sc, 0, min(n, 500)) for sc, n in grid]
    p = {f: np.concatenate([q[f] for q in parts]) for f in ai.FIELDS}
    n = len(p["v0"])
    t0 = time.perf_counter()
    oracle.rollout(m, p, threads=cores)
    dt = time.perf_counter() - t0
    res["batched_grid"] = {"value": n / dt, "unit": UNIT,
                           "sample": f"{len(grid)} grid scenarios x <= 500 samples ({n} rollouts), "
                                     f"{dt:.2f} s on {cores} threads"}
    mt = ai.ttc_model()
    scen = ai.ttc_scenarios(64, seed=4)[::8]
    thr = ai.ttc_thresholds(256)[::32]
    ps = [oracle.sample(mt, sc, 0, 500) for sc in scen]
    q = {f: np.concatenate([x[f] for x in ps]) for f in ai.FIELDS}
    t0 = time.perf_counter()
    total = 0
    for th in thr:
        oracle.rollout(ai.replace(mt, ttc_thr=float(th)), q, threads=cores)
        total += len(q["v0"])
    dt = time.perf_counter() - t0
    res["ttc_sweep"] = {"value": total / dt, "unit": UNIT,
                        "sample": f"{len(thr)} thresholds x {len(scen)} scenarios x 500 samples "
                                  f"({total} rollouts), {dt:.2f} s on {cores} threads"}
    return res


def cpu_baseline(model, scenario, n_sample: int, configs: bool = False):
    """The oracle as it stands, on all host cores, on the first n_sample samples
    of the workload (the same sampler stream); extrapolated per rollout.  With
    ``configs``, also on samples of the batched-grid and TTC-sweep workloads."""
    import oracle
    cores = os.cpu_count() or 1
    p = oracle.sample(model, scenario, 0, n_sample)
    t0 = time.perf_counter()
    out = oracle.rollout(model, p, threads=cores)
    dt = time.perf_counter() - t0
    steps = int(out["n_steps"].astype(np.int64).sum())
    # the same oracle on one thread, on 1/cores of the sample
    n1 = max(1, n_sample // cores)
    t1 = time.perf_counter()
    oracle.rollout(model, {f: v[:n1] for f, v in p.items()}, threads=1)
    dt1 = time.perf_counter() - t1
    line = {"value": n_sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample} of the N-sample workload (same seed), "
                      f"{steps} RK4 steps, {dt:.2f} s wall on {cores} threads",
            "steps_per_s": steps / dt,
            "single_thread": {"value": n1 / dt1, "unit": UNIT,
                              "sample": f"first {n1} samples, {dt1:.2f} s on 1 thread"}}
    if configs:
        line["configs"] = cpu_baseline_configs(cores)
    return line


def serve_run(aeb, m, seconds: float, rate: float):
    """Serving workload: Poisson requests (rate/s for `seconds`), one scenario
    each with grid-style means and a road class, N log-uniform in [1e3, 1e6];
    latency from submit to statistics ready, against the 530 ms Monte Carlo
    budget (Sec. VI-F)."""
    reqs = ai.request_stream(rate=rate, duration=seconds, seed=3)
    srv = aeb.Server(m, aeb.FP32_COMP, arena_rows=1 << 23, chunk_samples=1 << 18,
                     wave_samples=1 << 21, max_waves_in_flight=2, sampler_threads=0,
                     max_request_samples=1_000_000)
    try:
        for k in range(4):  # warm-up: module load, first waves
            srv.poll(srv.submit(ai.replace(reqs[k][1], scenario_id=10_000 + k), 100_000))
        c0 = srv.counters()
        t0 = time.perf_counter()
        tickets = []
        for ta, sc, n in reqs:
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(sc, n))
        lat, rollouts = [], 0
        for tk in tickets:
            code, st, lt = srv.poll(tk)
            if code != aeb.OK:
                raise RuntimeError(f"serving request failed: {code}")
            lat.append(lt.total_ms)
            rollouts += st.n
        wall = time.perf_counter() - t0
        c1 = srv.counters()
    finally:
        srv.close()
    lat = np.array(lat)
    q = lambda p: float(np.quantile(lat, p, method="inverted_cdf"))
    return {"requests": len(lat), "duration_s": seconds, "rate_per_s": rate,
            "p50_ms": q(0.5), "p99_ms": q(0.99), "p999_ms": q(0.999), "max_ms": float(lat.max()),
            "budget_ms": 530.0, "p99_within_budget": q(0.99) < 530.0,
            "rollouts": int(rollouts), "rollouts_per_s": rollouts / wall,
            "offered_rollouts_per_s": rollouts / seconds, "waves": int(c1.waves - c0.waves),
            "precision": "fp32-compensated",
            "note": "rollouts_per_s is bounded by the offered load, not by the GPU"}


def batched_run(aeb, torch, dev, stream):
    """The scenario-grid workload: 4,096 scenarios (16 x 16 x 16 means) with
    per-scenario N log-uniform in [1e3, 6.4e4] (~6e7 rollouts), FP32-compensated,
    one captured graph per run (persistent launch + per-scenario reductions)."""
    m = ai.single_model()
    grid = ai.grid_scenarios(seed=2)
    total = sum(n for _, n in grid)
    host = aeb.alloc_params(total, device="cpu", pin=True)
    off = 0
    jobs = []
    for k, (sc, n) in enumerate(grid):
        aeb.aeb_sample_params(m, sc, 0, n, {f: host[f][off:off + n] for f in ai.FIELDS})
        jobs.append((off, off, n, 0.0))
        off += n
    P = {f: host[f].to(dev, non_blocking=True) for f in ai.FIELDS}
    O = aeb.alloc_outputs(total, device=dev, which=("status", "x_ref", "v_imp", "n_steps"))
    S = torch.empty(aeb.JOB_STATS_BYTES * len(jobs), dtype=torch.uint8, device=dev)
    plan = aeb.BatchPlan(m, jobs, P, aeb.FP32_COMP, O, S)
    plan.run(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        plan.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.close()
    ms = e0.elapsed_time(e1) / reps
    st = aeb.job_stats_from_buffer(S, len(jobs))
    assert sum(j.n for j in st) == total
    return {"scenarios": len(jobs), "rollouts": int(total), "ms_per_run": ms,
            "rollouts_per_s": total / (ms / 1e3), "launch": "one CUDA graph per run",
            "precision": "fp32-compensated"}


def sweep_run(aeb):
    """TTC-threshold sweep: 256 thresholds in [0.5, 4.0] s x 64 scenarios x
    1e5 samples (~1.64e9 rollouts), FP32-compensated, through aeb_ttc_sweep
    (host sampling, upload, batched launches, pooled Wilson intervals)."""
    m = ai.ttc_model()
    scen = ai.ttc_scenarios(64, seed=4)
    thr = ai.ttc_thresholds(256)
    t0 = time.perf_counter()
    res = aeb.aeb_ttc_sweep(m, scen, 100_000, thr, aeb.FP32_COMP)
    dt = time.perf_counter() - t0
    total = sum(r.n for r in res)
    pick = {f"{r.threshold:.2f}": [r.p_contact, r.ci_lo, r.ci_hi] for r in res[::51]}
    # per-threshold error against a binary64 rerun of a 1e6-sample subset (the first
    # 61 samples of each scenario at every threshold; the binary64 counts equal the
    # CPU oracle's, which the GPU tests check)
    sub = 61
    r64 = aeb.aeb_ttc_sweep(m, scen, sub, thr, aeb.FP64_PLAIN)
    r32 = aeb.aeb_ttc_sweep(m, scen, sub, thr, aeb.FP32_COMP)
    flips = [abs(a.n_contact - b.n_contact) for a, b in zip(r64, r32)]
    return {"rollouts": int(total), "seconds": dt, "rollouts_per_s": total / dt,
            "p_contact_ci95_at": pick, "precision": "fp32-compensated",
            "fp64_subset": {"rollouts": int(sum(r.n for r in r64)),
                            "max_contact_count_diff_per_threshold": int(max(flips)),
                            "thresholds_with_a_diff": int(sum(f > 0 for f in flips)),
                            "max_abs_p_contact_err": max(abs(a.p_contact - b.p_contact)
                                                         for a, b in zip(r64, r32))}}


def c1_sweep(aeb, torch, full: bool):
    """Throughput of both rollout kernels on the single-scenario workload at
    N = 1e3 ... 1e7 samples and dt = 1 ms and 0.1 ms (the first N samples of one
    seeded stream).  Per cell: CUDA-event time of one launch (mean of the timed
    repeats after one warm-up launch) and rollouts/s.  The binary64 kernel runs
    the cells of at most ~1e6 samples at 1 ms (~0.5 s each) unless ``full``;
    its N = 1e7, 1 ms cell is the headline's binary64 arm."""
    sizes = (1_000, 10_000, 100_000, 1_000_000, 10_000_000)
    sc = ai.single_scenario(seed=0)
    p = aeb.aeb_sample_params(ai.single_model(), sc, 0, sizes[-1])
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(sizes[-1], which=("status", "x_ref", "v_imp"))
    del p

    def timed(m, n, prec):
        Pn = {f: P[f][:n] for f in ai.FIELDS}
        On = {k: v[:n] for k, v in O.items()}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aeb.aeb_rollout(m, Pn, n, prec, On)
        e1.record()
        torch.cuda.synchronize()
        first = e0.elapsed_time(e1)
        reps = 5 if first < 50 else (2 if first < 2000 else 1)
        e0.record()
        for _ in range(reps):
            aeb.aeb_rollout(m, Pn, n, prec, On)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return {"ms": ms, "rollouts_per_s": n / (ms / 1e3), "repeats": reps}

    cells = []
    for dt in (1e-3, 1e-4):
        m = ai.single_model(dt=dt)
        for n in sizes:
            c = {"dt_ms": dt * 1e3, "n": n, "fp32_comp": timed(m, n, aeb.FP32_COMP)}
            if full or n * (1e-3 / dt) <= 1_000_000:
                c["fp64_plain"] = timed(m, n, aeb.FP64_PLAIN)
                c["fp32_over_fp64"] = c["fp32_comp"]["rollouts_per_s"] / c["fp64_plain"]["rollouts_per_s"]
            cells.append(c)
    del P, O
    return {"workload": "single scenario (config-0 distributions), first N samples of one stream",
            "timing": "one warm-up launch, then the mean of 1-5 launches (CUDA events)",
            "cells": cells}


def dt_study(aeb, torch):
    """Coarse-step fidelity and speed: the same 1e6 samples of the single-scenario
    workload rolled out (FP32-compensated) at dt = 0.1 ms (the reference) and at
    0.5 to 20 ms.  Per dt: launch time, rollouts/s, P(contact), mean stopping
    distance, mean impact speed, and against the reference the share of samples
    whose outcome (stop / contact) changed and the stopping-distance and
    impact-speed differences of samples with the same outcome.  The brake onset
    is quantised to the step (n dt >= t_delay), so part of the error is O(dt)."""
    N = 1_000_000
    sc = ai.single_scenario(seed=0)
    p = aeb.aeb_sample_params(ai.single_model(), sc, 0, N)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    which = ("status", "x_ref", "v_imp", "n_steps")
    res, ref = [], None
    for dt in (1e-4, 5e-4, 1e-3, 2e-3, 5e-3, 1e-2, 2e-2):
        m = ai.single_model(dt=dt)
        O = aeb.alloc_outputs(N, which=which)
        aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        o = {k: v.cpu().numpy() for k, v in O.items()}
        stop, cont = o["status"] == 0, o["status"] == 1
        row = {"dt_ms": dt * 1e3, "ms": ms, "rollouts_per_s": N / (ms / 1e3),
               "steps_per_rollout": float(o["n_steps"].mean()),
               "p_contact": float(cont.mean()), "mean_d_stop_m": float(o["x_ref"][stop].mean()),
               "mean_v_imp_mps": float(o["v_imp"][cont].mean())}
        if ref is None:
            ref = o
        else:
            bs = stop & (ref["status"] == 0)
            bc = cont & (ref["status"] == 1)
            dd = np.abs(o["x_ref"][bs] - ref["x_ref"][bs])
            dv = np.abs(o["v_imp"][bc] - ref["v_imp"][bc])
            row.update({"outcome_changed": float((o["status"] != ref["status"]).mean()),
                        "d_stop_abs_err_mean_m": float(dd.mean()),
                        "d_stop_abs_err_max_m": float(dd.max()),
                        "v_imp_abs_err_mean_mps": float(dv.mean()),
                        "p_contact_err": row["p_contact"] - float((ref["status"] == 1).mean())})
        res.append(row)
        del O
    return {"samples": N, "reference_dt_ms": 0.1, "precision": "fp32-compensated", "by_dt": res}


def moving_lead_run(aeb, torch):
    """Moving lead: 1e7 samples with a short headway, d0 ~ U(12, 40) m, behind a
    lead at 50 km/h that brakes at 6 m/s^2 from t = 0 (FP32-compensated, one
    launch after a warm-up, device-resident parameters), with P(contact) and
    the mean closing speed at impact."""
    N = 10_000_000
    m = ai.lead_braking_model()
    p = aeb.aeb_sample_params(m, ai.lead_braking_scenario(seed=0), 0, N)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(N, which=("status", "x_ref", "v_imp", "n_steps"))
    aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    S = aeb.alloc_stats()
    aeb.aeb_reduce(O, N, aeb.hist_spec(), S)
    st = aeb.stats_from_buffer(S)
    del P, O
    return {"samples": N, "ms": ms, "rollouts_per_s": N / (ms / 1e3),
            "steps_per_rollout": st.steps / N, "p_contact": st.n_contact / st.n,
            "mean_closing_speed_at_impact_mps": st.sum_v / max(st.n_contact, 1),
            "lead": {"v0_mps": m.lead_v0, "decel_mps2": m.lead_decel},
            "precision": "fp32-compensated"}


def perception_run(aeb, torch):
    """Per-step perception of the TTC trigger: 2e6 samples of the single-scenario
    distributions, TTC threshold 2 s, with readings carrying 1 m of noise,
    missing with probability 0.2 and 50 ms old, against the plain trigger on the
    same samples (FP32-compensated; time per launch and P(contact))."""
    N = 2_000_000
    base = ai.ttc_model(thr=2.0)
    p = aeb.aeb_sample_params(base, ai.single_scenario(seed=0), 0, N)
    P = {f: torch.from_numpy(p[f]).cuda() for f in ai.FIELDS}
    O = aeb.alloc_outputs(N, which=("status", "x_ref", "v_imp", "n_steps"))
    out = {}
    for name, m in (("plain", base),
                    ("perception", ai.replace(base, **PERCEPTION))):
        aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        S = aeb.alloc_stats()
        aeb.aeb_reduce(O, N, aeb.hist_spec(), S)
        st = aeb.stats_from_buffer(S)
        out[name] = {"ms": ms, "rollouts_per_s": N / (ms / 1e3), "p_contact": st.n_contact / st.n,
                     "steps_per_rollout": st.steps / N}
    del P, O
    return {"samples": N, "ttc_thr_s": 2.0,
            "readings": {"sigma_m": 1.0, "drop": 0.2, "latency_s": 0.05}, **out,
            "precision": "fp32-compensated"}


def rare_event_run(aeb, torch):
    """Rare-event estimation for the paper preset (Eq. 11-15): P(D_stop > 135 m)
    by plain Monte Carlo on 1e7 nominal samples and by importance sampling on
    1e6 samples of a proposal (faster cars, lower friction, downhill) with
    likelihood-ratio weights (FP32-compensated rollouts, device-resident inputs;
    the time is the rollout plus the reduction).  The variance reduction is
    p (1 - p) over the weighted estimator's variance per sample."""
    import math
    m = ai.paper_model()
    nominal = ai.paper_scenario(seed=11)
    h0 = 135.0
    res = {}
    for name, n in (("plain", 10_000_000), ("importance", 1_000_000)):
        if name == "plain":
            cols = aeb.aeb_sample_params(m, nominal, 0, n)
            w = np.ones(n)
        else:
            cols, w = aeb.aeb_sample_params_is(m, nominal, ai.rare_event_proposal(nominal), 0, n)
        P = {f: torch.from_numpy(cols[f]).cuda() for f in ai.FIELDS}
        W = torch.from_numpy(w).cuda()
        O = aeb.alloc_outputs(n, which=("status", "x_ref"))
        S = torch.zeros(aeb.WSTATS_BYTES, dtype=torch.uint8, device="cuda")
        aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aeb.aeb_rollout(m, P, n, aeb.FP32_COMP, O)
        aeb.aeb_reduce_weighted(O, W, n, h0, S)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = aeb.aeb_is_estimate(aeb.wstats_from_buffer(S))
        res[name] = {"samples": n, "ms": ms, "p": r.p, "se": r.se, "ci95": [r.ci_lo, r.ci_hi]}
        del P, W, O
    pl, im = res["plain"], res["importance"]
    p_ref = pl["p"]
    vr = p_ref * (1 - p_ref) / (im["se"] ** 2 * im["samples"]) if im["se"] > 0 else None
    # time to reach the same standard error: t * se^2 scales as 1 / samples
    speedup = (pl["ms"] * pl["se"] ** 2) / (im["ms"] * im["se"] ** 2) if im["se"] > 0 else None
    return {"event": "D_stop > 135 m (paper preset, no lead)", **res,
            "variance_reduction_per_sample": vr, "time_to_equal_se_speedup": speedup,
            "z_between_estimates": (im["p"] - pl["p"]) / math.hypot(im["se"], pl["se"]),
            "precision": "fp32-compensated"}


def fp32_error_table(aeb, torch, O32, O64, st32, st64):
    """FP32-compensated outputs against the binary64 ones on the same samples
    (the bounds of the parity tests, measured over the whole launch): per-sample
    errors of every output on the device (reading only) and the moments of the
    two reductions."""
    s32, s64 = O32["status"], O64["status"]
    same = s32 == s64
    stop = same & (s64 == 0)
    cont = same & (s64 == 1)
    x64 = O64["x_ref"][stop]
    rel = ((O32["x_ref"][stop] - x64).abs() / x64.abs().clamp_min(1e-3))
    ns_eq = same & (O32["n_steps"] == O64["n_steps"])
    xr64 = O64["x_raw"][ns_eq]
    xr_rel = ((O32["x_raw"][ns_eq] - xr64).abs() / xr64.abs().clamp_min(1e-3))
    dte = (O32["t_end"][stop] - O64["t_end"][stop]).abs()
    dvi = (O32["v_imp"][cont] - O64["v_imp"][cont]).abs()
    a, b = aeb.aeb_stats_summary(st32), aeb.aeb_stats_summary(st64)
    f = lambda t: float(t.max()) if t.numel() else 0.0
    return {
        "samples": int(s64.numel()),
        "flag_disagree": int((~same).sum()),
        "onset_disagree": int((O32["n_onset"] != O64["n_onset"]).sum()),
        "n_steps_disagree": int((same & (O32["n_steps"] != O64["n_steps"])).sum()),
        "x_ref_rel_max": f(rel), "x_ref_rel_mean": float(rel.mean()) if rel.numel() else 0.0,
        "x_raw_rel_max": f(xr_rel),
        "stop_t_end_abs_max_s": f(dte), "v_imp_abs_max_mps": f(dvi),
        "sum_d_rel": abs(st32.sum_d - st64.sum_d) / abs(st64.sum_d),
        "mean_d_rel": abs(a.mean_d - b.mean_d) / abs(b.mean_d),
        "std_d_rel": abs(a.std_d - b.std_d) / abs(b.std_d),
        "mean_v_rel": abs(a.mean_v - b.mean_v) / abs(b.mean_v) if b.n_contact else None,
        "p_contact_abs": abs(a.p_contact - b.p_contact),
        "bounds": "x_ref, x_raw <= 1e-5 relative; flags only where |gap| < 1e-3 m; "
                  "moments follow (parity tests)"}


def pooled_stats(aeb, torch, dist, S, world, dev):
    """The exchange step of a sharded run: every rank's fixed-size statistics,
    all-gathered and merged in rank order with aeb_stats_merge (counts and
    histograms exact; the same bits every run)."""
    if dist:
        parts = [torch.empty_like(S) for _ in range(world)]
        dist.all_gather(parts, S)
    else:
        parts = [S]
    acc = aeb.empty_stats(aeb.hist_spec())
    for part in parts:
        aeb.aeb_stats_merge(acc, aeb.stats_from_buffer(part))
    sm = aeb.aeb_stats_summary(acc)
    lo, hi = aeb.aeb_hist_quantile(acc, 0.99)
    return {"ranks": world, "n": int(sm.n), "n_contact": int(sm.n_contact),
            "n_stop": int(sm.n_stop), "p_contact": sm.p_contact,
            "p_contact_ci95": [sm.p_contact_lo, sm.p_contact_hi],
            "mean_d_m": sm.mean_d, "std_d_m": sm.std_d, "d_stop_q99_bin_m": [lo, hi],
            "how": "all_gather of aeb_stats, aeb_stats_merge in rank order"}


PERCEPTION = dict(perc_sigma=1.0, perc_drop=0.2, perc_latency=0.05, perc_seed=1)


def model_of(args):
    if args.ttc_thr is not None:
        m = ai.ttc_model(thr=args.ttc_thr, dt=args.dt)
        return ai.replace(m, **PERCEPTION) if args.perception else m
    return ai.single_model(dt=args.dt)


def config(args, world, precision="fp32-compensated"):
    trig = "immediate trigger" if args.ttc_thr is None else f"TTC trigger at {args.ttc_thr:g} s"
    if args.ttc_thr is not None and args.perception:
        trig += " with per-step readings (1 m noise, 20 % dropout, 50 ms latency)"
    return {"workload": f"single scenario, N={args.n} samples per GPU, dt={args.dt * 1e3:g} ms, "
                        f"10 s horizon, lead at d0, per-axle caps, {trig}",
            "n_samples_per_gpu": args.n, "dt_s": args.dt, "precision": precision,
            "l2": "inputs 800 MB per GPU > 129 MB L2, no flush",
            "parallelism": f"replicas x{world} (independent sample shards)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    m = model_of(args)
    sc = ai.single_scenario(seed=0)
    import oracle
    cores = os.cpu_count() or 1
    n_step = max(1000, args.cpu_sample // 2)
    p = oracle.sample(m, sc, 0, n_step)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.rollout(m, {f: v[:2000] for f, v in p.items()}, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rollout(m, p, threads=cores)
    dt = time.perf_counter() - t0
    v = n_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config(args, world, precision="binary64 CPU oracle (plain definition)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_step} samples of the workload per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2604_27193_gb300 as aeb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    aeb.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    N = args.n
    m = model_of(args)
    sc = ai.replace(ai.single_scenario(seed=0), scenario_id=rank)  # each rank its own shard

    # host sampling into pinned buffers, then resident device copies
    t0 = time.perf_counter()
    host = aeb.alloc_params(N, device="cpu", pin=True)
    aeb.aeb_sample_params(m, sc, 0, N, host)
    t_sample = time.perf_counter() - t0
    P = {f: host[f].to(dev, non_blocking=True) for f in ai.FIELDS}
    O = aeb.alloc_outputs(N, device=dev, which=("status", "x_ref", "v_imp", "n_steps"))
    S = aeb.alloc_stats(dev)
    hist = aeb.hist_spec()
    torch.cuda.synchronize()

    def step(prec):
        aeb.aeb_rollout(m, P, N, prec, O, stream)
        aeb.aeb_reduce(O, N, hist, S, stream)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---- headline: FP32-compensated step -------------------------------
    for _ in range(args.warmup):
        step(aeb.FP32_COMP)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for e0, e1, e2 in ev:
            e0.record(stream)
            aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O, stream)
            e1.record(stream)
            aeb.aeb_reduce(O, N, hist, S, stream)
            e2.record(stream)
        end.record(stream)
        barrier()
    ms_total = max_over_ranks(start.elapsed_time(end))
    roll_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1, _ in ev)
    red_ms = statistics.mean(e1.elapsed_time(e2) for _, e1, e2 in ev)
    st = aeb.stats_from_buffer(S)
    steps_per_launch = int(st.steps)
    value = world * N * args.steps / (ms_total / 1e3)
    achieved = steps_per_launch * FLOPS_PER_STEP / (roll_ms / 1e3) / 1e12

    # ---- end to end through the public host-buffer call ------------------
    # (right after the headline, before the binary64 arm's seconds at full power)
    aeb.aeb_evaluate(m, host, N, aeb.FP32_COMP, hist, stream=stream)  # sizes the buffers
    barrier()
    e2e_steps = max(2, min(args.steps, 5))
    with ClockSampler(local) as clk_e2e:
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            aeb.aeb_evaluate(m, host, N, aeb.FP32_COMP, hist, stream=stream)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
    # the box's pinned host-to-device copy rate (outside the timed region): the
    # e2e figure hides the uploads behind the rollouts only while they are fast
    # enough (growing chunks, each uploaded during the previous one's rollouts)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for f in ai.FIELDS:
        P[f].copy_(host[f], non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 8 * len(ai.FIELDS) * N / (c0.elapsed_time(c1) / 1e3) / 1e9
    e2e = {"value": world * N * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * len(ai.FIELDS) * N, "d2h_bytes_per_step": aeb.STATS_BYTES,
           "api": "aeb_evaluate (pinned host params -> host stats)",
           "h2d_copy_gbs": h2d_gbs, "clocks": clk_e2e.summary()}
    # ---- FP64 plain on the same samples ----------------------------------
    pooled = pooled_stats(aeb, torch, dist, S, world, dev)
    fp64 = None
    if not args.no_fp64:
        # the binary64 step writes every output, so that the FP32 error can be
        # stated for each; one untimed FP32 launch gives the FP32 side
        O64 = aeb.alloc_outputs(N, device=dev)
        S64 = aeb.alloc_stats(dev)

        def step64():
            aeb.aeb_rollout(m, P, N, aeb.FP64_PLAIN, O64, stream)
            aeb.aeb_reduce(O64, N, hist, S64, stream)

        step64()
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.fp64_steps):
            step64()
        s1.record(stream)
        barrier()
        ms64 = max_over_ranks(s0.elapsed_time(s1)) / args.fp64_steps
        O32 = aeb.alloc_outputs(N, device=dev)
        S32 = aeb.alloc_stats(dev)
        aeb.aeb_rollout(m, P, N, aeb.FP32_COMP, O32, stream)
        aeb.aeb_reduce(O32, N, hist, S32, stream)
        torch.cuda.synchronize()
        err = fp32_error_table(aeb, torch, O32, O64, aeb.stats_from_buffer(S32),
                               aeb.stats_from_buffer(S64))
        del O32, O64, S32, S64
        fp64 = {"value": world * N / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "steps": args.fp64_steps, "warmup": 1, "dtype": "f64",
                "achieved_tflops": steps_per_launch * FLOPS_PER_STEP / (ms64 / 1e3) / 1e12,
                "peak_tflops_nominal": FP64_PEAK_TFLOPS,
                "note": "no fused multiply-add on this path: its bound is the binary64 "
                        "add/multiply rate (measured_pipe_peaks.fp64_add_tops)",
                "fp32_error": err}

    # the same, from the seed: host sampling (all host threads) inside the
    # step, each chunk drawn while the previous one uploads and rolls out
    t1 = time.perf_counter()
    aeb.aeb_sample_params(m, sc, 0, N, host)
    ts = time.perf_counter() - t1  # the sampler alone, for the record
    aeb.aeb_evaluate_scenario(m, sc, 0, N, aeb.FP32_COMP, hist, stream=stream)  # staging
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        aeb.aeb_evaluate_scenario(m, sc, 0, N, aeb.FP32_COMP, hist, stream=stream)
    barrier()
    e2ws_s = max_over_ranks(time.perf_counter() - t0)
    e2e_sampling = {"value": world * N * e2e_steps / e2ws_s, "unit": UNIT,
                    "host_sampling_s_alone": ts, "host_threads": os.cpu_count(),
                    "h2d_bytes_per_step": 8 * len(ai.FIELDS) * N,
                    "d2h_bytes_per_step": aeb.STATS_BYTES,
                    "api": "aeb_evaluate_scenario (host sampling of each 2^20-sample chunk "
                           "overlapped with the upload and rollout of the one before)"}

    peaks = aeb.aeb_pipe_peaks(stream)
    if rank != 0:  # the remaining lines are single-GPU measurements, taken by rank 0
        if dist:
            dist.destroy_process_group()
        return
    # the serving run and the extra lines are single-GPU measurements: the N = 1
    # line carries them, a multi-GPU line only its own sharded numbers
    single = world == 1
    serving = None
    if single and args.serve_seconds > 0:
        serving = serve_run(aeb, m, args.serve_seconds, args.serve_rate)
    del P, O
    torch.cuda.empty_cache()
    batched = sweep = dts = moving = percep = rare = c1 = None
    if single:
        ex = args.extras

        def run(name, fn):
            if name not in ex:
                return None
            r = fn()
            torch.cuda.empty_cache()
            return r

        batched = run("grid", lambda: batched_run(aeb, torch, dev, stream))
        sweep = run("sweep", lambda: sweep_run(aeb))
        dts = run("dt", lambda: dt_study(aeb, torch))
        c1 = run("c1", lambda: c1_sweep(aeb, torch, args.c1_full))
        moving = run("lead", lambda: moving_lead_run(aeb, torch))
        percep = run("perception", lambda: perception_run(aeb, torch))
        rare = run("rare", lambda: rare_event_run(aeb, torch))

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config(args, world),
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "roofline": {"bound": "alu", "kernel": "k_rollout_fp32", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": FP32_TRAFFIC_BYTES_PER_SAMPLE * N if N >= 2_000_000 else None,
                     "traffic_source": "ncu dram__bytes_read+write of k_rollout_fp32 at N=2e6 "
                                       "(profiles/rollout_fp32_single_scenario_n2e6.md), "
                                       "scaled by samples",
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (unit counts, max clock)",
                     "flops_per_launch": steps_per_launch * FLOPS_PER_STEP,
                     "launch_ms": roll_ms,
                     "note": "flops counted from the 73-op binary64 definition of a step; the "
                             "kernel runs 18 binary32 instructions per step (12 FFMA, 2 paired "
                             "FFMA2, 4 FADD), so frac may exceed 1 without skipped work; "
                             "issue.frac is the headroom measure",
                     "issue": {"thread_inst_per_step": FP32_THREAD_INST_PER_STEP,
                               "achieved": steps_per_launch * FP32_THREAD_INST_PER_STEP
                                           / (roll_ms / 1e3),
                               "peak": FP32_ISSUE_PEAK, "unit": "lane-instructions/s",
                               "frac": steps_per_launch * FP32_THREAD_INST_PER_STEP
                                       / (roll_ms / 1e3) / FP32_ISSUE_PEAK}},
        "kernels_ms": {"rollout_fp32": roll_ms, "reduce": red_ms},
        "measured_pipe_peaks": {"fp32_fma_tflops": peaks[0], "fp64_fma_tflops": peaks[1],
                                "fp64_add_tops": peaks[2],
                                "how": "aeb_pipe_peaks: 8 independent FMA/add chains per thread"},
        "fp64_plain": fp64,
        "serving": serving,
        "batched_grid": batched,
        "ttc_sweep": sweep,
        "dt_study": dts,
        "n_dt_sweep": c1,
        "moving_lead": moving,
        "perception": percep,
        "rare_event": rare,
        "fp32_over_fp64": (value / fp64["value"]) if fp64 else None,
        "rk4_steps_per_s": world * steps_per_launch * args.steps / (ms_total / 1e3),
        "steps_per_rollout": steps_per_launch / N,
        "host_sampling_s": t_sample,
        "stats": {"n_stop": int(st.n_stop), "n_contact": int(st.n_contact),
                  "n_horizon": int(st.n_horizon), "p_contact": st.n_contact / st.n},
        "pooled": pooled,
        "e2e_with_sampling": e2e_sampling,
    }
    if single and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m, sc, args.cpu_sample, configs=not args.no_extras)
    # the whole headline metric in one compact block, last in the line
    head = {"fp32_comp_rollouts_per_s": value,
            "fp64_plain_rollouts_per_s": fp64["value"] if fp64 else None,
            "fp32_over_fp64": (value / fp64["value"]) if fp64 else None,
            "fp32_roofline_frac": achieved / FP32_PEAK_TFLOPS,
            "e2e_rollouts_per_s": e2e["value"],
            "e2e_with_sampling_rollouts_per_s": e2e_sampling["value"]}
    if fp64:
        e = fp64["fp32_error"]
        head["fp32_error"] = {k: e[k] for k in ("x_ref_rel_max", "x_raw_rel_max", "flag_disagree",
                                                "mean_d_rel", "std_d_rel", "mean_v_rel")}
    if serving:
        head["serving"] = {k: serving[k] for k in ("requests", "p50_ms", "p99_ms", "p999_ms",
                                                   "max_ms", "budget_ms", "p99_within_budget")}
    line["headline"] = head
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
