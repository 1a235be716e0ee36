#!/usr/bin/env python3
"""Benchmark of the GB300 FFA period search.

Workload (default ``survey``): one 2^26-sample float32 series at 64 us (white
noise + AR(1) red noise + a 7.3 s pulsar), searched over 1-30 s periods with
per-octave downsampling, the paper's default dereddening window and
Algorithm 1 widths up to 10 % duty.  One step = the whole search of one
series (downsampling, dereddening, normalisation, FFA fold and scoring of
every base period of every octave, candidate extraction).

Metric: FFA search rate in input samples x trials per second: for every base
period, (data rows x P0 samples folded) x (M trials produced), summed, per
second.  ``value`` is timed on the device with CUDA events, inputs already
resident; ``e2e`` times the same step through the public API from pinned
host memory (host->device copy of the series and device->host read of the
candidate list inside the timed region).

--impl reference times the CPU oracle (the plain FP64 implementation used
for parity) on a bounded sample of the same workload on the host cores.
Multi-GPU (--gpus N under torchrun): every rank searches its own series
(weak scaling); there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
METRIC = "FFA search rate (input samples*trials/s)"
UNIT = "samples*trials/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["survey", "plain"], default="survey")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-budget-s", type=float, default=20.0,
                    help="target CPU seconds of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(name: str):
    from paper_1703_05581_gb300 import synth
    if name == "survey":
        s = synth.SURVEY
        kw = dict(tsamp=s["tsamp"], period_min=s["period_min_s"], period_max=s["period_max_s"],
                  duty=s["duty"])
        desc = {"workload": "survey: 2^26 f32 samples at 64 us, white + AR(1) red noise, 7.3 s "
                            "pulsar; periods 1-30 s, 5 octaves, widths to 10% duty, exact "
                            "running-median dereddening (W=62501)",
                "n_samples": s["n"], "tsamp_s": s["tsamp"], "period_range_s": [1.0, 30.0]}
        return kw, s["n"], (lambda seed: synth.survey_series(seed=seed)), desc
    p = synth.PLAIN
    kw = dict(tsamp=p["tsamp"], period_min=256 * p["tsamp"], period_max=512 * p["tsamp"],
              widths=p["widths"])
    desc = {"workload": "plain: 65536 f32 samples at 2.048 ms, 0.8 s pulsar, P0 256..511, "
                        "widths 1-16", "n_samples": p["n"], "tsamp_s": p["tsamp"]}
    return kw, p["n"], (lambda seed: synth.plain_series(seed=seed)), desc


def plan_units(entries) -> float:
    e = entries
    return float(np.sum(e["m_data"].astype(np.float64) * e["p0"] * e["m_rows"]))


def fold_score_bytes(entries, in_bytes: int = 4) -> np.ndarray:
    """Algorithmic bytes of fold+score per octave: read the octave series once per
    base period (data rows x P0 samples) and write one 16-byte record per trial."""
    out = np.zeros(64)
    for o in np.unique(entries["octave"]):
        e = entries[entries["octave"] == o]
        out[o] = float(np.sum(in_bytes * e["m_data"].astype(np.float64) * e["p0"] + 16.0 * e["m_rows"]))
    return out


# GB300 FP32/INT32 lane peak for ALU-bound kernels: 152 SMs x 128 lanes x 2070 MHz
# (the maximum SM clock); one algorithmic operation per lane per clock.
ALU_LANES = 152 * 128
ALU_MAX_MHZ = 2070.0
# DRAM bytes per profile bin of one k_score2 launch (read + write), from the
# ncu capture summarised in profiles/k_score2_p0_20000_m4096.md:
# (329.25 MB + 11.89 MB) / (4096 * 20000).  Set to None when the kernel changes.
SCORE_DRAM_BYTES_PER_ELEM = (329247232 + 11889920) / (4096 * 20000)


def score_ops(entries) -> np.ndarray:
    """Algorithmic operations of one scoring launch (a base period's M trials):
    per bin, the fused last FFA stage's add, per width a box add and a max,
    one deviation |x - median|, and at least one comparison per bin for each of
    the two order-statistic selections (median, MAD)."""
    e = entries
    return e["m_rows"].astype(np.float64) * e["p0"] * (1.0 + 2.0 * e["n_widths"] + 3.0)


def sampled(entries, octave, sample):
    """Entries whose launches the library times: every sample-th of the octave."""
    idx = np.flatnonzero(entries["octave"] == octave)
    return entries[idx[::sample]]


def measured_peaks():
    if os.path.exists(PEAKS_PATH):
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        smax = np.array([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for i, nm in enumerate(names):
            if any(r[5 + i].lower() == "active" for r in rows):
                reasons.append(nm)
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(smax)),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def cpu_oracle_sample(kw, n, make, budget_s: float):
    """Time the oracle on a bounded sample of the workload and scale it to the
    metric.  Sample: the running-median dereddening of a 2^20-sample slice
    (scaled by the samples of every octave) plus the fold + scoring of a few
    base periods spread over the octaves (scaled by their share of the
    workload's samples x trials)."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    try:  # each base period folds in up to ~3 GB of host memory: bound the threads by it
        with open("/proc/meminfo") as f:
            avail_kb = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable"))
        threads = max(1, min(threads, int(avail_kb / (4 << 20))))
    except (OSError, StopIteration, ValueError):
        pass
    ocfg = oracle.Config(**{k: v for k, v in kw.items() if k != "widths"},
                         widths=kw.get("widths", ()), fold_type=oracle.FOLD_F64)
    rows, nt, win = oracle.plan(ocfg, n)
    total_units = plan_units(rows)
    x = make(7)
    # dereddening of a slice, single thread, scaled to every octave's samples
    sl = min(n, 1 << 20)
    raw = oracle.downsample(x[:sl], 1)
    t0 = time.perf_counter()
    if win > 1:
        oracle.running_median(raw, win)
    t_med = time.perf_counter() - t0
    n_oct = int(rows["octave"].max()) + 1
    all_samples = sum(n >> o for o in range(n_oct))
    t_detrend = t_med * all_samples / sl
    # fold + score: one base period per host thread, evenly spaced over the plan (so the
    # octaves are represented in proportion to their base periods), run in parallel
    idx = np.unique(np.linspace(0, rows.size - 1, min(threads, rows.size)).astype(int))
    sub = rows[idx]
    n_oct = int(rows["octave"].max()) + 1
    z = oracle.octave_series(ocfg, x[: n]) if n <= (1 << 22) else None
    if z is None:
        # the dereddened series themselves are not needed for timing: fold white noise
        z = [np.random.default_rng(o).standard_normal(n >> o) for o in range(n_oct)]
    t0 = time.perf_counter()
    oracle.fold_score_rows(oracle.FOLD_F64, z, sub, nthreads=threads)
    t_fs = time.perf_counter() - t0
    sample_units = plan_units(sub)
    t_total = t_fs * total_units / sample_units + t_detrend
    rate = total_units / t_total
    return {
        "value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
        "sample": (f"oracle (FP64) fold+Algorithm 1 of {sub.size} base periods spread over "
                   f"{n_oct} octaves ({sample_units:.3g} of {total_units:.3g} samples*trials, "
                   f"{t_fs:.1f} s on {threads} threads) plus the running median of a {sl}-sample "
                   f"slice ({t_med:.1f} s, 1 thread), both scaled to the whole workload"),
        "est_step_s": t_total,
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    kw, n, make, desc = workload(args.workload)
    per_step = max(5.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(kw, n, make, per_step)
        if i >= args.warmup:
            vals.append(r["value"])
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["est_step_s"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1703_05581_gb300 import ffa

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    kw, n, make, desc = workload(args.workload)
    cfg = ffa.Config(**kw)
    plan = ffa.Plan(cfg, n)
    x = make(int(synth_seed(args.workload)) + rank)
    x_pinned = torch.from_numpy(x).pin_memory()
    xs = x_pinned.to(dev)
    ws = plan.workspace(dev)
    rec = plan.records(dev)
    status = ffa.status_word(dev)
    stream = torch.cuda.Stream(dev)
    units = plan_units(plan.entries)
    fs_bytes = fold_score_bytes(plan.entries)

    def step():
        ffa.search(plan, xs, workspace=ws, records=rec, status=status, stream=stream)

    # fold pass depths tuned for this plan's shapes (untimed), then warm-up
    # (which also surfaces device-side check failures before timing)
    n_tuned = ffa.autotune(plan, ws, stream=stream)
    for _ in range(args.warmup):
        step()
    ffa.wait(status, stream=stream)
    cands, best = ffa.candidates(plan, rec, ws, snr_min=8.0, top_k=16, status=status,
                                 stream=stream)

    # timed region: device events on the launching stream
    sampler = ClockSampler(local)
    ffa.timing_read()  # clear
    ffa.timing_enable(True)
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    l0 = ffa.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    ev1.synchronize()
    launches = ffa.launch_count() - l0
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    ffa.timing_enable(False)
    phase_ms, phase_cnt = ffa.timing_read()
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    ffa.wait(status, stream=stream)

    # end to end through the public API from pinned host memory
    d2h = 0
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        with torch.cuda.stream(stream):
            xs.copy_(x_pinned, non_blocking=True)
        step()
        c, b = ffa.candidates(plan, rec, ws, snr_min=8.0, top_k=16, status=status, stream=stream)
        d2h += 1064 + 24 * len(c)  # control block + candidate entries copied back
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())

    if rank == 0:
        value = units * world * args.steps / (ms_max / 1e3)
        e2e_value = units * world * args.e2e_steps / e2e_s
        peak, peak_kind = measured_peaks()
        # fold + score phase: HBM view (algorithmic bytes of the search's fold+score)
        fs_ms = phase_ms[1]
        fs_cnt = np.maximum(phase_cnt[1], 1)
        oct_ms = fs_ms / fs_cnt
        tot_bytes = float(np.sum(fs_bytes[: len(oct_ms)] * (phase_cnt[1] > 0)))
        tot_ms = float(np.sum(oct_ms * (phase_cnt[1] > 0)))
        hbm_achieved = tot_bytes / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else 0.0
        prep_ms = float(np.sum(phase_ms[0] / np.maximum(phase_cnt[0], 1)))
        # dominant kernel: k_score2, timed per launch on sampled base periods
        sc_ops = sc_ms = sc_elems = sc_n = fo_ms = 0.0
        for o in range(plan.n_octaves):
            if phase_cnt[3][o] == 0:
                continue
            sub = sampled(plan.entries, o, ffa.TIMING_SAMPLE)
            reps = phase_cnt[3][o] / max(len(sub), 1)  # timed steps
            sc_ops += float(score_ops(sub).sum()) * reps
            sc_elems += float((sub["m_rows"].astype(np.float64) * sub["p0"]).sum()) * reps
            sc_ms += float(phase_ms[3][o])
            fo_ms += float(phase_ms[2][o])
            sc_n += float(phase_cnt[3][o])
        alu_peak = ALU_LANES * ALU_MAX_MHZ * 1e6 / 1e12
        alu_achieved = sc_ops / (sc_ms / 1e3) / 1e12 if sc_ms > 0 else 0.0
        traffic = (SCORE_DRAM_BYTES_PER_ELEM * sc_elems / sc_n
                   if SCORE_DRAM_BYTES_PER_ELEM and sc_n else None)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(desc, l2="inputs and fold planes larger than L2 (no flush needed)",
                           trials=int(plan.n_trials), base_periods=int(plan.n_periods),
                           autotuned_fold_shapes=int(n_tuned),
                           samples_x_trials=units),
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": alu_achieved / alu_peak, "traffic": traffic,
                         "kernel": "k_score2 (Algorithm 1 + fused last FFA stage), mean over "
                                   f"{int(sc_n)} sampled launches",
                         "ops": "per bin: last-stage add + 2 per width + 3 (selections, deviation)",
                         "peak_from": "152 SMs x 128 FP32/INT32 lanes x 2070 MHz",
                         "score_ms_per_launch": sc_ms / max(sc_n, 1),
                         "fold_ms_per_launch": fo_ms / max(sc_n, 1),
                         "hbm": {"achieved_gbs": hbm_achieved, "peak_gbs": peak, "peak_kind": peak_kind,
                                 "frac": hbm_achieved / peak,
                                 "bytes": "algorithmic: 4*M_data*P0 + 16*M per base period"},
                         "phase_ms_per_step": {"prep": prep_ms, "fold_score": tot_ms}},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": d2h // max(1, args.e2e_steps)},
            "gpu_launches": int(launches),
            "best_candidate": {"period_s": float(cands["period_s"][0]) if len(cands) else None,
                               "snr": float(cands["snr"][0]) if len(cands) else None},
        }
        if not args.no_cpu_baseline:
            cb = cpu_oracle_sample(kw, n, make, args.cpu_budget_s)
            cb.pop("est_step_s", None)
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def synth_seed(name: str) -> int:
    from paper_1703_05581_gb300 import synth
    return synth.SURVEY["seed"] if name == "survey" else synth.PLAIN["seed"]


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
