"""Serving workload: a Poisson stream of FFA searches through the
continuous-batching server (ffa_server_*), reporting p50/p99 latency beside
throughput.

Requests: lengths log-uniform in [2^20, 2^25] samples at 64 us; minimum
period log-uniform in [0.5 s, min(30 s, T_obs / 16)], maximum
min(60 s, P_min * 2^U{1..3}, T_obs / 8); half FP32, half int8; 5 % carry a
pulsar (period uniform in the range, FWHM 1-5 %, S/N 8-20); D0 is the
smallest power of two keeping P_min within 16384 bins.  Series are
slices of one pre-generated pinned noise buffer (distinct offsets), so that
generating them does not pace the stream.

    python -m paper_1703_05581_gb300.serve_bench [--rate 200] [--requests 48]
        [--budget-gb 120] [--slots 8] [--seed 5]

prints one JSON line.  At --rate 0 the requests arrive all at once
(capacity measurement).
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np
import torch

from . import ffa, synth

TSAMP = 64e-6


def make_requests(count: int, rate: float, seed: int, pool: np.ndarray):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        if rate > 0:
            t += float(rng.exponential(1.0 / rate))
        n = int(2 ** rng.uniform(20, 25))
        t_obs = n * TSAMP
        pmin = float(np.exp(rng.uniform(np.log(0.5), np.log(min(30.0, t_obs / 16)))))
        pmax = min(60.0, pmin * 2 ** int(rng.integers(1, 4)), t_obs / 8)
        off = int(rng.integers(0, pool.size - n))
        x = pool[off:off + n]
        if rng.random() < 0.05:
            x = x.copy()
            p = float(rng.uniform(pmin, pmax)) / TSAMP
            x += synth.gaussian_pulse_train(n, p, float(rng.uniform(0.01, 0.05)), float(rng.random()),
                                            float(rng.uniform(8.0, 20.0))).astype(np.float32)
        prec = ffa.FOLD_I8 if rng.random() < 0.5 else ffa.FOLD_F32
        # pre-downsampling: the smallest power of two keeping P_min within 16384 bins
        d0 = 1
        while pmin / (TSAMP * d0) > 16384:
            d0 *= 2
        cfg = ffa.Config(tsamp=TSAMP, period_min=pmin, period_max=pmax, precision=prec, downsample0=d0)
        out.append((t, cfg, x))
    return out


def units(cfg, n) -> float:
    e = ffa.Plan(cfg, n).entries
    return float(np.sum(e["m_data"].astype(np.float64) * e["p0"] * e["m_rows"]))


def profile_bins(cfg, n) -> float:
    """Folded-profile bins a request scores (M * P0 per base period): the
    work of the fold's last stage and of the scorer, whatever the rows."""
    e = ffa.Plan(cfg, n).entries
    return float(np.sum(e["p0"].astype(np.float64) * e["m_rows"]))


def run(rate: float, count: int, budget: int, slots: int, seed: int) -> dict:
    pool = torch.empty(1 << 26, dtype=torch.float32).pin_memory().numpy()
    pool[:] = np.random.default_rng(seed).standard_normal(pool.size, dtype=np.float32)
    reqs = make_requests(count, rate, seed + 1, pool)
    srv = ffa.Server(budget, n_slots=slots)
    tickets = [None] * len(reqs)
    peak_used = [0]
    done = threading.Event()

    def watch():
        while not done.is_set():
            peak_used[0] = max(peak_used[0], srv.stats()[2])
            time.sleep(0.01)

    def feed():
        t0 = time.perf_counter()
        for i, (ta, cfg, x) in enumerate(reqs):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(cfg, x, snr_min=8.0, top_k=16)

    wt = threading.Thread(target=watch, daemon=True)
    wt.start()
    t0 = time.perf_counter()
    ft = threading.Thread(target=feed)
    ft.start()
    lat, qd, runs = [], [], []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.001)
        _, _, _, tm = srv.wait(tickets[i])
        qd.append(tm[0])
        runs.append(tm[1])
        lat.append(tm[2])
    wall = time.perf_counter() - t0
    ft.join()
    done.set()
    srv.close()
    tot_units = sum(units(c, x.size) for _, c, x in reqs)
    tot_bins = sum(profile_bins(c, x.size) for _, c, x in reqs)
    lat = np.array(lat)
    return {
        "metric": "FFA serving latency", "offered_rate_req_s": rate, "requests": len(reqs),
        "slots": slots, "budget_bytes": budget, "peak_arena_bytes": int(peak_used[0]),
        "wall_s": wall, "throughput_req_s": len(reqs) / wall,
        "throughput_samples_trials_s": tot_units / wall,
        "throughput_profile_bins_s": tot_bins / wall,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean())},
        "queued_ms_p50": float(np.percentile(qd, 50)), "running_ms_p50": float(np.percentile(runs, 50)),
        "workload": "lengths 2^20-2^25 at 64 us, periods 0.5-60 s, half FP32 / half int8, 5 % pulsars",
    }


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps(run(a.rate, a.requests, int(a.budget_gb * (1 << 30)), a.slots, a.seed)), flush=True)


if __name__ == "__main__":
    main()
