"""False-alarm statistics of the FFA search (Section 4.3).

Searches noise-only series with Algorithm 1 or 2, accumulates the S/N
histogram of every trial on the device (ffa_snr_histogram), maps each S/N to
its Gaussian-equivalent sigma (ffa_sigma_gauss: the fraction of trials at or
above it put through the upper-tail normal quantile), and reads the exact S/N
at a given sigma as an order statistic of all trials (the r-th largest, with
r = ceil(trials * Q(sigma)), gathered per series by ffa_candidates and merged).

    python -m paper_1703_05581_gb300.noise_stats [--series 26] [--scorer 1|2]

runs the paper's configuration (26 series of 2^26 samples at 64 us, D0 = 32,
1-20 s, about 10^8 trials), prints one JSON line per scorer.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import ffa, shard, synth

EDGES = np.round(np.arange(0.0, 40.0001, 0.05), 2).astype(np.float32)


def upper_tail(sigma: float) -> float:
    return 0.5 * math.erfc(sigma / math.sqrt(2.0))


def run(n_series: int = synth.NOISE["n_series"], n: int = synth.NOISE["n"],
        scorer: int = ffa.SCORE_ALG1, sigmas=(4.0, 5.0), seed0: int = synth.NOISE["seed"],
        dev=None, edges=EDGES, series=None) -> dict:
    """Search n_series white-noise series; return the histogram, the sigma of
    each edge and the exact S/N at each requested sigma."""
    dev = torch.device("cuda", 0) if dev is None else dev
    cfg = ffa.Config(tsamp=synth.NOISE["tsamp"], period_min=synth.NOISE["period_min_s"],
                     period_max=synth.NOISE["period_max_s"],
                     downsample0=synth.NOISE["downsample0"], scorer=scorer)
    plan = ffa.Plan(cfg, n)
    total = plan.n_trials * n_series
    ranks = {s: max(1, math.ceil(total * upper_tail(s))) for s in sigmas}
    top_k = max(ranks.values())
    if top_k > 4096:
        raise ValueError("too few trials for the requested sigmas")
    ws, rec, st = plan.workspace(dev), plan.records(dev), ffa.status_word(dev)
    counts = torch.zeros(len(edges) + 1, dtype=torch.int64, device=dev)
    lists = []
    t_gpu = 0.0
    for i in range(n_series):
        x = series(i) if series is not None else synth.white_series(seed0 + i, n)
        xd = torch.from_numpy(x).to(dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ffa.search(plan, xd, workspace=ws, records=rec, status=st)
        ffa.snr_histogram(rec, plan.n_trials, edges, counts)
        c, _ = ffa.candidates(plan, rec, ws, snr_min=-1e30, top_k=top_k, status=st)
        t_gpu += time.perf_counter() - t0
        c = c.copy()
        c["trial"] += i * plan.n_trials  # distinct keys across series
        lists.append(c)
    top = shard.merge_candidates(lists, top_k)
    h = counts.cpu().numpy().astype(np.uint64)
    return {"trials": int(total), "counts": h, "edges": np.asarray(edges),
            "sigma": ffa.sigma_gauss(h),
            "snr_at_sigma": {s: float(top["snr"][r - 1]) for s, r in ranks.items()},
            "ranks": ranks, "gpu_s": t_gpu}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--series", type=int, default=synth.NOISE["n_series"])
    ap.add_argument("--scorer", type=int, default=0, choices=[0, 1, 2],
                    help="1 or 2 for one algorithm, 0 for both")
    args = ap.parse_args()
    for sc in ([1, 2] if args.scorer == 0 else [args.scorer]):
        r = run(args.series, scorer=ffa.SCORE_ALG1 if sc == 1 else ffa.SCORE_ALG2)
        print(json.dumps({"algorithm": sc, "series": args.series, "trials": r["trials"],
                          "snr_at_sigma": r["snr_at_sigma"], "ranks": r["ranks"],
                          "gpu_s": round(r["gpu_s"], 3)}), flush=True)


if __name__ == "__main__":
    main()
