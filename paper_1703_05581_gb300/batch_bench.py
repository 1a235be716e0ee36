"""Batched FP32 and int8 searches (the DM-trial batch) against each other and
against the FP64 oracle on sampled base periods.

    python -m paper_1703_05581_gb300.batch_bench [--series 16] [--check 2] [--seed 3]

Series follow the batch recipe (lengths uniform in [2^22, 2^23] at 512 us,
white + AR(1) red noise, 5 % with pulsars of 0.5-20 s, FWHM 1-5 %, S/N
8-20), searched from 0.5 to 20 s with duty 0.2.  Both precisions run through
ffa_search_batch (one workspace, series after series) and are timed with CUDA
events; prints one JSON line with each form's samples*trials/s, the best-trial
agreement and the S/N differences, and for `check` series the largest S/N
error of each form against the oracle's FP64 fold + Algorithm 1 on 8 sampled
trials of 4 base periods per octave.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from . import ffa, synth

KW = dict(tsamp=512e-6, period_min=0.5, period_max=20.0, duty=0.2)


def run(n_series: int, n_check: int, seed: int) -> dict:
    dev = torch.device("cuda", 0)
    specs = synth.batch_specs(n_series, 1 << 22, 1 << 23, seed)
    series = [synth.make_series(s) for s in specs]
    xs = [torch.from_numpy(x).to(dev) for x in series]
    out = {}
    recs = {}
    for name, prec in (("fp32", ffa.FOLD_F32), ("int8", ffa.FOLD_I8)):
        plans = [ffa.Plan(ffa.Config(**KW, precision=prec), x.size) for x in series]
        ws = torch.empty(max(p.workspace_bytes for p in plans), dtype=torch.uint8, device=dev)
        rr = [p.records(dev) for p in plans]
        st = ffa.status_word(dev)
        ffa.search_batch(plans[:1], xs[:1], workspace=ws, records=rr[:1], status=st)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ffa.search_batch(plans, xs, workspace=ws, records=rr, status=st)
        e1.record()
        ffa.wait(st)
        ms = e0.elapsed_time(e1)
        units = sum(float(np.sum(p.entries["m_data"].astype(np.float64) * p.entries["p0"] * p.entries["m_rows"]))
                    for p in plans)
        out[name] = {"ms": ms, "samples_trials_per_s": units / (ms / 1e3),
                     "input_bytes": int(sum(x.numel() * x.element_size() for x in xs))}
        recs[name] = (plans, [ffa.records_numpy(r, p.n_trials) for r, p in zip(rr, plans)])
    p32, r32 = recs["fp32"]
    _, r8 = recs["int8"]
    same_best = [int(np.argmax(a["snr"])) == int(np.argmax(b["snr"])) for a, b in zip(r32, r8)]
    d = np.concatenate([np.abs(a["snr"].astype(np.float64) - b["snr"]) for a, b in zip(r32, r8)])
    out["int8_vs_fp32"] = {"same_best_fraction": float(np.mean(same_best)),
                           "snr_abs_diff_median": float(np.median(d)),
                           "snr_abs_diff_p99": float(np.percentile(d, 99)),
                           "snr_abs_diff_max": float(d.max())}
    if n_check > 0:
        import oracle
        oracle.build()
        rng = np.random.default_rng(seed)
        err = {"fp32": 0.0, "int8": 0.0}
        for i in range(min(n_check, n_series)):
            ocfg = oracle.Config(**KW, fold_type=oracle.FOLD_F64)
            z = oracle.octave_series(ocfg, series[i])
            rows, _, _ = oracle.plan(ocfg, series[i].size)
            for o in np.unique(rows["octave"]):
                for ri in rng.choice(np.flatnonzero(rows["octave"] == o), 4, replace=False):
                    r = rows[ri]
                    p0, md, m = int(r["p0"]), int(r["m_data"]), int(r["m_rows"])
                    for k in rng.integers(0, m, 8):
                        ref = oracle.score_alg1(oracle.fold_trial(z[o], p0, md, m, int(k)),
                                                r["widths"][: r["n_widths"]])["snr"]
                        t = int(r["first_trial"]) + int(k)
                        err["fp32"] = max(err["fp32"], abs(float(r32[i]["snr"][t]) - float(ref)))
                        err["int8"] = max(err["int8"], abs(float(r8[i]["snr"][t]) - float(ref)))
        out["max_abs_snr_err_vs_fp64_oracle"] = err
    out["series"] = n_series
    out["workload"] = ("batch: lengths U[2^22, 2^23] at 512 us, white + AR(1) red noise, 5 % pulsars; "
                       "0.5-20 s, duty 0.2")
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--series", type=int, default=16)
    ap.add_argument("--check", type=int, default=2)
    ap.add_argument("--seed", type=int, default=3)
    a = ap.parse_args()
    print(json.dumps(run(a.series, a.check, a.seed)), flush=True)


if __name__ == "__main__":
    main()
