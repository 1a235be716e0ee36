"""Kernel-level timing of the FFA search (CUDA events on the launching stream).

    python -m paper_1703_05581_gb300.kernel_bench fold-score [--p0 P --m-data D --m M --widths W] [--reps R]
        times the fold of one base period (ffa_fold, all stages) and Algorithm 1 on
        its M profiles (ffa_score) on random FP32 data; default: the survey shapes
        P0 = 15625 / 20000 / 31249 (octave 0) and 15625 (octave 4).
    python -m paper_1703_05581_gb300.kernel_bench search [--workload survey|plain]
        one whole search with per-octave phase timings (preparation, fold + score).

Used for the ncu captures summarised under profiles/.
"""
from __future__ import annotations

import argparse
import ctypes as C
import time

import numpy as np
import torch

from . import ffa

SURVEY_SHAPES = [(15625, 4294, 8192, 12), (20000, 3355, 4096, 12), (31249, 2147, 4096, 13),
                 (15625, 268, 512, 12)]


def fold_score(p0: int, md: int, m: int, nw: int, reps: int, dev) -> None:
    z = torch.randn(md * p0 + 1, device=dev, dtype=torch.float32)
    plane = torch.empty((m, p0), device=dev)
    tmp = torch.empty_like(plane)
    widths = np.array([2 ** i for i in range(nw)], np.int32)
    rec = torch.empty((m, 4), dtype=torch.int32, device=dev)
    st = ffa.status_word(dev)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def fold():
        ffa._check(ffa._lib.ffa_fold(ffa._ptr(z), ffa.FOLD_F32, p0, md, m, ffa._ptr(plane),
                                     ffa._ptr(tmp), s))

    def score():
        ffa._check(ffa._lib.ffa_score(ffa._ptr(plane), ffa.FOLD_F32, m, p0,
                                      widths.ctypes.data_as(C.c_void_p), nw, ffa._ptr(rec),
                                      ffa._ptr(st), s))

    for f, name in ((fold, "fold"), (score, "score")):
        f()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        print(f"p0={p0} m_data={md} m={m} {name}: {ms:.3f} ms ({m * p0 / ms / 1e6:.2f} Gelem/s)",
              flush=True)


def search(workload: str, dev) -> None:
    import bench  # repository root on sys.path when run from there

    kw, n, make, _ = bench.workload(workload)
    plan = ffa.Plan(ffa.Config(**kw), n)
    x = torch.from_numpy(make(2)).to(dev)
    ws, rec, st = plan.workspace(dev), plan.records(dev), ffa.status_word(dev)
    ffa.timing_read()
    ffa.timing_enable(True)
    t0 = time.time()
    ffa.search(plan, x, workspace=ws, records=rec, status=st)
    ffa.wait(st)
    t1 = time.time()
    ffa.timing_enable(False)
    ms, _ = ffa.timing_read()
    print(f"search wall {t1 - t0:.3f} s, {plan.n_trials} trials, {plan.n_periods} base periods")
    print("prep ms per octave", np.round(ms[0][:plan.n_octaves], 3).tolist())
    print("fold+score ms per octave", np.round(ms[1][:plan.n_octaves], 3).tolist())


def main() -> None:
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("fold-score")
    a.add_argument("--p0", type=int)
    a.add_argument("--m-data", type=int)
    a.add_argument("--m", type=int)
    a.add_argument("--widths", type=int, default=12)
    a.add_argument("--reps", type=int, default=3)
    b = sub.add_parser("search")
    b.add_argument("--workload", default="survey", choices=["survey", "plain"])
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    if args.cmd == "fold-score":
        shapes = SURVEY_SHAPES if args.p0 is None else [(args.p0, args.m_data, args.m, args.widths)]
        for p0, md, m, nw in shapes:
            fold_score(p0, md, m, nw, args.reps, dev)
    else:
        search(args.workload, dev)


if __name__ == "__main__":
    main()
