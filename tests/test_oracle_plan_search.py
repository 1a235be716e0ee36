"""Pins for the oracle's search plan (Section 2.1 padding, Section 2.3 octaves)
and for the whole search on the plain 65 536-sample workload.

Plan pins: counts printed in the paper, reproduced from the plan with the
HTRU-S LowLat series shape assumed (2^26 samples of 64 us): about 10^8 trials
over 26 series for a 1-20 s search at D0 = 32, split about evenly between
1-2 s and 2-20 s (Section 4.1.2), and about 1.9 million profiles for a
1-10 s search at D0 = 64 (Section 5).
"""
import numpy as np
import pytest

from paper_1703_05581_gb300 import synth


def cfg_plain(orc, fold_type=0):
    ts = synth.PLAIN["tsamp"]
    return orc.Config(tsamp=ts, period_min=256 * ts, period_max=512 * ts,
                      widths=(1, 2, 4, 8, 16), fold_type=fold_type)


def test_plan_paper_counts(orc):
    n, ts = 1 << 26, 64e-6
    rows, nt, _ = orc.plan(orc.Config(tsamp=ts, period_min=1.0, period_max=20.0,
                                      downsample0=32), n)
    assert 0.8e8 < 26 * nt < 1.3e8
    per = orc.trial_periods(rows, orc.Config(tsamp=ts, period_min=1.0, period_max=20.0,
                                             downsample0=32))
    lo, hi = int(np.sum(per < 2.0)), int(np.sum(per >= 2.0))
    assert 4e7 < 26 * lo < 6.5e7 and 4e7 < 26 * hi < 6.5e7
    _, nt64, _ = orc.plan(orc.Config(tsamp=ts, period_min=1.0, period_max=10.0,
                                     downsample0=64), n)
    assert abs(nt64 - 1.9e6) < 0.1e6


def test_plan_bins_vary_by_two(orc):
    """n_bin = P0 ranges over [Pmin, 2 Pmin) within an octave (Section 4.1.2)."""
    rows, _, _ = orc.plan(orc.Config(tsamp=64e-6, period_min=1.0, period_max=20.0,
                                     downsample0=32), 1 << 26)
    for o in np.unique(rows["octave"]):
        p = rows["p0"][rows["octave"] == o]
        assert p.min() == rows["p0"].min() and p.max() < 2 * p.min()


def test_plan_plain_workload(orc):
    rows, nt, w = orc.plan(cfg_plain(orc), 65536)
    assert len(rows) == 256 and w == 1025
    assert list(rows["p0"][[0, -1]]) == [256, 511]
    m = dict(zip(rows["p0"].tolist(), rows["m_rows"].tolist()))
    assert all(m[p] == 256 for p in range(256, 509)) and all(m[p] == 128 for p in (509, 510, 511))
    assert nt == int(rows["m_rows"].sum())
    assert np.all(rows["m_data"] == 65536 // rows["p0"])


def test_plan_survey_workload(orc):
    cfg = orc.Config(tsamp=64e-6, period_min=1.0, period_max=30.0, duty=0.1)
    rows, nt, w = orc.plan(cfg, 1 << 26)
    assert w == 62501
    assert np.bincount(rows["octave"]).tolist() == [15625] * 4 + [13672]
    assert abs(nt - 1.294e8) < 0.01e8
    # widths: powers of two up to the first one above 10 % of P0
    r = rows[0]
    ws = r["widths"][: r["n_widths"]]
    assert ws[-1] > 0.1 * r["p0"] and ws[-2] <= 0.1 * r["p0"]


def test_trial_periods_eq2(orc):
    cfg = cfg_plain(orc)
    rows, nt, _ = orc.plan(cfg, 65536)
    per = orc.trial_periods(rows, cfg)
    ts = cfg.tsamp
    first = rows["first_trial"]
    assert np.allclose(per[first] / ts, rows["p0"])
    assert np.allclose(per[first + rows["m_rows"] - 1] / ts, rows["p0"] + 1)


def test_plain_search_finds_pulsar(orc):
    """0.8 s pulsar at 2.048 ms = 390.625 samples: P0 = 390, trial ~ 0.625 (M-1)."""
    x = synth.plain_series()
    cfg = cfg_plain(orc)
    rows, nt, _ = orc.plan(cfg, x.size)
    rec = orc.search(cfg, x, nthreads=4)
    b = orc.best(rec)
    i = int(np.searchsorted(rows["first_trial"], b, side="right") - 1)
    p0, k = int(rows["p0"][i]), b - int(rows["first_trial"][i])
    assert p0 == 390
    assert abs(k - 0.625 * (rows["m_rows"][i] - 1)) <= 2
    assert rec["width"][b] in (4, 8, 16)
    assert rec["snr"][b] > 9.0


def test_plain_search_f32_and_int_paths(orc):
    x = synth.plain_series()
    r64 = orc.search(cfg_plain(orc, 0), x, nthreads=4)
    r32 = orc.search(cfg_plain(orc, 1), x, nthreads=4)
    r8 = orc.search(cfg_plain(orc, 2), x, nthreads=4)
    assert np.max(np.abs(r32["snr"] - r64["snr"])) < 1e-3
    assert orc.best(r32) == orc.best(r64)
    # int8 (x16, rint) loses a little S/N but finds the same candidate region
    b8, b64 = orc.best(r8), orc.best(r64)
    assert abs(b8 - b64) <= 2
    assert np.corrcoef(r8["snr"], r64["snr"])[0, 1] > 0.98
