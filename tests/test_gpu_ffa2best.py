"""GPU parity of ffa2best (Section 2.3.3 candidate selection) against the
oracle: on the periodograms of real searches, and on synthetic periodograms
built to stress the chunked peak walk (long runs with no terminating record,
peaks on chunk boundaries, more peaks than the filter considers)."""
import os

import numpy as np
import pytest

from oracle import ffa2best as fb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05581_gb300 import ffa
    return ffa


@pytest.fixture(scope="module")
def dev():
    import torch
    return torch.device("cuda", 0)


def plain_cfg(F):
    from paper_1703_05581_gb300 import synth
    ts = synth.PLAIN["tsamp"]
    return F.Config(tsamp=ts, period_min=256 * ts, period_max=512 * ts, widths=(1, 2, 4, 8, 16))


def oracle_select(F, plan, rec_np, n_samples, tsamp, d0, th, sel_max=4096, cap=256):
    """The oracle's ffa2best on the same periodogram; when there are more
    peaks than the device filter considers, restricted to the strongest."""
    e = plan.entries
    per = np.concatenate([(int(r["p0"]) + np.arange(int(r["m_rows"])) / (int(r["m_rows"]) - 1))
                          * (tsamp * d0 * 2.0 ** int(r["octave"])) for r in e])
    p0s = np.repeat(e["p0"], e["m_rows"])
    t_obs = n_samples * tsamp
    snr = rec_np["snr"]
    pk = fb.peaks(snr, th["snr_min"], th["drop_frac"], th["drop_abs"])
    order = sorted(pk, key=lambda i: (-float(snr[i]), i))[:sel_max]
    dl = np.zeros(len(snr))
    for i in order:
        dl[i] = float(rec_np["width"][i]) / float(p0s[i])
    kept = fb.select(snr, per, dl, t_obs, th["group"], th["primes_max"], th["harm_tol"],
                     order=order, cap=cap, margin=th["group_margin"])
    return kept, len(pk), per


THRESHOLDS = [
    dict(snr_min=6.0, drop_frac=0.1, drop_abs=0.5, group=True, primes_max=31, harm_tol=1e-5,
         group_margin=0.16),
    dict(snr_min=6.0, drop_frac=0.1, drop_abs=0.5, group=False, primes_max=0, harm_tol=1e-5,
         group_margin=0.16),
    dict(snr_min=5.0, drop_frac=0.05, drop_abs=0.0, group=True, primes_max=97, harm_tol=1e-3,
         group_margin=0.0),
    dict(snr_min=7.0, drop_frac=0.0, drop_abs=1.0, group=True, primes_max=2, harm_tol=0.0,
         group_margin=0.3),
]


def check(F, plan, rec, ws, rec_np, n_samples, tsamp, d0, th, cap=256):
    got, n_peaks = F.ffa2best(plan, rec, ws, cap=cap, **th)
    kept, n_pk, per = oracle_select(F, plan, rec_np, n_samples, tsamp, d0, th, cap=cap)
    assert n_peaks == n_pk
    assert got["trial"].tolist() == kept
    t = got["trial"]
    assert np.array_equal(got["period_s"], per[t])
    assert np.array_equal(got["snr"], rec_np["snr"][t])
    assert np.array_equal(got["width"], rec_np["width"][t])
    assert np.array_equal(got["phase"], rec_np["phase"][t])
    first = plan.entries["first_trial"]
    ei = np.searchsorted(first, t, side="right") - 1
    assert np.array_equal(got["p0"], plan.entries["p0"][ei])
    assert np.array_equal(got["k"], t - first[ei])
    return got, n_peaks


@pytest.mark.parametrize("ti", range(len(THRESHOLDS)))
def test_plain_search_periodogram(F, dev, ti):
    import torch
    from paper_1703_05581_gb300 import synth
    x = synth.plain_series()
    plan = F.Plan(plain_cfg(F), x.size)
    ws = plan.workspace(dev)
    rec = F.search(plan, torch.from_numpy(x).to(dev), workspace=ws)
    rec_np = F.records_numpy(rec, plan.n_trials)
    got, _ = check(F, plan, rec, ws, rec_np, x.size, synth.PLAIN["tsamp"], 1, THRESHOLDS[ti])
    assert len(got) > 0 and abs(got["period_s"][0] - 0.8) < 2e-3
    # a small cap is the prefix of the full list
    few, _ = F.ffa2best(plan, rec, ws, cap=2, **THRESHOLDS[ti])
    assert few["trial"].tolist() == got["trial"][:2].tolist()


def test_several_octaves(F, dev):
    import torch
    from paper_1703_05581_gb300 import synth
    spec = synth.SeriesSpec(n=1 << 19, seed=21, red_coef=0.999, red_std=0.3,
                            pulsar_period=3.3 / 512e-6, pulsar_fwhm_frac=0.02, pulsar_snr=25.0)
    x = synth.make_series(spec)
    plan = F.Plan(F.Config(tsamp=512e-6, period_min=0.5, period_max=6.0, duty=0.2), x.size)
    ws = plan.workspace(dev)
    rec = F.search(plan, torch.from_numpy(x).to(dev), workspace=ws)
    rec_np = F.records_numpy(rec, plan.n_trials)
    for th in THRESHOLDS[:3]:
        check(F, plan, rec, ws, rec_np, x.size, 512e-6, 1, th)


def synthetic(F, dev, plan, kind, seed):
    import torch
    n = plan.n_trials
    rng = np.random.default_rng(seed)
    if kind == "walk":      # long excursions above every threshold, across many chunks
        s = 8.0 + np.cumsum(rng.standard_normal(n)) * 0.05
    elif kind == "teeth":   # a peak every other record
        s = np.where(np.arange(n) % 2 == 0, 10.0, 0.0) + rng.uniform(0, 1e-3, n)
    elif kind == "edges":   # peaks just before / after every 2048-record chunk boundary
        s = rng.uniform(0, 2, n)
        b = np.arange(2048, n, 2048)
        s[b - 1] = 12.0
        s[b] = 11.5
        s[(b + 1)[b + 1 < n]] = 30.0
    else:                   # white-noise-like levels
        s = rng.gamma(2.0, 2.0, n)
    s = s.astype(np.float32)
    rec_np = np.zeros(n, F.RECORD_DTYPE)
    rec_np["snr"] = s
    rec_np["width"] = rng.choice([1, 2, 4, 8, 16], n)
    rec_np["phase"] = rng.integers(0, 256, n)
    rec = torch.from_numpy(rec_np.view(np.int32).reshape(n, 4).copy()).to(dev)
    return rec, rec_np


@pytest.mark.parametrize("kind,seed", [("walk", 1), ("walk", 2), ("edges", 3), ("noise", 4),
                                       ("teeth", 5)])
def test_synthetic_periodograms(F, dev, kind, seed):
    from paper_1703_05581_gb300 import synth
    plan = F.Plan(plain_cfg(F), 65536)
    ws = plan.workspace(dev)
    rec, rec_np = synthetic(F, dev, plan, kind, seed)
    ts = synth.PLAIN["tsamp"]
    for th in (THRESHOLDS[0], THRESHOLDS[2], dict(THRESHOLDS[1], snr_min=9.0, drop_frac=0.0,
                                                   drop_abs=0.0)):
        _, n_peaks = check(F, plan, rec, ws, rec_np, 65536, ts, 1, th)
        if kind == "teeth" and th["snr_min"] <= 9.0:
            assert n_peaks > 4096          # the radix-select path


@pytest.mark.parametrize("exact", [False, True])
def test_more_peaks_than_the_buffer(F, dev, exact):
    """Over 65 536 peaks: the radix narrowing walks keep exactly the
    strongest 4096; with every S/N equal the narrowing runs down to the
    trial-index bits of the keys."""
    import torch
    from paper_1703_05581_gb300 import synth
    plan = F.Plan(plain_cfg(F), 1 << 18)
    assert plan.n_trials > 2 * 65536
    ws = plan.workspace(dev)
    rec, rec_np = synthetic(F, dev, plan, "teeth", 0)
    if exact:
        rec_np["snr"] = np.where(rec_np["snr"] > 5, np.float32(10.0), np.float32(0.0))
        rec = torch.from_numpy(rec_np.view(np.int32).reshape(-1, 4).copy()).to(dev)
    th = dict(snr_min=9.0, drop_frac=0.0, drop_abs=0.0, group=True, primes_max=31, harm_tol=1e-5,
              group_margin=0.16)
    _, n_peaks = check(F, plan, rec, ws, rec_np, 1 << 18, synth.PLAIN["tsamp"], 1, th)
    assert n_peaks > 65536


def test_arguments(F, dev):
    plan = F.Plan(plain_cfg(F), 1 << 16)
    ws = plan.workspace(dev)
    rec, _ = synthetic(F, dev, plan, "teeth", 0)
    # raising the baseline above the teeth leaves nothing
    got, n_peaks = F.ffa2best(plan, rec, ws, snr_min=11.0)
    assert n_peaks == 0 and len(got) == 0
    for bad in (dict(drop_frac=1.5), dict(drop_abs=-1.0), dict(harm_tol=0.5), dict(group_margin=1.0)):
        with pytest.raises(F.FFAError) as ei:
            F.ffa2best(plan, rec, ws, snr_min=6.0, **bad)
        assert ei.value.status == F.ERR_ARG
    with pytest.raises(F.FFAError) as ei:
        F.ffa2best(plan, rec, ws, snr_min=6.0, primes_max=101)
    assert ei.value.status == F.ERR_UNSUPPORTED
