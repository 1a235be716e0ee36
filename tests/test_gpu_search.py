"""End-to-end GPU parity of the whole search (Section 2.3 pipeline) against the
CPU oracle: the plain 65 536-sample workload in full, the int8 path, the
candidate extraction, edge cases, and the 2^26-sample survey workload on
sampled trials."""
import math
import os

import numpy as np
import pytest
from parity import check_records, trial_profiles

pytestmark = pytest.mark.gpu

SNR_TOL = 1e-3


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


def run(F, dev, kw, x, top_k=32, snr_min=6.0):
    import torch
    plan = F.Plan(F.Config(**kw), x.size)
    xs = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    ws = plan.workspace(dev)
    st = F.status_word(dev)
    rec = F.search(plan, xs, workspace=ws, status=st)
    F.wait(st)
    cands, best = F.candidates(plan, rec, ws, snr_min=snr_min, top_k=top_k, status=st)
    return plan, F.records_numpy(rec, plan.n_trials), cands, best


def okw(kw, fold_type):
    d = dict(kw)
    for k in ("in_type", "precision"):
        d.pop(k, None)
    return dict(d, fold_type=fold_type)


def compare_records(orc, ocfg, x, got, ref, tol=SNR_TOL):
    """S/N within tol, identical flags, width/phase identical except at the
    oracle's near-ties (top-2 gap < 1e-3); returns the near-tie count."""
    rows, _, _ = orc.plan(ocfg, x.size)
    return check_records(got, ref, trial_profiles(orc, ocfg, x, rows), tol=tol)


def same_best(got, ref, best, orc):
    """The identical best (P0, trial, width, phase): the same periodogram index
    (hence octave, P0 and trial) and the same width and phase there."""
    assert best == orc.best(ref)
    assert (int(got["width"][best]), int(got["phase"][best])) == \
        (int(ref["width"][best]), int(ref["phase"][best]))


def plain_kw():
    from paper_1703_05581_gb300 import synth
    ts = synth.PLAIN["tsamp"]
    return dict(tsamp=ts, period_min=256 * ts, period_max=512 * ts, widths=(1, 2, 4, 8, 16))


def test_plain_workload_vs_fp64_oracle(F, orc, dev):
    from paper_1703_05581_gb300 import synth
    x = synth.plain_series()
    kw = plain_kw()
    plan, got, cands, best = run(F, dev, kw, x)
    ocfg = orc.Config(**okw(kw, orc.FOLD_F64))
    ref = orc.search(ocfg, x, nthreads=os.cpu_count())
    compare_records(orc, ocfg, x, got, ref)
    same_best(got, ref, best, orc)
    e = plan.entries[np.searchsorted(plan.entries["first_trial"], best, side="right") - 1]
    assert e["p0"] == 390
    # the candidate list is the top of the GPU periodogram, best first
    order = np.lexsort((np.arange(got.size), -got["snr"].astype(np.float64)))
    top = order[: len(cands)]
    assert np.array_equal(cands["trial"], top[got["snr"][top] >= 6.0])
    assert cands["trial"][0] == best
    assert abs(cands["period_s"][0] - 0.8) < 0.8 * 2e-3


def test_plain_workload_vs_fp32_oracle(F, orc, dev):
    """Same FP32 input and add tree: records match the FP32-fold oracle closely."""
    from paper_1703_05581_gb300 import synth
    x = synth.plain_series(seed=11)
    kw = plain_kw()
    _, got, _, best = run(F, dev, kw, x)
    ocfg = orc.Config(**okw(kw, orc.FOLD_F32))
    ref = orc.search(ocfg, x, nthreads=os.cpu_count())
    compare_records(orc, ocfg, x, got, ref, tol=1e-4)
    same_best(got, ref, best, orc)


def test_int8_path_matches_int_oracle(F, orc, dev):
    """The int8 search end to end.  The device's int8 codes equal the oracle's
    except for 1-LSB flips where 16 z lies on a .5 tie that the two FP64
    reduction orders round apart (counted); the oracle's exact int fold and
    scoring of the device's own codes reproduce every GPU record bit for bit;
    the int8 result's agreement with the FP64 search is stated."""
    import torch
    from paper_1703_05581_gb300 import synth
    x = synth.plain_series(seed=3)
    kw = dict(plain_kw(), precision=F.FOLD_I8)
    plan, got, _, best = run(F, dev, kw, x)
    ocfg = orc.Config(**okw(kw, orc.FOLD_I8))
    q_orc = orc.octave_series(ocfg, x)[0]
    resid = F.detrend(F.downsample(torch.from_numpy(x).to(dev), 1), plan.window)
    q_dev = F.normalise(resid, F.FOLD_I8)[0].cpu().numpy()
    diff = q_dev.astype(np.int32) - q_orc.astype(np.int32)
    flips = np.flatnonzero(diff)
    assert np.all(np.abs(diff) <= 1)
    z64 = orc.octave_series(orc.Config(**okw(plain_kw(), orc.FOLD_F64)), x)[0]
    frac = np.abs(16.0 * z64[flips]) % 1.0
    assert np.all(np.abs(frac - 0.5) < 1e-9), frac
    print(f"int8 quantiser: {flips.size} 1-LSB flips of {q_dev.size} codes")
    rows, _, _ = orc.plan(ocfg, x.size)
    ref = orc.fold_score_rows(orc.FOLD_I8, [q_dev], rows, nthreads=os.cpu_count())
    assert np.array_equal(got["snr"], ref["snr"].astype(np.float32))
    assert np.array_equal(got["width"], ref["width"]) and np.array_equal(got["phase"], ref["phase"])
    assert np.array_equal(got["flags"], ref["flags"])
    same_best(got, ref, best, orc)
    # int8 vs FP64: correlation of the periodograms (error stated in the design notes)
    ref_f64 = orc.search(orc.Config(**okw(kw, orc.FOLD_F64)), x, nthreads=os.cpu_count())
    assert np.corrcoef(got["snr"], ref_f64["snr"])[0, 1] > 0.98


def test_int8_bit_exact_on_identical_codes(F, orc, dev):
    """Fold + score of the same int8 codes: every record identical."""
    import torch
    from paper_1703_05581_gb300 import synth
    x = synth.plain_series(seed=4)
    kw = plain_kw()
    ocfg = orc.Config(**okw(kw, orc.FOLD_I8))
    q = orc.octave_series(ocfg, x)[0]
    rows, nt, _ = orc.plan(ocfg, x.size)
    qd = torch.from_numpy(q).to(dev)
    for r in rows[::37]:
        p0, md, m = int(r["p0"]), int(r["m_data"]), int(r["m_rows"])
        plane = F.fold(qd, p0, md, m)
        ws = r["widths"][: r["n_widths"]]
        got = F.score(plane, ws).cpu().numpy().view(F.RECORD_DTYPE).reshape(-1)
        qr = np.zeros((m, p0), np.int64)
        qr[:md] = q[: md * p0].astype(np.int64).reshape(md, p0)
        ref_plane = orc.fold(qr)
        assert np.array_equal(plane.cpu().numpy().astype(np.int64), ref_plane)
        ref = np.array([orc.score_alg1(ref_plane[k], ws) for k in range(m)])
        assert np.array_equal(got["snr"], ref["snr"].astype(np.float32))
        assert np.array_equal(got["phase"], ref["phase"]) and np.array_equal(got["width"], ref["width"])


def test_u8_input_and_predownsampling(F, orc, dev):
    rng = np.random.default_rng(8)
    x = rng.integers(90, 160, size=1 << 18).astype(np.uint8)
    kw = dict(tsamp=1e-3, period_min=0.3, period_max=1.1, duty=0.2, downsample0=4,
              in_type=F.IN_U8)
    _, got, _, best = run(F, dev, kw, x)
    ocfg = orc.Config(**okw(kw, orc.FOLD_F64))
    ref = orc.search(ocfg, x, nthreads=os.cpu_count())
    compare_records(orc, ocfg, x, got, ref)
    same_best(got, ref, best, orc)


def test_several_octaves_small(F, orc, dev):
    from paper_1703_05581_gb300 import synth
    spec = synth.SeriesSpec(n=1 << 19, seed=21, red_coef=0.999, red_std=0.3,
                            pulsar_period=3.3 / 512e-6, pulsar_fwhm_frac=0.02, pulsar_snr=25.0)
    x = synth.make_series(spec)
    kw = dict(tsamp=512e-6, period_min=0.5, period_max=6.0, duty=0.2)
    plan, got, cands, best = run(F, dev, kw, x)
    assert plan.n_octaves == 4
    ocfg = orc.Config(**okw(kw, orc.FOLD_F64))
    ref = orc.search(ocfg, x, nthreads=os.cpu_count())
    compare_records(orc, ocfg, x, got, ref)
    same_best(got, ref, best, orc)


def test_edge_cases(F, orc, dev):
    import torch
    # empty plan: nothing to do, no records
    plan, got, cands, best = run(F, dev, dict(tsamp=1e-3, period_min=1.0, period_max=2.0),
                                 np.zeros(100, np.float32))
    assert plan.n_trials == 0 and best == -1 and len(cands) == 0
    # a series just long enough for two rows at one base period
    x = np.random.default_rng(2).standard_normal(41).astype(np.float32)
    kw = dict(tsamp=1.0, period_min=20.0, period_max=21.0, widths=(1, 2))
    plan, got, _, best = run(F, dev, kw, x)
    ocfg = orc.Config(**okw(kw, orc.FOLD_F64))
    ref = orc.search(ocfg, x)
    assert plan.n_trials == 2
    compare_records(orc, ocfg, x, got, ref)
    # workspace too small is rejected on the host
    plan = F.Plan(F.Config(**plain_kw()), 65536)
    xs = torch.zeros(65536, dtype=torch.float32, device=dev)
    with pytest.raises(F.FFAError) as ei:
        F.search(plan, xs, workspace=torch.empty(1024, dtype=torch.uint8, device=dev))
    assert ei.value.status == F.ERR_OOM


def test_entry_ranges_and_batch(F, orc, dev):
    """Two ranges of base periods give the full search's records and candidates;
    a batch of uneven series gives each series' own search."""
    import torch
    from paper_1703_05581_gb300 import shard, synth
    x = synth.plain_series(seed=9)
    kw = plain_kw()
    plan = F.Plan(F.Config(**kw), x.size)
    xs = torch.from_numpy(x).to(dev)
    ws = plan.workspace(dev)
    full = F.search(plan, xs, workspace=ws)
    cf, bf = F.candidates(plan, full, ws, snr_min=6.0, top_k=20)
    full_np = F.records_numpy(full, plan.n_trials)
    parts = shard.split_entries(plan.entries, 3)
    rec = plan.records(dev)
    lists, bests = [], []
    for b, e in parts:
        F.search_entries(plan, xs, b, e, workspace=ws, records=rec)
        c, bb = F.candidates_entries(plan, b, e, rec, ws, snr_min=6.0, top_k=20)
        lists.append(c)
        bests.append(bb)
    got = F.records_numpy(rec, plan.n_trials)
    assert np.array_equal(got.view(np.uint8), full_np.view(np.uint8))
    merged = shard.merge_candidates(lists, 20)
    assert np.array_equal(merged["trial"], cf["trial"])
    assert bf in bests
    # batch of uneven series
    series = [synth.make_series(synth.SeriesSpec(n=n, seed=40 + i)) for i, n in
              enumerate([30000, 65536, 47000])]
    plans = [F.Plan(F.Config(**kw), s.size) for s in series]
    ts = [torch.from_numpy(s).to(dev) for s in series]
    outs = F.search_batch(plans, ts)
    for p, t, o in zip(plans, ts, outs):
        one = F.search(p, t)
        assert torch.equal(one[: p.n_trials], o[: p.n_trials])


@pytest.mark.slow
def test_survey_workload_sampled(F, orc, dev):
    """2^26 samples at 64 us, 1-30 s, the benchmark's configuration: the whole
    search on the GPU, checked on sampled trials the oracle computes one by
    one (its own dereddened series, FP64 fold of that trial, Algorithm 1)."""
    import torch
    from paper_1703_05581_gb300 import synth
    x = synth.survey_series()
    kw = dict(tsamp=64e-6, period_min=1.0, period_max=30.0, duty=0.1)
    plan, got, cands, best = run(F, dev, kw, x, top_k=16, snr_min=8.0)
    ocfg = orc.Config(**okw(kw, orc.FOLD_F64))
    rows, nt, _ = orc.plan(ocfg, x.size)
    assert nt == got.size
    z = orc.octave_series(ocfg, x)
    rng = np.random.default_rng(0)
    picks = []
    for o in range(len(z)):
        sel = np.flatnonzero(rows["octave"] == o)
        picks += [int(i) for i in rng.choice(sel, 2, replace=False)]
    # the best record's base period as well
    bi = int(np.searchsorted(rows["first_trial"], best, side="right") - 1)
    picks.append(bi)
    for i in picks:
        r = rows[i]
        o, p0, md, m = int(r["octave"]), int(r["p0"]), int(r["m_data"]), int(r["m_rows"])
        ks = [0, m - 1, int(rng.integers(0, m))]
        if i == bi:
            ks.append(int(best - r["first_trial"]))
        for k in ks:
            prof = orc.fold_trial(z[o], p0, md, m, k)
            ref = orc.score_alg1(prof, r["widths"][: r["n_widths"]])
            g = got[int(r["first_trial"]) + k]
            check_records(np.array([g]), np.array([ref]), lambda _: prof)
    # the candidate list starts with the periodogram's best record (with this
    # recipe's red noise Algorithm 1's best is a red-noise detection, not the
    # injected 7.3 s pulsar: the behaviour Section 4.1.2 reports)
    assert cands["trial"][0] == best
    assert float(cands["snr"][0]) == float(got["snr"].max())
