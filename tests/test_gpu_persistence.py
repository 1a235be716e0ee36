"""Input clipping and the persistence score (Section 5) on the GPU, against
the oracle: the clipped FP32 search within the FP32 tolerance of the oracle's
fold and Algorithm 1 of the clipped series, and the persistence of every trial
exact against the oracle's integer fold of the 0/1 series."""
import os

import numpy as np
import pytest

from oracle import persistence as ps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05581_gb300 import ffa
    return ffa


def burst_series(amp=200.0):
    """The plain series (0.8 s pulsar) with a 60-sample burst of interference."""
    from paper_1703_05581_gb300 import synth
    x = synth.plain_series(seed=12).copy()
    x[30000:30060] += np.float32(amp)
    return x


def kw_plain():
    from paper_1703_05581_gb300 import synth
    ts = synth.PLAIN["tsamp"]
    return dict(tsamp=ts, period_min=256 * ts, period_max=512 * ts, widths=(1, 2, 4, 8, 16))


def oracle_z64(orc, kw, x):
    return orc.octave_series(orc.Config(**kw, fold_type=orc.FOLD_F64), x)


def test_clipping_parity_and_effect(F, orc):
    import torch
    dev = torch.device("cuda", 0)
    x = burst_series()
    kw = kw_plain()
    xs = torch.from_numpy(x).to(dev)
    # without clipping the burst outshines the pulsar
    plan0 = F.Plan(F.Config(**kw), x.size)
    r0 = F.records_numpy(F.search(plan0, xs), plan0.n_trials)
    per = orc.trial_periods(orc.plan(orc.Config(**kw), x.size)[0], orc.Config(**kw))
    b0 = int(np.argmax(r0["snr"]))
    assert abs(per[b0] - 0.8) > 0.01 and r0["snr"][b0] > 20
    # clipped at 4 sigma: parity with the oracle's search of the clipped series
    plan = F.Plan(F.Config(**kw, clip_sigma=4.0), x.size)
    got = F.records_numpy(F.search(plan, xs), plan.n_trials)
    z = [ps.clip(z, 4.0).astype(np.float32) for z in oracle_z64(orc, kw, x)]
    rows, _, _ = orc.plan(orc.Config(**kw), x.size)
    ref = orc.fold_score_rows(orc.FOLD_F32, z, rows, nthreads=os.cpu_count())
    d = np.abs(got["snr"].astype(np.float64) - ref["snr"])
    assert d.max() <= 1e-4, d.max()
    assert int(np.argmax(got["snr"])) == orc.best(ref)
    assert abs(per[orc.best(ref)] - 0.8) < 2e-3
    # int8 codes of the clipped value
    plan8 = F.Plan(F.Config(**kw, clip_sigma=4.0, precision=F.FOLD_I8), x.size)
    g8 = F.records_numpy(F.search(plan8, xs), plan8.n_trials)
    q = [ps.quantise(ps.clip(z, 4.0)) for z in oracle_z64(orc, kw, x)]
    r8 = orc.fold_score_rows(orc.FOLD_I8, q, rows, nthreads=os.cpu_count())
    assert np.mean(g8["snr"] == r8["snr"].astype(np.float32)) > 0.99


@pytest.mark.parametrize("cutoff,clip,precision", [(2.0, 0.0, 0), (1.0, 4.0, 0), (2.5, 0.0, 1)])
def test_persistence_exact(F, orc, cutoff, clip, precision):
    import torch
    dev = torch.device("cuda", 0)
    x = burst_series()
    kw = kw_plain()
    cfg = F.Config(**kw, clip_sigma=clip, persistence=True, persist_cutoff=cutoff, precision=precision)
    plan = F.Plan(cfg, x.size)
    xs = torch.from_numpy(x).to(dev)
    rec, pers = F.search_persistence(plan, xs)
    got = F.records_numpy(rec, plan.n_trials)
    pg = pers[: plan.n_trials].cpu().numpy().view(np.uint32)
    # the records are the plain search's, bit for bit
    plain = F.records_numpy(F.search(plan, xs), plan.n_trials)
    assert np.array_equal(got.view(np.uint8), plain.view(np.uint8))
    b = ps.bits(oracle_z64(orc, kw, x)[0], cutoff)
    for e in plan.entries:
        f, m = int(e["first_trial"]), int(e["m_rows"])
        want = ps.persistence(orc.fold, b, int(e["p0"]), int(e["m_data"]), m,
                              got["width"][f:f + m], got["phase"][f:f + m])
        assert np.array_equal(pg[f:f + m].astype(np.int64), want), int(e["p0"])


def test_persistence_arguments(F):
    import torch
    dev = torch.device("cuda", 0)
    kw = kw_plain()
    plan = F.Plan(F.Config(**kw), 65536)
    with pytest.raises(F.FFAError) as ei:
        F.search_persistence(plan, torch.zeros(65536, device=dev))
    assert ei.value.status == F.ERR_ARG
    with pytest.raises(F.FFAError):
        F.Plan(F.Config(**kw, clip_sigma=-1.0), 65536)
