"""The serving loop (continuous batching over ffa_search): every request's
periodogram and candidates are the same alone and in a concurrent mix of
uneven lengths, period ranges and precisions admitted against a small HBM
budget; oversized requests are refused at submission."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05581_gb300 import ffa
    return ffa


def mix(F, count=10, seed=5):
    from paper_1703_05581_gb300 import synth
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(2 ** rng.uniform(16, 19.5))
        ts = 2.048e-3
        pmin = float(rng.uniform(0.5, 1.0))
        pmax = min(pmin * 2 ** int(rng.integers(1, 3)), n * ts / 8)
        spec = synth.SeriesSpec(n=n, seed=100 + i, pulsar_period=(pmin * 1.3) / ts,
                                pulsar_snr=15.0 if i % 3 == 0 else 0.0)
        x = synth.make_series(spec)
        cfg = F.Config(tsamp=ts, period_min=pmin, period_max=pmax,
                       precision=F.FOLD_I8 if i % 2 else F.FOLD_F32)
        reqs.append((cfg, x))
    return reqs


def alone(F, cfg, x):
    import torch
    dev = torch.device("cuda", 0)
    plan = F.Plan(cfg, x.size)
    ws = plan.workspace(dev)
    rec = F.search(plan, torch.from_numpy(x).to(dev), workspace=ws)
    c, b = F.candidates(plan, rec, ws, snr_min=6.0, top_k=8)
    return F.records_numpy(rec, plan.n_trials), c, b


def test_same_alone_and_in_the_mix(F):
    reqs = mix(F)
    need = [F.request_bytes(c, x.size) for c, x in reqs]
    # a budget of about three requests: the rest queue and are admitted as memory frees up
    budget = int(sorted(need)[-1] + sorted(need)[-2] + sorted(need)[-3]) + (1 << 20)
    srv = F.Server(budget, n_slots=4)
    try:
        tickets = [srv.submit(c, x, snr_min=6.0, top_k=8, records=True) for c, x in reqs]
        out = [srv.wait(t, timeout_ms=600000) for t in tickets]
    finally:
        srv.close()
    queued_any = False
    for (cfg, x), (cands, best, rec, times) in zip(reqs, out):
        r1, c1, b1 = alone(F, cfg, x)
        assert np.array_equal(rec.view(np.uint8), r1.view(np.uint8))
        assert np.array_equal(cands, c1) and best == b1
        assert times[0] >= 0 and times[1] > 0 and abs(times[2] - times[0] - times[1]) < 1e-6
        queued_any |= times[0] > 1.0
    assert queued_any  # the budget made some requests wait


def test_refuses_oversized_request(F):
    (cfg, x), = mix(F, count=1)
    srv = F.Server(1 << 20, n_slots=1)
    try:
        with pytest.raises(F.FFAError) as ei:
            srv.submit(cfg, x)
        assert ei.value.status == F.ERR_OOM
        assert srv.stats() == (0, 0, 0)
    finally:
        srv.close()
