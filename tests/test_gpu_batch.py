"""Batched searches (ffa_search_batch): base periods of many series folded and
scored together must give every series exactly the records of its own
search (the same kernels, add tree and scorer shape), for FP32 and int8
folds and for Algorithm 2; mixed configurations and short workspaces are
rejected on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(tsamp=512e-6, period_min=0.5, period_max=20.0, duty=0.2)


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05581_gb300 import ffa
    return ffa


def _series(count, lo, hi, seed):
    from paper_1703_05581_gb300 import synth
    return [synth.make_series(s) for s in synth.batch_specs(count, lo, hi, seed, pulsar_frac=0.3)]


@pytest.mark.parametrize("prec,scorer", [("f32", 0), ("i8", 0), ("f32", 1)])
def test_batch_equals_each_series_alone(F, prec, scorer):
    import torch
    dev = torch.device("cuda", 0)
    xs = _series(9, 1 << 17, 1 << 19, 11 + scorer)
    p = F.FOLD_F32 if prec == "f32" else F.FOLD_I8
    cfg = F.Config(**KW, precision=p, scorer=scorer)
    plans = [F.Plan(cfg, x.size) for x in xs]
    ts = [torch.from_numpy(x).to(dev) for x in xs]
    st = F.status_word(dev)
    outs = F.search_batch(plans, ts, status=st)
    F.wait(st)
    assert sum(pl.n_octaves for pl in plans) > 2 * len(plans)
    for pl, t, o in zip(plans, ts, outs):
        one = F.search(pl, t)
        assert torch.equal(one[: pl.n_trials], o[: pl.n_trials]), pl.n
    # fewer launches than one search per series
    l0 = F.launch_count()
    F.search_batch(plans, ts, status=st)
    l_batch = F.launch_count() - l0
    l0 = F.launch_count()
    for pl, t in zip(plans, ts):
        F.search(pl, t)
    l_solo = F.launch_count() - l0
    torch.cuda.synchronize()
    assert l_batch < l_solo


def test_batch_rejects_mixed_and_short(F):
    import torch
    dev = torch.device("cuda", 0)
    xs = _series(2, 1 << 16, 1 << 17, 5)
    plans = [F.Plan(F.Config(**KW), xs[0].size), F.Plan(F.Config(**dict(KW, duty=0.1)), xs[1].size)]
    ts = [torch.from_numpy(x).to(dev) for x in xs]
    with pytest.raises(F.FFAError) as ei:
        F.search_batch(plans, ts)
    assert ei.value.status == F.ERR_ARG
    plans = [F.Plan(F.Config(**KW), x.size) for x in xs]
    with pytest.raises(F.FFAError) as ei:
        F.search_batch(plans, ts, workspace=torch.empty(1 << 20, dtype=torch.uint8, device=dev))
    assert ei.value.status == F.ERR_OOM
