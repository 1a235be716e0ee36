"""The fold autotuner (stages per HBM pass and column-tile width): tuning changes no
result, only the time; searches before and after tuning give identical periodograms."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_results(F, precision):
    import torch
    from paper_1703_05581_gb300 import synth
    dev = torch.device("cuda", 0)
    spec = synth.SeriesSpec(n=1 << 20, seed=31, red_coef=0.999, red_std=0.3,
                            pulsar_period=2.2 / 512e-6, pulsar_snr=20.0)
    x = synth.make_series(spec)
    plan = F.Plan(F.Config(tsamp=512e-6, period_min=0.5, period_max=8.0, precision=precision), x.size)
    ws = plan.workspace(dev)
    xs = torch.from_numpy(x).to(dev)
    r0 = F.records_numpy(F.search(plan, xs, workspace=ws), plan.n_trials).copy()
    # one plane folded before tuning
    e = plan.entries[len(plan.entries) // 2]
    z = torch.randn(int(e["m_data"]) * int(e["p0"]) + 7, device=dev)
    if precision:
        z = (z * 16).round().clamp(-127, 127).to(torch.int8)
    p_before = F.fold(z, int(e["p0"]), int(e["m_data"]), int(e["m_rows"])).cpu().numpy()
    n = F.autotune(plan, ws)
    assert n >= 1
    r1 = F.records_numpy(F.search(plan, xs, workspace=ws), plan.n_trials)
    assert np.array_equal(r0.view(np.uint8), r1.view(np.uint8))
    p_after = F.fold(z, int(e["p0"]), int(e["m_data"]), int(e["m_rows"])).cpu().numpy()
    assert np.array_equal(p_before.view(np.uint8), p_after.view(np.uint8))
