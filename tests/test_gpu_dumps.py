"""The search's debug outputs (Section 2.3: ffancy can write the dereddened
series and the full suite of folded profiles of an FFA execution) against the
oracle: each octave's dereddened series bit for bit (exact downsampling and
running median), its normalised fold input to summation-order rounding, and a
base period's whole plane bit for bit against the oracle's FP32 (or int64)
fold of the device's own fold input."""
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


def _oracle_resid(orc, x, d0, win, octave):
    raw = orc.downsample(x, d0)
    for _ in range(octave):
        raw = orc.downsample(raw, 2)
    return raw - orc.running_median(raw, win) if win > 1 else raw


@pytest.mark.parametrize("precision", ["f32", "i8"])
def test_series_and_plane_dumps(F, orc, precision):
    import torch
    from paper_1703_05581_gb300 import synth
    dev = torch.device("cuda", 0)
    spec = synth.SeriesSpec(n=1 << 17, seed=77, red_coef=0.999, red_std=0.3,
                            pulsar_period=1.3 / 512e-6, pulsar_fwhm_frac=0.03, pulsar_snr=20.0)
    x = synth.make_series(spec)
    prec = F.FOLD_F32 if precision == "f32" else F.FOLD_I8
    cfg = F.Config(tsamp=512e-6, period_min=0.5, period_max=3.5, duty=0.2, precision=prec)
    plan = F.Plan(cfg, x.size)
    assert plan.n_octaves >= 3
    xs = torch.from_numpy(x).to(dev)
    ws = plan.workspace(dev)
    ocfg = orc.Config(tsamp=512e-6, period_min=0.5, period_max=3.5, duty=0.2,
                      fold_type=orc.FOLD_F32 if precision == "f32" else orc.FOLD_I8)
    z_orc = orc.octave_series(ocfg, x)
    for o in range(plan.n_octaves):
        resid = F.search_series(plan, xs, o, F.DUMP_RESID, workspace=ws).cpu().numpy()
        assert np.array_equal(resid, _oracle_resid(orc, x, 1, plan.window, o))
        z = F.search_series(plan, xs, o, F.DUMP_Z, workspace=ws).cpu().numpy()
        if precision == "f32":
            np.testing.assert_allclose(z, z_orc[o], rtol=1e-6, atol=1e-6)
        else:
            assert np.max(np.abs(z.astype(np.int32) - z_orc[o].astype(np.int32))) <= 1
        # one base period per octave: its whole plane against the oracle's fold of z
        sel = np.flatnonzero(plan.entries["octave"] == o)
        i = int(sel[len(sel) // 2])
        e = plan.entries[i]
        p0, md, m = int(e["p0"]), int(e["m_data"]), int(e["m_rows"])
        plane = F.search_plane(plan, xs, i, workspace=ws).cpu().numpy()
        rows = np.zeros((m, p0), np.float32 if precision == "f32" else np.int64)
        rows[:md] = z[: md * p0].reshape(md, p0)
        assert np.array_equal(plane.astype(rows.dtype), orc.fold(rows))


def test_dump_arguments(F):
    import torch
    dev = torch.device("cuda", 0)
    cfg = F.Config(tsamp=1e-3, period_min=0.3, period_max=0.5)
    plan = F.Plan(cfg, 1 << 14)
    xs = torch.zeros(1 << 14, dtype=torch.float32, device=dev)
    with pytest.raises(F.FFAError):
        F._check(F._lib.ffa_search_plane(plan._h, F._ptr(xs), plan.n_periods, F._ptr(plan.workspace(dev)),
                                         plan.workspace_bytes, F._ptr(xs), None, None))
    with pytest.raises(F.FFAError):
        F._check(F._lib.ffa_search_series(plan._h, F._ptr(xs), plan.n_octaves, F.DUMP_Z,
                                          F._ptr(plan.workspace(dev)), plan.workspace_bytes, F._ptr(xs),
                                          None, None))
