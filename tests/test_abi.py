"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-side planner agrees with the oracle's plan."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ffa():
    from paper_1703_05581_gb300 import build_lib
    build_lib.build()
    from paper_1703_05581_gb300 import ffa as mod
    return mod


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(ffa\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_exports_every_declared_symbol(ffa):
    import ctypes
    lib = ctypes.CDLL(ffa.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(ffa.EXPORTS) | {"ffa_plan_destroy"}


def test_sigma_gauss_host(ffa):
    """The histogram-to-sigma mapping (host only) against scipy's normal
    quantile: sigma at each edge = Q^-1(fraction of trials at or above it)."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.integers(0, 10**6, size=int(rng.integers(3, 60))).astype(np.uint64)
        c[-1] = max(int(c[-1]), 1)
        got = ffa.sigma_gauss(c)
        tail = np.cumsum(c[::-1].astype(np.float64))[::-1][1:] / float(c.sum())
        assert np.allclose(got, -sp.ndtri(tail), rtol=0, atol=1e-9)
    # an empty top bin maps to +inf; one trial in 10^12 is 7.03 sigma
    c = np.array([0, 10**12 - 1, 1, 0], np.uint64)
    got = ffa.sigma_gauss(c)
    assert got[-1] == np.inf and abs(got[1] - 7.034483825) < 1e-6
    with pytest.raises(ffa.FFAError):
        ffa.sigma_gauss(np.zeros(4, np.uint64))


def test_status_strings(ffa):
    for s in range(8):
        assert ffa._lib.ffa_status_string(s)


CONFIGS = [
    (65536, dict(tsamp=2.048e-3, period_min=256 * 2.048e-3, period_max=512 * 2.048e-3,
                 widths=(1, 2, 4, 8, 16))),
    (1 << 26, dict(tsamp=64e-6, period_min=1.0, period_max=30.0, duty=0.1)),
    (1 << 26, dict(tsamp=64e-6, period_min=1.0, period_max=30.0, duty=0.1, downsample0=64)),
    ((1 << 22) + 12345, dict(tsamp=512e-6, period_min=0.5, period_max=20.0, duty=0.2)),
    (5000, dict(tsamp=1e-3, period_min=0.1, period_max=0.35, duty=0.2, min_rows=4)),
    (100, dict(tsamp=1e-3, period_min=0.2, period_max=0.4)),
]


@pytest.mark.parametrize("n,kw", CONFIGS)
def test_planner_matches_oracle(ffa, orc, n, kw):
    plan = ffa.Plan(ffa.Config(**kw), n)
    rows, nt, w = orc.plan(orc.Config(**kw), n)
    assert plan.n_trials == nt and plan.window == w and plan.n_periods == len(rows)
    for k in ("octave", "p0", "m_data", "m_rows", "n_widths", "n_octave", "first_trial"):
        assert np.array_equal(plan.entries[k], rows[k]), k
    assert np.array_equal(plan.entries["widths"], rows["widths"])
    if nt:
        assert np.allclose(plan.periods(), orc.trial_periods(rows, orc.Config(**kw)))


def test_plan_argument_errors(ffa):
    bad = [dict(tsamp=0.0, period_min=1.0, period_max=2.0),
           dict(tsamp=1e-3, period_min=2.0, period_max=1.0),
           dict(tsamp=1e-3, period_min=1.0, period_max=2.0, downsample0=0),
           dict(tsamp=1e-3, period_min=1.0, period_max=2.0, duty=0.0)]
    for kw in bad:
        with pytest.raises(ffa.FFAError) as ei:
            ffa.Plan(ffa.Config(**kw), 1000)
        assert ei.value.status == ffa.ERR_ARG
    with pytest.raises(ffa.FFAError) as ei:
        ffa.Plan(ffa.Config(tsamp=1e-3, period_min=1.0, period_max=2.0, widths=(1, 3)), 1000)
    assert ei.value.status == ffa.ERR_UNSUPPORTED
    # base periods beyond the scorer's 32768-bin envelope ask for pre-downsampling
    with pytest.raises(ffa.FFAError) as ei:
        ffa.Plan(ffa.Config(tsamp=1e-5, period_min=1.0, period_max=2.0), 1 << 22)
    assert ei.value.status == ffa.ERR_UNSUPPORTED


def test_empty_plan(ffa):
    plan = ffa.Plan(ffa.Config(tsamp=1e-3, period_min=1.0, period_max=2.0), 10)
    assert plan.n_trials == 0 and plan.n_periods == 0


def test_workspace_covers_buffers(ffa):
    plan = ffa.Plan(ffa.Config(**CONFIGS[1][1]), CONFIGS[1][0])
    n0 = 1 << 26
    biggest = int((plan.entries["m_rows"].astype(np.int64) * plan.entries["p0"]).max())
    assert plan.workspace_bytes >= 8 * n0 * 2 + 4 * n0 + 8 * biggest


def test_server_request_bytes(ffa):
    """Arena bytes of a serving request (host only): series, periodogram and
    workspace, each rounded up to 256 bytes."""
    al = lambda x: (x + 255) // 256 * 256
    for n, kw in CONFIGS[:4]:
        for prec in (0, 1):
            cfg = ffa.Config(**kw, precision=prec)
            plan = ffa.Plan(cfg, n)
            want = al(4 * n) + al(16 * max(plan.n_trials, 1)) + al(plan.workspace_bytes)
            assert ffa.request_bytes(cfg, n) == want
    u8 = ffa.Config(**CONFIGS[0][1], in_type=ffa.IN_U8)
    plan = ffa.Plan(u8, 65536)
    assert ffa.request_bytes(u8, 65536) == al(65536) + al(16 * plan.n_trials) + al(plan.workspace_bytes)


def test_plan_periods_eq2():
    """ffa_plan_periods: Eq. 2 with N = M * P0, written out here from the plan
    entries; a range in the middle of the periodogram, and bounds errors."""
    from paper_1703_05581_gb300 import ffa
    cfg = ffa.Config(tsamp=64e-6, period_min=1.0, period_max=5.0, downsample0=32)
    plan = ffa.Plan(cfg, 1 << 22)
    want = []
    for e in plan.entries:
        m, p0 = int(e["m_rows"]), int(e["p0"])
        scale = 64e-6 * 32 * 2.0 ** int(e["octave"])
        want += [(p0 + k * p0 / (m * p0 - p0)) * scale for k in range(m)]
    want = np.array(want)
    got = plan.periods()
    assert got.size == plan.n_trials
    np.testing.assert_allclose(got, want, rtol=1e-15)
    mid = plan.periods(1000, 777)
    assert np.array_equal(mid, got[1000:1777])
    with pytest.raises(ffa.FFAError):
        plan.periods(plan.n_trials - 1, 2)
