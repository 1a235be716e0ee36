"""GPU parity of each step of the search against the CPU oracle, through the
C ABI: downsampling and dereddening (bit-exact), normalisation (FP64 stats),
the FFA fold (bit-exact in FP32 and int32), and Algorithm 1 scoring."""
import math

import numpy as np
import pytest
from parity import check_records

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


def T(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


# ---------------------------------------------------------------------------
# downsampling
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,factor,n", [(np.float32, 1, 1000), (np.float32, 2, 100001),
                                            (np.float32, 64, 1 << 20), (np.uint8, 32, 77777),
                                            (np.float64, 2, 1 << 20), (np.float64, 3, 999)])
def test_downsample_bit_exact(F, orc, dev, dtype, factor, n):
    rng = np.random.default_rng(n + factor)
    if dtype == np.uint8:
        x = rng.integers(0, 256, n).astype(np.uint8)
    else:
        x = rng.standard_normal(n).astype(dtype)
    got = F.downsample(T(x, dev), factor).cpu().numpy()
    assert np.array_equal(got, orc.downsample(x, factor))


# ---------------------------------------------------------------------------
# dereddening (running median)
# ---------------------------------------------------------------------------
def _detrend_case(F, orc, dev, x, w):
    import torch
    st = F.status_word(dev)
    got = F.detrend(T(x, dev), w, status=st).cpu().numpy()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = x - orc.running_median(x, w | 1)
    assert np.array_equal(got, ref), np.flatnonzero(got != ref)[:10]


@pytest.mark.parametrize("n,w", [(1000, 1), (1000, 3), (5000, 127), (70000, 129), (70000, 1025),
                                 (300000, 3909), (2_000_000, 62501), (50_000, 62501),
                                 (900, 1025), (4099, 1025), (1025, 1025), (1, 1025)])
def test_detrend_bit_exact(F, orc, dev, n, w):
    rng = np.random.default_rng(n * 7 + w)
    x = rng.standard_normal(n) + 0.3 * np.cumsum(rng.standard_normal(n)) / math.sqrt(n + 1)
    _detrend_case(F, orc, dev, x, w)


def test_detrend_red_noise_octave_sums(F, orc, dev):
    from paper_1703_05581_gb300 import synth
    x = synth.make_series(synth.SeriesSpec(n=1 << 20, seed=5, red_coef=0.999, red_std=0.3))
    raw = orc.downsample(x, 1)
    for _ in range(3):
        raw = orc.downsample(raw, 2)  # sums of 8 float samples, exact in FP64
    _detrend_case(F, orc, dev, raw, 3909)


def test_detrend_ties_and_constant_runs(F, orc, dev):
    rng = np.random.default_rng(3)
    x = rng.integers(-3, 4, size=200_000).astype(np.float64)  # heavy ties
    _detrend_case(F, orc, dev, x, 4001)
    y = rng.standard_normal(300_000)
    y[50_000:150_000] = 0.0  # a long constant run (dropout)
    _detrend_case(F, orc, dev, y, 8001)
    _detrend_case(F, orc, dev, np.full(20_000, 2.5), 1025)


# ---------------------------------------------------------------------------
# normalisation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [10, 1000, 1 << 20, 3_000_001])
def test_normalise(F, orc, dev, n):
    rng = np.random.default_rng(n)
    r = rng.standard_normal(n) * 2.5 + 0.7
    z, stats = F.normalise(T(r, dev), F.FOLD_F32)
    q, _ = F.normalise(T(r, dev), F.FOLD_I8)
    z64, z32, q_ref, mean, std, _ = orc.normalise(r)
    st = stats.cpu().numpy()
    # FP64 sums in a different order: agreement to ~n * eps relative at worst
    assert abs(st[0] - mean) <= 1e-15 * n * max(1.0, abs(mean))
    assert abs(st[1] - std) <= 1e-15 * n * std
    z = z.cpu().numpy()
    # the FP64 reductions differ only in summation order: z agrees to the last bit
    # except where z64 lies within that rounding of a float boundary
    diff = z != z32
    assert diff.sum() <= max(2, n // 10**6)
    if diff.any():
        assert np.max(np.abs(z[diff] - z32[diff]) / np.spacing(np.abs(z32[diff]))) <= 1
    qd = q.cpu().numpy() != q_ref
    assert qd.sum() <= max(2, n // 10**6)


# ---------------------------------------------------------------------------
# the FFA fold
# ---------------------------------------------------------------------------
FOLD_CASES = [(1, 1, 1), (7, 1, 1), (3, 2, 2), (5, 3, 4), (17, 20, 32), (255, 33, 64),
              (256, 256, 256), (257, 130, 256), (390, 168, 256), (1000, 600, 1024),
              (4097, 100, 128), (31249, 9, 16), (300, 3000, 4096), (17, 5000, 8192)]


@pytest.mark.parametrize("p0,m_data,m", FOLD_CASES)
def test_fold_f32_bit_exact(F, orc, dev, p0, m_data, m):
    rng = np.random.default_rng(p0 * 31 + m)
    z = rng.standard_normal(m_data * p0 + 3).astype(np.float32)
    got = F.fold(T(z, dev), p0, m_data, m).cpu().numpy()
    rows = np.zeros((m, p0), np.float32)
    rows[:m_data] = z[: m_data * p0].reshape(m_data, p0)
    ref = orc.fold(rows)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("p0,m_data,m", FOLD_CASES[:-2])
def test_fold_int_bit_exact(F, orc, dev, p0, m_data, m):
    rng = np.random.default_rng(p0 * 17 + m)
    q = rng.integers(-127, 128, m_data * p0).astype(np.int8)
    got = F.fold(T(q, dev), p0, m_data, m).cpu().numpy()
    rows = np.zeros((m, p0), np.int64)
    rows[:m_data] = q.astype(np.int64).reshape(m_data, p0)
    assert np.array_equal(got.astype(np.int64), orc.fold(rows))


def test_fold_close_to_fp64(F, orc, dev):
    """FP32 fold vs the FP64 oracle: within 1e-5 of each row's RMS."""
    rng = np.random.default_rng(9)
    p0, m_data, m = 15625, 4294, 8192
    z = rng.standard_normal(m_data * p0)
    got = F.fold(T(z.astype(np.float32), dev), p0, m_data, m)
    for k in [0, 1, 1000, 5000, 8191]:
        ref = orc.fold_trial(z, p0, m_data, m, k)
        g = got[k].cpu().numpy().astype(np.float64)
        rms = math.sqrt(float(np.mean(ref * ref)))
        assert np.max(np.abs(g - ref)) <= 1e-5 * rms


# ---------------------------------------------------------------------------
# Algorithm 1 scoring
# ---------------------------------------------------------------------------
def _profiles(rng, count, p0, kind):
    x = rng.standard_normal((count, p0)) * 40.0
    for i in range(count):
        if i % 3 == 0:
            w = int(rng.integers(1, max(2, p0 // 8)))
            j = int(rng.integers(0, p0))
            idx = (j + np.arange(w)) % p0
            x[i, idx] += rng.uniform(5, 40) * 40.0 / math.sqrt(w)
    if kind == "int":
        return np.rint(x).astype(np.int32)
    return x.astype(np.float32)


def _check_records(got, ref, profiles, tol):
    """S/N within tol, identical flags, and width/phase identical except where
    the oracle's S/N at the GPU's choice is within 1e-3 of its best."""
    return check_records(got, ref, lambda i: profiles[i].astype(np.float64), tol=tol)


@pytest.mark.parametrize("p0,widths", [(1, (1,)), (2, (1, 2)), (9, (1, 2, 4)), (256, (1, 2, 4, 8, 16)),
                                       (511, (1, 2, 4, 8, 16, 32, 64, 128)),
                                       (1953, tuple(2 ** i for i in range(10))),
                                       (2048, tuple(2 ** i for i in range(12))),
                                       (4093, tuple(2 ** i for i in range(11))),
                                       (8192, tuple(2 ** i for i in range(12))),
                                       (10007, tuple(2 ** i for i in range(12))),
                                       (15625, tuple(2 ** i for i in range(12))),
                                       (16384, tuple(2 ** i for i in range(13))),
                                       (31249, tuple(2 ** i for i in range(13))),
                                       (32768, tuple(2 ** i for i in range(14)))])
def test_score_float(F, orc, dev, p0, widths):
    import torch
    rng = np.random.default_rng(p0)
    count = 24 if p0 > 4000 else 96
    prof = _profiles(rng, count, p0, "float")
    st = F.status_word(dev)
    rec = F.score(T(prof, dev), widths, status=st)
    got = rec.cpu().numpy().view(F.RECORD_DTYPE).reshape(-1)[:count]
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = np.array([orc.score_alg1(prof[i].astype(np.float64), widths) for i in range(count)])
    _check_records(got, ref, prof, 1e-3)


@pytest.mark.parametrize("p0,widths", [(5, (1, 2, 4)), (256, (1, 2, 4, 8, 16)),
                                       (1953, tuple(2 ** i for i in range(10))),
                                       (6000, tuple(2 ** i for i in range(11))),
                                       (12000, tuple(2 ** i for i in range(12))),
                                       (15625, tuple(2 ** i for i in range(12)))])
def test_score_int_bit_exact(F, orc, dev, p0, widths):
    rng = np.random.default_rng(p0 + 1)
    count = 24 if p0 > 4000 else 96
    prof = _profiles(rng, count, p0, "int")
    rec = F.score(T(prof, dev), widths)
    got = rec.cpu().numpy().view(F.RECORD_DTYPE).reshape(-1)[:count]
    ref = np.array([orc.score_alg1(prof[i].astype(np.int64), widths) for i in range(count)])
    assert np.array_equal(got["snr"], ref["snr"].astype(np.float32))
    assert np.array_equal(got["width"], ref["width"]) and np.array_equal(got["phase"], ref["phase"])
    assert np.array_equal(got["flags"], ref["flags"])


def test_score_degenerate_profiles(F, orc, dev):
    p0 = 300
    prof = np.zeros((4, p0), np.float32)
    prof[1] = 3.0
    prof[2, 10] = 7.0           # MAD = 0 with a spike
    prof[3] = np.arange(p0) % 2  # two values: median 0.5, MAD 0.5
    rec = F.score(T(prof, dev), (1, 2, 4))
    got = rec.cpu().numpy().view(F.RECORD_DTYPE).reshape(-1)
    ref = np.array([orc.score_alg1(prof[i].astype(np.float64), (1, 2, 4)) for i in range(4)])
    assert np.array_equal(got["flags"], ref["flags"])
    assert np.allclose(got["snr"], ref["snr"], atol=1e-6)
