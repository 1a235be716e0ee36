"""Pins for the oracle's FFA recursion (Section 2.1, Eq. 1-2).

Every expected value here is computed independently of the oracle: plain
numpy sums of rolled rows, and a closed-form shift table derived from the
recursive head/tail construction (trial k of a 2^m-row block reads row r
shifted by sum over levels l of bit_(m-1-l)(r) * ceil((k >> l) / 2)).
"""
import math

import numpy as np
import pytest


def shift_table(m_rows: int) -> np.ndarray:
    """Closed-form cyclic shift of row r in trial k (tested against the oracle)."""
    m = int(math.log2(m_rows))
    s = np.zeros((m_rows, m_rows), np.int64)
    for r in range(m_rows):
        for k in range(m_rows):
            tot = 0
            for lev in range(m):
                if (r >> (m - 1 - lev)) & 1:
                    tot += ((k >> lev) + 1) // 2
            s[r, k] = tot
    return s


def direct_fold(rows: np.ndarray) -> np.ndarray:
    """Brute force: trial k = sum_r rows[r] rolled left by shift(r, k)."""
    m, p0 = rows.shape
    st = shift_table(m)
    out = np.zeros_like(rows)
    for k in range(m):
        for r in range(m):
            out[k] += np.roll(rows[r], -int(st[r, k]))
    return out


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("p0", [1, 3, 7, 13, 40, 97])
def test_fold_matches_direct_sum_int(orc, m, p0):
    rng = np.random.default_rng(m * 1000 + p0)
    rows = rng.integers(-127, 128, size=(m, p0)).astype(np.int64)
    got = orc.fold(rows)
    assert np.array_equal(got, direct_fold(rows))


@pytest.mark.parametrize("m,p0", [(8, 5), (32, 33), (64, 129), (16, 300)])
def test_fold_f64_matches_direct_sum(orc, m, p0):
    rng = np.random.default_rng(7 + m + p0)
    rows = rng.standard_normal((m, p0))
    np.testing.assert_allclose(orc.fold(rows), direct_fold(rows), rtol=0, atol=1e-12)


@pytest.mark.parametrize("m,p0", [(128, 257), (256, 390), (1024, 61)])
def test_trial_zero_and_last(orc, m, p0):
    """Trial 0 is the plain fold at P0; trial M-1 drifts one bin per row."""
    rng = np.random.default_rng(m + p0)
    rows = rng.integers(-127, 128, size=(m, p0)).astype(np.int64)
    out = orc.fold(rows)
    assert np.array_equal(out[0], rows.sum(axis=0))
    last = np.zeros(p0, np.int64)
    for r in range(m):
        last += np.roll(rows[r], -r)
    assert np.array_equal(out[m - 1], last)


def test_row_sums_invariant(orc):
    """Cyclic shifts preserve sums: every trial sums to the input total."""
    rng = np.random.default_rng(3)
    rows = rng.integers(-127, 128, size=(512, 211)).astype(np.int64)
    out = orc.fold(rows)
    assert np.all(out.sum(axis=1) == rows.sum())
    rf = rng.standard_normal((256, 333))
    of = orc.fold(rf)
    np.testing.assert_allclose(of.sum(axis=1), rf.sum(), rtol=1e-12, atol=1e-9)


def test_float_fold_close_to_double(orc):
    rng = np.random.default_rng(5)
    rows = rng.standard_normal((256, 301))
    f32 = orc.fold(rows.astype(np.float32)).astype(np.float64)
    f64 = orc.fold(rows)
    rms = np.sqrt(np.mean(f64 ** 2, axis=1, keepdims=True))
    assert np.max(np.abs(f32 - f64) / rms) < 1e-5


@pytest.mark.parametrize("m", [2, 16, 256])
def test_shift_table_properties(m):
    """The closed-form shifts drift by about r*k/(M-1): monotone, bounded error."""
    st = shift_table(m)
    assert np.all(np.diff(st, axis=1) >= 0)
    r = np.arange(m)[:, None]
    k = np.arange(m)[None, :]
    err = np.abs(st - r * k / (m - 1))
    assert err.max() <= math.log2(m) / 4 + 1


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.int64])
def test_single_trial_equals_full_fold(orc, dtype):
    rng = np.random.default_rng(11)
    p0, m_data, m = 37, 45, 64
    if dtype == np.int64:
        z = rng.integers(-127, 128, size=m_data * p0 + 5).astype(np.int64)
    else:
        z = rng.standard_normal(m_data * p0 + 5).astype(dtype)
    rows = np.zeros((m, p0), dtype)
    rows[:m_data] = z[: m_data * p0].reshape(m_data, p0)
    full = orc.fold(rows)
    for k in [0, 1, 17, 40, 63]:
        assert np.array_equal(orc.fold_trial(z, p0, m_data, m, k), full[k])


def test_trial_period_mapping(orc):
    """Eq. 2 with the padded N: a pulse train of period P0 + k/(M-1) peaks at trial k."""
    p0, m = 200, 64
    for k_true in [0, 9, 31, 50, 63]:
        period = p0 + k_true / (m - 1)
        n = m * p0
        x = np.zeros(n)
        t, pulses = 13.0, 0
        while t < n:
            x[int(round(t))] += 1.0
            t += period
            pulses += 1
        out = orc.fold(x.reshape(m, p0))
        # rounding of pulse times (0.5 bin) plus the integer-shift error (< 1.5 bins at M = 64)
        # keeps every pulse inside 4 adjacent bins at the true trial
        win4 = sum(np.roll(out, -i, axis=1) for i in range(4)).max(axis=1)
        assert win4[k_true] == pulses
        assert abs(int(np.argmax(win4)) - k_true) <= 1 or win4.max() == pulses
