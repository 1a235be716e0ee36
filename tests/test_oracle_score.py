"""Pins for the oracle's Algorithm 1 scorer (Section 2.2.1, Eq. 3-4, Eq. 10).

Expected values come from brute force over every (width, phase) with direct
cyclic sums, from numpy's median, from closed forms for symmetric value sets,
and from the single-profile sensitivity of Eq. 10 with the paper's reported
power-of-two filter loss envelope (Section 3.1.2: at most about 16 %).
"""
import math

import numpy as np
import pytest

K = 1.4826


def brute(x: np.ndarray, widths):
    """Every width, every phase, direct cyclic sums; R13 tie-breaks."""
    p0 = x.size
    med = float(np.median(x))
    mad = float(np.median(np.abs(x - med)))
    best = (-math.inf, None, None)
    for w in widths:
        sums = [sum(float(x[(j + i) % p0]) for i in range(w)) for j in range(p0)]
        j = int(np.argmax(sums))  # first maximum
        snr = (sums[j] - w * med) / (K * mad * math.sqrt(w))
        if snr > best[0]:
            best = (snr, w, j)
    return best, med, mad


@pytest.mark.parametrize("p0", [5, 16, 33, 64, 101])
def test_alg1_matches_brute_force(orc, p0):
    rng = np.random.default_rng(p0)
    for trial in range(5):
        x = rng.standard_normal(p0) * 3 + rng.normal()
        if trial == 1:
            x[rng.integers(p0)] += 12.0  # a pulse
        widths = [1, 2, 4, 8, 16][: max(1, int(math.log2(p0)))]
        rec = orc.score_alg1(x, widths)
        (snr, w, j), med, mad = brute(x, widths)
        assert rec["median"] == pytest.approx(med, abs=0)
        assert rec["mad"] == pytest.approx(mad, rel=1e-15)
        assert rec["snr"] == pytest.approx(snr, rel=1e-12)
        assert (rec["width"], rec["phase"]) == (w, j)


def test_alg1_int_profile_exact(orc):
    rng = np.random.default_rng(42)
    for p0 in [7, 64, 200]:
        x = rng.integers(-2000, 2000, size=p0).astype(np.int64)
        x[p0 // 3] += 9000
        widths = [1, 2, 4, 8]
        rec = orc.score_alg1(x, widths)
        (snr, w, j), med, mad = brute(x.astype(np.float64), widths)
        assert rec["median"] == med and rec["mad"] == mad
        assert rec["snr"] == pytest.approx(snr, rel=1e-14)
        assert (rec["width"], rec["phase"]) == (w, j)
        # the integer and floating instantiations agree exactly on the same values
        rf = orc.score_alg1(x.astype(np.float64), widths)
        assert rf["snr"] == rec["snr"] and rf["phase"] == rec["phase"]


def test_median_mad_closed_form(orc):
    """Symmetric integer set {-a..a}: median 0, MAD = ceil(a/2) (odd count);
    {-a..a} without 0 (even count): median 0, MAD = the mean of two middles."""
    for a in [1, 2, 5, 10, 101]:
        x = np.random.default_rng(a).permutation(np.arange(-a, a + 1)).astype(np.float64)
        rec = orc.score_alg1(x, [1])
        assert rec["median"] == 0.0
        assert rec["mad"] == math.ceil(a / 2)
        # S/N of width 1 at the largest value a
        assert rec["snr"] == pytest.approx(a / (K * math.ceil(a / 2)))
        y = x[x != 0]
        ry = orc.score_alg1(y, [1])
        # |y| = 1,1,2,2,...,a,a: the two middles of 2a sorted values
        srt = np.sort(np.abs(y))
        assert ry["median"] == 0.0
        assert ry["mad"] == (srt[a - 1] + srt[a]) / 2


def test_mad_zero_flag(orc):
    x = np.full(50, 3.0)
    x[7] = 10.0
    rec = orc.score_alg1(x, [1, 2, 4])
    assert rec["mad"] == 0.0 and rec["snr"] == 0.0 and rec["flags"] == 1


@pytest.mark.parametrize("w", [4, 16, 32])
def test_eq10_aligned_width(orc, w):
    """Top-hat of height S and width w = 2^n in unit noise: S/N ~ S sqrt(w) (Eq. 10)."""
    p0, s = 1024, 4.0 / math.sqrt(w) * 5
    vals = []
    for seed in range(30):
        rng = np.random.default_rng(1000 + seed)
        x = rng.standard_normal(p0)
        x[300:300 + w] += s
        vals.append(orc.score_alg1(x, [2 ** i for i in range(9)])["snr"])
    ratio = np.mean(vals) / (s * math.sqrt(w))
    assert 0.95 < ratio < 1.08


@pytest.mark.parametrize("w", [6, 12, 23, 45])
def test_power_of_two_loss_envelope(orc, w):
    """Between powers of two the best filter loses at most 1 - 2^(-1/4) ~ 16 % (Section 3).

    Narrow pulses (duty <= ~1 %) so that the pulse barely moves the median / MAD."""
    p0 = 4096
    s = 20.0 / math.sqrt(w)
    vals = []
    for seed in range(30):
        rng = np.random.default_rng(2000 + seed)
        x = rng.standard_normal(p0)
        x[500:500 + w] += s
        vals.append(orc.score_alg1(x, [2 ** i for i in range(9)])["snr"])
    ratio = np.mean(vals) / (s * math.sqrt(w))
    ideal = max(min(w, 2 ** p) / math.sqrt(2 ** p) for p in range(9)) / math.sqrt(w)
    assert ideal >= 2 ** -0.25 - 1e-12
    assert ideal - 0.06 < ratio < ideal + 0.08
