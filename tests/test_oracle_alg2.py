"""Pins for the oracle's Algorithm 2 (Section 2.2.2, Eq. 5): a brute force
with explicit exclusion sets, closed forms on an alternating baseline (one of
which only holds with the window centred on the box's centre), the Eq. 10
sensitivity of the fixed-width "Ref" form on top-hat pulses, and the
white-noise statement of Section 4.3 that the two algorithms' S/N
distributions are largely similar."""
import math

import numpy as np
import pytest


def brute_alg2(x, widths, frac=0.2):
    """Every box written out; the window is the set of profile bins within
    cyclic distance h of the winning box's centre j* + w//2; I_av and sigma
    are numpy's mean and population std of the remaining raw bins."""
    p0 = x.size
    h = int(math.floor(frac * p0 / 2))
    best = (-math.inf, None, None)
    for w in widths:
        b = np.array([sum(x[(j + i) % p0] for i in range(w)) for j in range(p0)])
        j = int(np.argmax(b))  # first position of the maximum
        c = (j + w // 2) % p0
        off = [k for k in range(p0) if min((k - c) % p0, (c - k) % p0) > h]
        if len(off) < 2:
            continue
        av = float(np.mean(x[off]))
        sd = float(np.std(x[off]))
        if sd <= 0:
            continue
        a = (b[j] - w * av) / (sd * math.sqrt(w))
        if a > best[0]:
            best = (a, w, j)
    return best


@pytest.mark.parametrize("p0", [10, 37, 64, 150])
def test_alg2_matches_brute_force(orc, p0):
    rng = np.random.default_rng(p0 + 5)
    for trial in range(4):
        x = rng.standard_normal(p0) * 2 + 1.5
        if trial % 2:
            x[rng.integers(p0)] += 9.0
        widths = [1, 2, 4, 8][: max(1, int(math.log2(p0)) - 1)]
        rec = orc.score_alg2(x, widths)
        a, w, j = brute_alg2(x, widths)
        assert rec["snr"] == pytest.approx(a, rel=1e-10)
        assert (rec["width"], rec["phase"]) == (w, j)


def test_alg2_closed_form_alternating_baseline(orc):
    """Width 1, baseline +1/-1 alternating, one pulse of height S at bin 50 of
    100: the 21 bins 40..60 are excluded, leaving 20 (+1) and 20 (-1) below and
    19 (+1) and 20 (-1) above: mean -1/79, std sqrt(1 - 1/79^2)."""
    p0, s = 100, 7.0
    x = np.where(np.arange(p0) % 2 == 0, 1.0, -1.0)
    x[50] = s
    rec = orc.score_alg2(x, [1])
    mean = -1.0 / 79
    sd = math.sqrt(1.0 - mean * mean)
    assert rec["phase"] == 50
    assert rec["median"] == pytest.approx(mean, abs=1e-14)
    assert rec["mad"] == pytest.approx(sd, rel=1e-14)
    assert rec["snr"] == pytest.approx((s - mean) / sd, rel=1e-13)


def test_alg2_closed_form_window_centre(orc):
    """Alternating +1/-1 baseline with a top-hat of height S on bins 48..51.
    Width 4: the boxes away from the pulse sum to 0, the best is 4S at bin 48,
    centre 50, window 40..60 -> 39 (+1) and 40 (-1) remain, mean -1/79;
    A_4 = (4S + 4/79) / (2 sd).  Width 2: best 2S at bin 48, centre 49, window
    39..59 -> 40 (+1) and 39 (-1) remain, mean +1/79; A_2 = (2S - 2/79) /
    (sqrt(2) sd).  A window centred on j* itself would give width 2 the mean
    -1/79 instead."""
    p0, s = 100, 7.0
    x = np.where(np.arange(p0) % 2 == 0, 1.0, -1.0)
    x[48:52] = s
    sd = math.sqrt(1.0 - 1.0 / 79 ** 2)
    r2 = orc.score_alg2(x, [2])
    assert (r2["width"], r2["phase"]) == (2, 48)
    assert r2["median"] == pytest.approx(1.0 / 79, abs=1e-14)
    assert r2["snr"] == pytest.approx((2 * s - 2.0 / 79) / (math.sqrt(2) * sd), rel=1e-13)
    r4 = orc.score_alg2(x, [1, 2, 4])
    assert (r4["width"], r4["phase"]) == (4, 48)
    assert r4["median"] == pytest.approx(-1.0 / 79, abs=1e-14)
    assert r4["mad"] == pytest.approx(sd, rel=1e-14)
    assert r4["snr"] == pytest.approx((4 * s + 4.0 / 79) / (2 * sd), rel=1e-13)


@pytest.mark.parametrize("w", [4, 16, 32])
def test_alg2_ref_eq10(orc, w):
    """Fixed matched width (the paper's "Ref" form): S/N ~ S sqrt(w) (Eq. 10)."""
    p0, s = 1024, 20.0 / math.sqrt(w)
    vals = []
    for seed in range(30):
        rng = np.random.default_rng(3000 + seed)
        x = rng.standard_normal(p0)
        x[200:200 + w] += s
        vals.append(orc.score_alg2(x, [w])["snr"])
    assert 0.95 < np.mean(vals) / (s * math.sqrt(w)) < 1.1


def test_alg2_degenerate(orc):
    rec = orc.score_alg2(np.full(40, 2.0), [1, 2])
    assert rec["flags"] == 1 and rec["snr"] == 0.0


def test_white_noise_similar_to_algorithm1(orc):
    """Section 4.3: on white noise the two algorithms' S/N distributions are
    largely similar.  Folded white noise gives profiles of independent
    Gaussian bins; with the false-alarm study's profile lengths (489..977
    bins at 2.048 ms, widths to the first over 20 % of the profile), the
    upper quantiles of the two scores (2 and 2.5 sigma_gauss) agree within a
    few per cent.  Taking I_av and sigma from the filtered bins instead makes
    Algorithm 2's quantiles 25-40 % higher."""
    from scipy.stats import norm
    rng = np.random.default_rng(4303)
    n = 12000
    a1 = np.empty(n)
    a2 = np.empty(n)
    for i in range(n):
        p0 = int(rng.integers(489, 978))
        widths = []
        w = 1
        while True:
            widths.append(w)
            if w > 0.2 * p0:
                break
            w *= 2
        x = rng.standard_normal(p0)
        a1[i] = orc.score_alg1(x, widths)["snr"]
        a2[i] = orc.score_alg2(x, widths)["snr"]
    for sig in (2.0, 2.5):
        q = 1.0 - norm.sf(sig)
        q1, q2 = np.quantile(a1, q), np.quantile(a2, q)
        assert abs(q2 / q1 - 1.0) < 0.06, (sig, q1, q2)
