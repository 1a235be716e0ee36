"""Pins for the oracle's Algorithm 2 (Section 2.2.2, Eq. 5): brute force with
explicit exclusion sets, a closed form on an alternating baseline, and the
Eq. 10 sensitivity of the fixed-width "Ref" form on top-hat pulses."""
import math

import numpy as np
import pytest


def brute_alg2(x, widths, frac=0.2):
    p0 = x.size
    h = int(math.floor(frac * p0 / 2))
    best = (-math.inf, None, None)
    for w in widths:
        b = np.array([sum(x[(j + i) % p0] for i in range(w)) for j in range(p0)])
        j = int(np.argmax(b))
        off = [k for k in range(p0) if min((k - j) % p0, (j - k) % p0) > h]
        if len(off) < 2:
            continue
        av = float(np.mean(b[off]))
        sd = float(np.std(b[off]))
        if sd <= 0:
            continue
        a = (b[j] - av) / sd
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
