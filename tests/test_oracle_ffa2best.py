"""Pins for the oracle's candidate selection (ffa2best, Section 2.3.3):
hand-worked periodograms for the peak separation, closed forms of the smeared
response, the prime-fraction harmonic table, a characterisation of the greedy
selection checked by brute force, and the plain workload end to end."""
import math
import os

import numpy as np
import pytest

from oracle import ffa2best as fb
from paper_1703_05581_gb300 import synth


# ---- R18 peak separation -------------------------------------------------------------

@pytest.mark.parametrize("snr,base,frac,ab,want", [
    ([0, 5, 10, 12, 11, 3, 0], 9, 0.1, 1, [3]),                  # one peak
    ([10, 12, 2, 9.5, 15, 1], 9, 0.1, 1, [1, 4]),                # two, separated by a fall
    ([10, 12, 11.5, 12.5, 1], 9, 0.1, 1, [3]),                   # 11.5 is not a 10 % fall
    ([10, 12, 11, 12.5, 1], 9, 0.01, 5, [3]),                    # fractional fall without the absolute one
    ([10, 12, 6, 12.5, 1], 9, 0.01, 5, [1, 3]),                  # both: a new candidate at 12.5
    ([20, 17, 15, 13], 9, 0.1, 1, [0, 1, 2, 3]),                 # a falling slope splits
    ([1, 2, 3, 8.9], 9, 0.1, 1, []),                             # never reaches the baseline
    ([10, 10, 10, 0], 9, 0.1, 1, [0]),                           # plateau: the earliest
    ([0, 9, 11], 9, 0.1, 1, [2]),                                # open at the end
    ([9, 0, 9, 0], 9, 0.0, 0.0, [0, 2]),                         # zero thresholds
    ([], 9, 0.1, 1, []),
])
def test_peaks_worked_examples(snr, base, frac, ab, want):
    assert fb.peaks(np.array(snr, np.float32), base, frac, ab) == want


def test_peaks_invariants_random():
    """On random periodograms: every peak reaches the baseline and is the
    maximum of its candidate; between consecutive peaks the S/N has fallen
    from the earlier one by both thresholds; no record reaching the baseline
    lies outside every candidate."""
    rng = np.random.default_rng(0)
    for trial in range(300):
        n = int(rng.integers(1, 80))
        s = (rng.gamma(2.0, 2.5, n)).astype(np.float32)
        base, frac, ab = 6.0, float(rng.choice([0.0, 0.05, 0.2])), float(rng.choice([0.0, 0.5, 2.0]))
        pk = fb.peaks(s, base, frac, ab)
        keep = 1.0 - frac
        assert all(float(s[i]) >= base for i in pk)
        starts = []
        for a, b in zip(pk, pk[1:] + [None]):
            # end of a's candidate: the first record after a that falls by both
            e = next((e for e in range(a + 1, n)
                      if float(s[e]) < float(s[a]) * keep and float(s[e]) < float(s[a]) - ab), n)
            assert all(float(s[t]) <= float(s[a]) for t in range(a + 1, e))
            if b is not None:
                assert e <= b
            starts.append(e)
        # records at/above baseline: inside [first start, ...) coverage
        first = next((i for i in range(n) if float(s[i]) >= base), None)
        if first is None:
            assert pk == []
        else:
            assert pk and pk[0] >= first
            assert float(s[pk[0]]) == max(float(v) for v in s[first:starts[0]])


# ---- R19 smeared response ------------------------------------------------------------

def test_smeared_response_closed_forms():
    # no period error: the full S/N
    assert fb.smeared(20.0, 0.01, 7.3, 7.3, 4000.0) == 20.0
    # drift of three duty cycles: width x4, S/N / 2 (the 1/sqrt(width) law)
    q, t, d = 2.0, 1000.0, 0.01
    p = q + 3 * d * q * q / t
    assert fb.smeared(20.0, d, p, q, t) == pytest.approx(10.0, rel=1e-12)
    # symmetric in the sign of the error
    assert fb.smeared(20.0, d, q - (p - q), q, t) == pytest.approx(10.0, rel=1e-12)
    # smeared over a whole turn: nothing left
    assert fb.smeared(20.0, d, q + q * q / t, q, t) == 0.0


# ---- R20 harmonics -------------------------------------------------------------------

def test_prime_fraction_table():
    ps = fb.primes_upto(31)
    assert ps == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31]
    fr = {(n, x) for x in ps for n in range(1, x)}
    vals = {n / x for n, x in fr}
    assert len(fr) == 149 and len(vals) == 149           # primes give no repeated fraction
    assert len(vals | {1 / v for v in vals}) == 298


@pytest.mark.parametrize("ratio,want", [
    (0.5, True), (2.0, True), (2 / 3, True), (1.5, True), (5 / 7, True), (31 / 30, True),
    (1 / 31, True), (1.0, False), (4.0, False), (0.25, False), (3 / 4, False), (37.0, False),
])
def test_harmonic_ratios(ratio, want):
    q = 1.7371
    assert fb.harmonic(q * ratio, q, 31, 1e-5) is want


def test_harmonic_tolerance_and_limit():
    q, tol = 2.318, 1e-4
    v = q * 5 / 7
    assert fb.harmonic(v * (1 + 0.5 * tol), q, 31, tol)
    assert not fb.harmonic(v * (1 + 2 * tol), q, 31, tol)
    assert fb.harmonic(q / 3, q, 3, tol) and not fb.harmonic(q / 3, q, 2, tol)
    assert not fb.harmonic(q / 2, q, 1, tol)


# ---- R21 greedy selection -------------------------------------------------------------

def test_select_characterisation_brute_force():
    """The kept set is the unique set in which no kept candidate matches a
    stronger kept one and every dropped candidate matches a stronger kept
    one; checked against every subset on small random lists."""
    rng = np.random.default_rng(5)
    t = 500.0
    for trial in range(60):
        n = int(rng.integers(1, 8))
        base = float(rng.uniform(1, 3))
        per = base * rng.choice([1, 0.5, 2, 1 / 3, 1.5, 0.25, 1.001, 1.0003, 3.7], n)
        snr = rng.uniform(6, 30, n).astype(np.float32)
        dl = rng.choice([0.01, 0.05, 0.2], n)

        def match(i, j):
            return (float(snr[i]) * 0.84 <= fb.smeared(float(snr[j]), dl[j], per[i], per[j], t)
                    or fb.harmonic(per[i], per[j], 31, 1e-5))

        order = sorted(range(n), key=lambda i: (-float(snr[i]), i))
        rank = {i: r for r, i in enumerate(order)}
        valid = []
        for mask in range(1 << n):
            ks = [i for i in range(n) if mask >> i & 1]
            ok = all(not match(i, j) for i in ks for j in ks if rank[j] < rank[i])
            ok = ok and all(any(match(i, j) for j in ks if rank[j] < rank[i])
                            for i in range(n) if i not in ks)
            if ok:
                valid.append(sorted(ks, key=rank.get))
        assert len(valid) == 1
        assert fb.select(snr, per, dl, t, True, 31, 1e-5) == valid[0]


def test_select_group_only_and_cap():
    snr = np.array([30, 20, 10, 9], np.float32)
    per = np.array([1.0, 1.0 + 1e-7, 2.0, 0.5])
    dl = np.full(4, 0.02)
    # grouping drops the near-identical period; harmonics drop 2.0 and 0.5
    assert fb.select(snr, per, dl, 1000.0, True, 31, 1e-5) == [0]
    # the margin: 20 is within 1/0.84 of the unsmeared 30 only with margin >= 1/3
    per2 = np.array([1.0, 1.0 + 0.02 * 3 / 1000.0])            # drift of 3 duty cycles: 30 -> 15
    assert fb.select(snr[:2], per2, dl[:2], 1000.0, True, 0, 1e-5) == [0, 1]
    assert fb.select(snr[:2], per2, dl[:2], 1000.0, True, 0, 1e-5, margin=0.26) == [0]
    assert fb.select(snr, per, dl, 1000.0, True, 0, 1e-5) == [0, 2, 3]
    assert fb.select(snr, per, dl, 1000.0, False, 0, 1e-5) == [0, 1, 2, 3]
    assert fb.select(snr, per, dl, 1000.0, False, 0, 1e-5, cap=2) == [0, 1]


# ---- end to end ----------------------------------------------------------------------

def test_plain_workload_selection(orc):
    """The plain series' pulsar (0.8 s) is the strongest candidate; grouping
    removes most of its twenty periodogram peaks within 1 % of its period;
    with a 0.1 % tolerance the harmonic matching removes its 2/3 harmonic;
    without grouping and harmonics every peak is kept."""
    ts = synth.PLAIN["tsamp"]
    cfg = orc.Config(tsamp=ts, period_min=256 * ts, period_max=512 * ts, widths=(1, 2, 4, 8, 16))
    x = synth.plain_series()
    rec = orc.search(cfg, x, nthreads=os.cpu_count())
    rows, nt, _ = orc.plan(cfg, x.size)
    per = orc.trial_periods(rows, cfg)
    p0s = np.repeat(rows["p0"], rows["m_rows"])
    t_obs = x.size * ts
    pk = fb.peaks(rec["snr"].astype(np.float32), 6.0, 0.1, 0.5)
    near = [i for i in pk if abs(per[i] - 0.8) < 0.008]
    assert len(near) >= 10
    kept = fb.ffa2best(rec, per, p0s, t_obs, 6.0, 0.1, 0.5, True, 31, 1e-5)
    assert 0 < len(kept) < len(pk)
    assert kept[0] == orc.best(rec)
    assert abs(per[kept[0]] - 0.8) < 2e-3
    assert sum(abs(per[i] - 0.8) < 0.008 for i in kept) <= 2
    h = per[kept[0]] * 2 / 3
    assert any(abs(per[i] - h) < 1e-3 * h for i in kept)
    kept3 = fb.ffa2best(rec, per, p0s, t_obs, 6.0, 0.1, 0.5, True, 31, 1e-3)
    assert not any(abs(per[i] - h) < 1e-3 * h for i in kept3)
    nog = fb.ffa2best(rec, per, p0s, t_obs, 6.0, 0.1, 0.5, False, 0, 1e-5)
    assert sorted(nog) == sorted(pk)
