"""Pins for the oracle's clipping and persistence score (Section 5): the
persistence of every trial against a brute-force count built from the
closed-form shift table of the FFA (not the recursion), the whole-profile
invariant, and a pulse train against a burst of the same energy."""
import numpy as np
import pytest

from oracle import persistence as ps


def shift(r, k, m):
    """Closed-form bins row r is read ahead in trial k of an m-stage FFA."""
    return sum(((r >> (m - 1 - l)) & 1) * (((k >> l) + 1) >> 1) for l in range(m))


def test_clip_and_quantise():
    z = np.array([-9.0, -4.0, -3.99, 0.0, 3.5, 4.0, 12.0])
    assert np.array_equal(ps.clip(z, 4.0), [-4.0, -4.0, -3.99, 0.0, 3.5, 4.0, 4.0])
    assert np.array_equal(ps.quantise(ps.clip(z, 4.0)), [-64, -64, -64, 0, 56, 64, 64])
    assert np.array_equal(ps.quantise(np.array([9.0, -9.0, 0.03125, 0.09375])), [127, -127, 0, 2])
    assert np.array_equal(ps.bits(z, 3.5), [0, 0, 0, 0, 0, 1, 1])


@pytest.mark.parametrize("m_data,m,p0", [(1, 1, 7), (2, 2, 5), (5, 8, 9), (13, 16, 11), (32, 32, 6),
                                         (20, 32, 37)])
def test_persistence_brute_force(orc, m_data, m, p0):
    rng = np.random.default_rng(m * 100 + p0)
    stages = m.bit_length() - 1
    b = (rng.random(m_data * p0 + 3) < 0.2).astype(np.int64)
    width = rng.integers(1, p0 + 1, m)
    phase = rng.integers(0, p0, m)
    got = ps.persistence(orc.fold, b, p0, m_data, m, width, phase)
    rows = b[: m_data * p0].reshape(m_data, p0)
    for k in range(m):
        win = set(((int(phase[k]) + np.arange(int(width[k]))) % p0).tolist())
        want = 0
        for r in range(m_data):
            s = shift(r, k, stages)
            for c in np.flatnonzero(rows[r]):
                if (int(c) - s) % p0 in win:
                    want += 1
        assert got[k] == want, (k, got[k], want)
    # the whole profile holds every above-cutoff sample of the data rows
    full = ps.persistence(orc.fold, b, p0, m_data, m, np.full(m, p0), np.zeros(m, int))
    assert np.all(full == rows.sum())


def test_pulsar_outscores_burst(orc):
    """Equal numbers of above-cutoff samples: spread one per period (a pulsar
    at P0 exactly, trial 0) or packed in one burst; folded at P0 the pulsar's
    window holds all of them, the burst at most the window width from each of
    the two rows it spans."""
    p0, m_data, m = 64, 32, 32
    pulsar = np.zeros(m_data * p0, np.int64)
    pulsar[np.arange(m_data) * p0 + 10] = 1
    burst = np.zeros(m_data * p0, np.int64)
    burst[500:500 + m_data] = 1
    w = np.full(m, 4)
    ph = np.full(m, 9)
    pp = ps.persistence(orc.fold, pulsar, p0, m_data, m, w, ph)
    pb = ps.persistence(orc.fold, burst, p0, m_data, m, w, np.full(m, 500 % p0))
    assert pp[0] == m_data
    assert pb.max() <= 2 * 4
