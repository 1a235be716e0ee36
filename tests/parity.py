"""Record comparison shared by the GPU parity tests.

The rule: every S/N within `tol` of the oracle's, identical flags, and a
(width, phase) that differs from the oracle's only at a near-tie, i.e. where
the oracle's own S/N at the GPU's choice is within `tie` (1e-3) of its best
(the tie rule of the best-candidate reading, R13).  The S/N at a given
(width, phase) is restated here from the paper's formulas (Algorithm 1:
Eq. 3-4 normalisation and a boxcar divided by sqrt(width); Algorithm 2:
Eq. 5 with the off-pulse window around the box's centre) so that the check
does not re-use the oracle's argmax.
"""
import math

import numpy as np

K_MAD = 1.4826
TIE = 1e-3


def box(prof, w, j):
    x = np.asarray(prof, np.float64)
    return float(x[(j + np.arange(w)) % x.size].sum())


def alg1_at(prof, w, j, med, mad):
    return (box(prof, w, j) - w * med) / (K_MAD * mad * math.sqrt(w))


def alg2_at(prof, w, j, frac=0.2):
    x = np.asarray(prof, np.float64)
    p0 = x.size
    h = int(math.floor(frac * p0 / 2))
    c = (j + w // 2) % p0
    k = np.arange(p0)
    d = np.minimum((k - c) % p0, (c - k) % p0)
    off = x[d > h]
    return (box(x, w, j) - w * off.mean()) / (off.std() * math.sqrt(w))


def check_records(got, ref, profile_of, tol=1e-3, tie=TIE, scorer=1, frac=0.2):
    """Compare GPU records with oracle records (SCORE_DTYPE, with median/mad).
    profile_of(i) returns trial i's folded profile (FP64).  Returns the number
    of near-ties (differing width or phase)."""
    assert got.size == ref.size
    assert np.array_equal(got["flags"], ref["flags"])
    d = np.abs(got["snr"].astype(np.float64) - ref["snr"])
    assert d.max(initial=0.0) <= tol, (float(d.max()), int(d.argmax()))
    mism = np.flatnonzero((got["width"] != ref["width"]) | (got["phase"] != ref["phase"]))
    for i in mism:
        w, j = int(got["width"][i]), int(got["phase"][i])
        prof = profile_of(int(i))
        if scorer == 1:
            alt = alg1_at(prof, w, j, float(ref["median"][i]), float(ref["mad"][i]))
        else:
            alt = alg2_at(prof, w, j, frac)
        assert float(ref["snr"][i]) - alt <= tie, (int(i), w, j, float(ref["snr"][i]), alt)
    return int(mism.size)


def trial_profiles(orc, ocfg, x, rows):
    """profile_of(i) for a whole search: trial i of the plan rows, folded by
    the oracle from its own (FP64) octave series."""
    z = [a.astype(np.int64) if a.dtype == np.int8 else a for a in orc.octave_series(ocfg, x)]
    first = rows["first_trial"].astype(np.int64)

    def profile_of(i):
        e = rows[int(np.searchsorted(first, i, side="right") - 1)]
        o, p0, md, m = int(e["octave"]), int(e["p0"]), int(e["m_data"]), int(e["m_rows"])
        return orc.fold_trial(z[o], p0, md, m, i - int(e["first_trial"])).astype(np.float64)
    return profile_of
