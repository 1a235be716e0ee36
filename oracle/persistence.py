"""Input clipping and the persistence score (Section 5), as the oracle.

TEST INFRASTRUCTURE ONLY (the oracle): plain numpy on top of the oracle's
literal FFA recursion (oracle.fold, int64); shares no code with the library.

Readings of the proposals in Section 5 (numbered after ffa2best's):
  R22 clipping caps the normalised series at +-clip (z is in units of the
      series' standard deviation, so the cap is clip sigma); the int8 code is
      taken from the capped value.
  R23 persistence: every sample of the normalised series scores 1 if it
      exceeds the cutoff and 0 otherwise; the 0/1 series is folded by the same
      FFA as the data (integer adds), and a trial's persistence is the sum of
      its folded 0/1 profile over the best boxcar window of that trial's
      score (width and phase of its record): the number of above-cutoff
      samples that make up the detected pulse.  A pulsar spreads them over
      many rows; a single burst contributes at most its own length.
"""
from __future__ import annotations

import numpy as np


def clip(z: np.ndarray, c: float) -> np.ndarray:
    """R22 for the FP path (c > 0)."""
    return np.minimum(np.maximum(z, -c), c)


def quantise(z64: np.ndarray) -> np.ndarray:
    """The int8 code of a (capped) FP64 normalised value: rint(16 z), +-127."""
    return np.clip(np.rint(16.0 * z64), -127, 127).astype(np.int8)


def bits(z: np.ndarray, cutoff: float) -> np.ndarray:
    """R23's 0/1 score of every sample."""
    return (np.asarray(z) > cutoff).astype(np.int64)


def persistence(fold, b: np.ndarray, p0: int, m_data: int, m: int, width, phase) -> np.ndarray:
    """R23 for every trial of one base period: fold the 0/1 series b as
    m_data rows of p0 (zero rows up to m), then sum each trial's profile over
    [phase, phase + width) cyclically.  `fold` is the oracle's FFA."""
    rows = np.zeros((m, p0), np.int64)
    rows[:m_data] = b[: m_data * p0].reshape(m_data, p0)
    plane = fold(rows)
    out = np.zeros(m, np.int64)
    for k in range(m):
        idx = (int(phase[k]) + np.arange(int(width[k]))) % p0
        out[k] = int(plane[k, idx].sum())
    return out
