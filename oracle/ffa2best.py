"""Candidate selection after the search, as ffa2best does it (Section 2.3.3).

TEST INFRASTRUCTURE ONLY (the oracle): plain Python loops over the whole
periodogram, written from the paper's description of ffa2best; the library
(its ffa2best entry point) shares no code with it.  All arithmetic is IEEE
binary64 (Python floats), S/N values are the periodogram's float32 values.

Readings of the description (Section 2.3.3), numbered after the search's:
  R18 peak separation.  Walk the periodogram in trial order, which is period
      order.  Outside a candidate, a record with S/N >= snr_min starts one;
      inside, the running maximum is the candidate's peak, and the candidate
      ends at the first record whose S/N is below both peak * (1 - drop_frac)
      and peak - drop_abs (it has fallen by both thresholds).  That record may
      itself start the next candidate.  A candidate still open at the end of
      the periodogram ends there.  Each candidate is represented by its peak
      record (the earliest one on equal S/N).
  R19 grouping by the smeared response.  Folding a pulse of duty cycle
      delta (best width / P0 of its peak) at a period off by dP over an
      observation of T seconds drifts it by T*|dP|/P^2 turns, so its
      expected S/N falls to S*sqrt(delta/(delta + T*|dP|/P^2)) (the
      1/sqrt(width) law of Eq. 7), and to nothing once the smeared width
      reaches a whole turn.  The measured responses of both algorithms
      depart from that law by up to about 16 % (Section 3.1), so a candidate
      whose S/N, times (1 - margin) with margin = 0.16 by default, is at most
      that expected response of a stronger kept candidate is that candidate,
      smeared, and is dropped.
  R20 harmonics.  For every prime x <= primes_max and integer 0 < n < x, a
      stronger kept candidate of period q predicts the periods q*(n/x) and
      q/(n/x); a weaker candidate of period p with |p - v| <= tol * v for a
      predicted v is harmonically related and dropped.
  R21 order.  Candidates are taken strongest first (ties: earlier trial); a
      candidate is compared only with the stronger candidates kept so far, so
      a dropped candidate drops nothing.
"""
from __future__ import annotations

import math

import numpy as np


def peaks(snr, snr_min: float, drop_frac: float, drop_abs: float) -> list[int]:
    """R18 over S/N values in period order; returns the peak indices."""
    keep = 1.0 - drop_frac
    out = []
    inside = False
    pk, pi = 0.0, -1
    for i in range(len(snr)):
        s = float(snr[i])
        if inside:
            if s > pk:
                pk, pi = s, i
            elif s < pk * keep and s < pk - drop_abs:
                out.append(pi)
                inside = False
        if not inside and s >= snr_min:
            inside, pk, pi = True, s, i
    if inside:
        out.append(pi)
    return out


def primes_upto(n: int) -> list[int]:
    return [p for p in range(2, n + 1) if all(p % d for d in range(2, math.isqrt(p) + 1))]


def smeared(snr_j: float, delta_j: float, p: float, q: float, t_obs: float) -> float:
    """R19: expected S/N at period p of a pulse of S/N snr_j and duty delta_j
    detected at period q, over t_obs seconds (0 once smeared over a turn)."""
    de = delta_j + t_obs * abs(p - q) / (q * q)
    if de >= 1.0:
        return 0.0
    return snr_j * math.sqrt(delta_j / de)


def harmonic(p: float, q: float, primes_max: int, tol: float) -> bool:
    """R20: is period p within tol of q * (n/x) or q / (n/x) for a prime x?"""
    for x in primes_upto(primes_max):
        for n in range(1, x):
            f = n / x
            for v in (q * f, q / f):
                if abs(p - v) <= tol * v:
                    return True
    return False


def fractions(primes_max: int) -> np.ndarray:
    """R20's fractions n/x, 0 < n < x, for every prime x <= primes_max."""
    return np.array([n / x for x in primes_upto(primes_max) for n in range(1, x)], np.float64)


def select(snr, periods, delta, t_obs: float, group: bool, primes_max: int, tol: float,
           order=None, cap: int | None = None, margin: float = 0.16) -> list[int]:
    """R19-R21 over a candidate list: indices into snr/periods/delta, kept
    ones strongest first.  `order` restricts the list (default: all).  Each
    candidate is tested against every kept one at once (numpy elementwise,
    the same binary64 operations as smeared() and harmonic())."""
    idx = list(range(len(snr))) if order is None else list(order)
    idx.sort(key=lambda i: (-float(snr[i]), i))
    shrink = 1.0 - margin
    fr = fractions(primes_max) if primes_max >= 2 else np.zeros(0)
    kq = np.zeros(len(idx))
    ks = np.zeros(len(idx))
    kd = np.zeros(len(idx))
    kept: list[int] = []
    for i in idx:
        p, s = float(periods[i]), float(snr[i])
        nk = len(kept)
        drop = False
        if nk:
            q, sj, dj = kq[:nk], ks[:nk], kd[:nk]
            if group:
                de = dj + t_obs * np.abs(p - q) / (q * q)
                resp = np.where(de >= 1.0, 0.0, sj * np.sqrt(dj / de))
                drop = bool(np.any(s * shrink <= resp))
            if not drop and fr.size:
                v = np.concatenate([q[:, None] * fr[None, :], q[:, None] / fr[None, :]], axis=1)
                drop = bool(np.any(np.abs(p - v) <= tol * v))
        if not drop:
            kq[nk], ks[nk], kd[nk] = p, s, float(delta[i])
            kept.append(i)
            if cap is not None and len(kept) == cap:
                break
    return kept


def ffa2best(records, periods, p0s, t_obs: float, snr_min: float, drop_frac: float,
             drop_abs: float, group: bool = True, primes_max: int = 31, tol: float = 1e-5,
             cap: int | None = None, margin: float = 0.16) -> list[int]:
    """The whole selection on a periodogram (records in trial order with
    fields snr and width; periods[i] in seconds; p0s[i] the bins of trial i's
    profile).  Returns kept trial indices, strongest first."""
    snr = records["snr"]
    pk = peaks(snr, snr_min, drop_frac, drop_abs)
    delta = {}
    for i in pk:
        delta[i] = float(records["width"][i]) / float(p0s[i])
    dl = np.zeros(len(snr))
    for i, d in delta.items():
        dl[i] = d
    return select(snr, periods, dl, t_obs, group, primes_max, tol, order=pk, cap=cap, margin=margin)
