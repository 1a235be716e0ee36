"""Splitting one search over several devices or processes, and merging.

Every base period of the search is independent (Section 2.1: one FFA
execution per P0), so a search shards into contiguous ranges of plan entries;
the only exchange is the small candidate lists, merged on the host with the
search's own order (higher S/N first, then the lower periodogram index, which
is the lower octave, P0 and trial).  Used by ffa.search_entries /
ffa.candidates_entries on each rank; no collective touches the data path.
"""
from __future__ import annotations

import numpy as np


def entry_cost(entries: np.ndarray) -> np.ndarray:
    """Relative work of each base period: the fold's M*P0*log2(M) adds plus
    scoring M*P0*(n_widths + 4)."""
    m = entries["m_rows"].astype(np.float64)
    p0 = entries["p0"].astype(np.float64)
    return m * p0 * (np.log2(np.maximum(m, 2.0)) + entries["n_widths"] + 4.0)


def split_entries(entries: np.ndarray, parts: int) -> list[tuple[int, int]]:
    """Contiguous ranges [b, e) of plan entries with about equal cost, one per part."""
    n = len(entries)
    if parts < 1:
        raise ValueError("parts must be >= 1")
    if n == 0:
        return [(0, 0)] * parts
    cum = np.concatenate([[0.0], np.cumsum(entry_cost(entries))])
    total = cum[-1]
    bounds = [0]
    for i in range(1, parts):
        b = int(np.searchsorted(cum, total * i / parts, side="left"))
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[i], bounds[i + 1]) for i in range(parts)]


def merge_candidates(lists, top_k: int) -> np.ndarray:
    """Merge per-rank candidate arrays (fields 'snr' and 'trial' at least):
    higher S/N first, ties to the lower trial index; keeps top_k."""
    lists = [np.asarray(x) for x in lists if len(x)]
    if not lists:
        return np.zeros(0, lists[0].dtype) if lists else np.zeros(0)
    allc = np.concatenate(lists)
    order = np.lexsort((allc["trial"], -allc["snr"].astype(np.float64)))
    return allc[order[:top_k]]
