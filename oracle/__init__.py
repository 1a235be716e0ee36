"""CPU oracle for the FFA period search (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.

The arithmetic lives in ``oracle.cpp`` (plain C++17, FP64, compiled with
``-ffp-contract=off``); this module compiles it on first use and marshals
numpy arrays through ctypes.  Functions follow the paper:

* ``downsample``            -- Section 2.3 pre-/per-octave downsampling
* ``running_median[_at]``   -- Section 2.3 dynamic running-median dereddening
* ``normalise``             -- FP64 mean / population-std normalisation (+ int8 code)
* ``fold`` / ``fold_trial`` -- Section 2.1 FFA recursion (Eq. 1-2, padding rule)
* ``score_alg1``            -- Section 2.2.1 Algorithm 1 (Eq. 3-4)
* ``score_alg2``            -- Section 2.2.2 Algorithm 2 (Eq. 5), with its fixed-width "Ref" form
* ``plan`` / ``search`` / ``best`` -- the whole search, ffancy-style

Parity is pinned by ``tests/test_oracle_*.py`` against brute force, closed
forms and invariants; no oracle function is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to oracle.cpp (g++, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Score(C.Structure):
    _fields_ = [("snr", C.c_double), ("median", C.c_double), ("mad", C.c_double),
                ("width", C.c_int32), ("phase", C.c_int32), ("flags", C.c_int32),
                ("pad", C.c_int32)]


SCORE_DTYPE = np.dtype([("snr", "<f8"), ("median", "<f8"), ("mad", "<f8"), ("width", "<i4"),
                        ("phase", "<i4"), ("flags", "<i4"), ("pad", "<i4")])


class _Cfg(C.Structure):
    _fields_ = [("tsamp", C.c_double), ("period_min", C.c_double), ("period_max", C.c_double),
                ("duty", C.c_double), ("downsample0", C.c_int32),
                ("detrend_window", C.c_int32), ("min_rows", C.c_int32),
                ("fold_type", C.c_int32), ("n_widths_fixed", C.c_int32),
                ("widths_fixed", C.c_int32 * 16)]


PLAN_DTYPE = np.dtype([("octave", "<i4"), ("p0", "<i4"), ("m_data", "<i4"), ("m_rows", "<i4"),
                       ("n_widths", "<i4"), ("widths", "<i4", (16,)), ("pad", "<i4"),
                       ("n_octave", "<i8"), ("first_trial", "<i8")])

FOLD_F64, FOLD_F32, FOLD_I8 = 0, 1, 2


@dataclass
class Config:
    """Search configuration, periods in seconds (ffancy-style, Section 2.3)."""

    tsamp: float
    period_min: float
    period_max: float
    duty: float = 0.2
    downsample0: int = 1
    detrend_window: int = 0
    min_rows: int = 2
    fold_type: int = FOLD_F64
    widths: tuple = field(default_factory=tuple)

    def c(self) -> _Cfg:
        c = _Cfg()
        c.tsamp, c.period_min, c.period_max, c.duty = (self.tsamp, self.period_min,
                                                       self.period_max, self.duty)
        c.downsample0, c.detrend_window, c.min_rows = (self.downsample0, self.detrend_window,
                                                       self.min_rows)
        c.fold_type = self.fold_type
        c.n_widths_fixed = len(self.widths)
        for i, w in enumerate(self.widths):
            c.widths_fixed[i] = int(w)
        return c


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i64 = C.c_int64
            for name in ("oracle_downsample_f32", "oracle_downsample_u8", "oracle_downsample_f64"):
                getattr(L, name).argtypes = [P, i64, i64, P]
            L.oracle_running_median_at.argtypes = [P, i64, i64, P, i64, P]
            L.oracle_running_median.argtypes = [P, i64, i64, P]
            L.oracle_normalise.argtypes = [P, i64, P, P, P, P]
            L.oracle_normalise.restype = C.c_int
            for name in ("oracle_fold_f64", "oracle_fold_f32", "oracle_fold_i64"):
                getattr(L, name).argtypes = [P, i64, i64, P]
            for name in ("oracle_trial_f64", "oracle_trial_f32", "oracle_trial_i64"):
                getattr(L, name).argtypes = [P, i64, i64, i64, i64, P]
            for name in ("oracle_score_alg1_f64", "oracle_score_alg1_i64"):
                getattr(L, name).argtypes = [P, i64, P, C.c_int32, P]
            L.oracle_score_alg2_f64.argtypes = [P, i64, P, C.c_int32, C.c_double, P]
            L.oracle_plan.argtypes = [P, i64, P, i64, P, P]
            L.oracle_plan.restype = i64
            L.oracle_octave_series.argtypes = [P, P, i64, C.c_int, P, P, P, P, C.c_int]
            L.oracle_octave_series.restype = C.c_int
            L.oracle_fold_score_rows.argtypes = [C.c_int, P, P, P, i64, P, C.c_int]
            L.oracle_search.argtypes = [P, P, i64, C.c_int, P, i64, C.c_int]
            L.oracle_search.restype = C.c_int
            L.oracle_best.argtypes = [P, i64]
            L.oracle_best.restype = i64
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def downsample(x: np.ndarray, factor: int) -> np.ndarray:
    x = np.ascontiguousarray(x)
    y = np.empty(x.size // factor, np.float64)
    fn = {np.dtype(np.float32): "oracle_downsample_f32", np.dtype(np.uint8): "oracle_downsample_u8",
          np.dtype(np.float64): "oracle_downsample_f64"}[x.dtype]
    getattr(lib(), fn)(_p(x), x.size, factor, _p(y))
    return y


def running_median(x: np.ndarray, window: int) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(x)
    lib().oracle_running_median(_p(x), x.size, int(window), _p(out))
    return out


def running_median_at(x: np.ndarray, window: int, idx) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.empty(idx.size, np.float64)
    lib().oracle_running_median_at(_p(x), x.size, int(window), _p(idx), idx.size, _p(out))
    return out


def normalise(r: np.ndarray):
    """Return (z64, z32, q, mean, std, degenerate)."""
    r = np.ascontiguousarray(r, np.float64)
    z64 = np.empty(r.size, np.float64)
    z32 = np.empty(r.size, np.float32)
    q = np.empty(r.size, np.int8)
    ms = np.zeros(2, np.float64)
    deg = lib().oracle_normalise(_p(r), r.size, _p(z64), _p(z32), _p(q), _p(ms))
    return z64, z32, q, float(ms[0]), float(ms[1]), bool(deg)


def fold(rows: np.ndarray) -> np.ndarray:
    """FFA of an (M, P0) array, M a power of two; dtype float64, float32 or int64."""
    rows = np.ascontiguousarray(rows)
    m, p0 = rows.shape
    assert m >= 1 and (m & (m - 1)) == 0
    out = np.empty_like(rows)
    fn = {np.dtype(np.float64): "oracle_fold_f64", np.dtype(np.float32): "oracle_fold_f32",
          np.dtype(np.int64): "oracle_fold_i64"}[rows.dtype]
    getattr(lib(), fn)(_p(rows), m, p0, _p(out))
    return out


def fold_trial(z: np.ndarray, p0: int, m_data: int, m: int, k: int) -> np.ndarray:
    """Trial k of the fold of z packed as m_data rows of p0 bins (+ zero rows up to m)."""
    z = np.ascontiguousarray(z)
    assert z.size >= m_data * p0
    out = np.empty(p0, z.dtype)
    fn = {np.dtype(np.float64): "oracle_trial_f64", np.dtype(np.float32): "oracle_trial_f32",
          np.dtype(np.int64): "oracle_trial_i64"}[z.dtype]
    getattr(lib(), fn)(_p(z), p0, m_data, m, k, _p(out))
    return out


def score_alg1(profile: np.ndarray, widths) -> np.ndarray:
    """Algorithm 1 on one profile; returns a SCORE_DTYPE record."""
    w = np.ascontiguousarray(widths, np.int32)
    rec = np.zeros(1, SCORE_DTYPE)
    if profile.dtype == np.int64:
        x = np.ascontiguousarray(profile)
        lib().oracle_score_alg1_i64(_p(x), x.size, _p(w), w.size, _p(rec))
    else:
        x = np.ascontiguousarray(profile, np.float64)
        lib().oracle_score_alg1_f64(_p(x), x.size, _p(w), w.size, _p(rec))
    return rec[0]


def score_alg2(profile: np.ndarray, widths, excl_frac: float = 0.2) -> np.ndarray:
    """Algorithm 2 (Section 2.2.2, Eq. 5) on one profile; median/mad fields hold I_av/sigma."""
    w = np.ascontiguousarray(widths, np.int32)
    rec = np.zeros(1, SCORE_DTYPE)
    x = np.ascontiguousarray(profile, np.float64)
    lib().oracle_score_alg2_f64(_p(x), x.size, _p(w), w.size, float(excl_frac), _p(rec))
    return rec[0]


def plan(cfg: Config, n: int):
    """Return (plan rows, n_trials, detrend window)."""
    c = cfg.c()
    nt = C.c_int64()
    win = C.c_int32()
    L = lib()
    count = L.oracle_plan(C.byref(c), n, None, 0, C.byref(nt), C.byref(win))
    rows = np.zeros(count, PLAN_DTYPE)
    L.oracle_plan(C.byref(c), n, _p(rows), count, C.byref(nt), C.byref(win))
    return rows, int(nt.value), int(win.value)


def octave_series(cfg: Config, series: np.ndarray):
    """Dereddened, normalised series per octave as the search folds them (list of arrays)."""
    series = np.ascontiguousarray(series)
    in_type = 1 if series.dtype == np.uint8 else 0
    if in_type == 0:
        series = np.ascontiguousarray(series, np.float32)
    n = series.size
    total = 0
    n_o = n // max(cfg.downsample0, 1)
    for _ in range(63):
        total += n_o
        n_o //= 2
    z64 = np.empty(total + 1, np.float64) if cfg.fold_type == FOLD_F64 else None
    z32 = np.empty(total + 1, np.float32) if cfg.fold_type == FOLD_F32 else None
    q = np.empty(total + 1, np.int8) if cfg.fold_type == FOLD_I8 else None
    offs = np.zeros(64, np.int64)
    c = cfg.c()
    n_oct = lib().oracle_octave_series(C.byref(c), _p(series), n, in_type,
                                        None if z64 is None else _p(z64),
                                        None if z32 is None else _p(z32),
                                        None if q is None else _p(q), _p(offs), 63)
    buf = z64 if z64 is not None else (z32 if z32 is not None else q)
    return [buf[offs[o]:offs[o + 1]].copy() for o in range(n_oct)]


def search(cfg: Config, series: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Whole search; one SCORE_DTYPE record per trial in (octave, P0, trial) order."""
    series = np.ascontiguousarray(series)
    in_type = 1 if series.dtype == np.uint8 else 0
    if in_type == 0:
        series = np.ascontiguousarray(series, np.float32)
    _, nt, _ = plan(cfg, series.size)
    rec = np.zeros(max(nt, 1), SCORE_DTYPE)
    c = cfg.c()
    rc = lib().oracle_search(C.byref(c), _p(series), series.size, in_type, _p(rec), rec.size,
                             int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_search failed: {rc}")
    return rec[:nt]


def fold_score_rows(fold_type: int, octaves: list, rows: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Fold and score the given plan rows; ``octaves`` = octave_series(...) output.

    Returns one SCORE_DTYPE record per trial of the rows, in row order."""
    buf = np.concatenate(octaves) if octaves else np.zeros(1)
    offs = np.zeros(64, np.int64)
    offs[1:len(octaves) + 1] = np.cumsum([o.size for o in octaves])
    sub = np.ascontiguousarray(rows.copy())
    sub["first_trial"] = np.concatenate([[0], np.cumsum(sub["m_rows"][:-1].astype(np.int64))])
    total = int(sub["m_rows"].astype(np.int64).sum())
    rec = np.zeros(max(total, 1), SCORE_DTYPE)
    lib().oracle_fold_score_rows(int(fold_type), _p(buf), _p(offs), _p(sub), len(sub), _p(rec),
                                 int(nthreads))
    return rec[:total]


def best(records: np.ndarray) -> int:
    records = np.ascontiguousarray(records, SCORE_DTYPE)
    return int(lib().oracle_best(_p(records), records.size))


def trial_periods(plan_rows: np.ndarray, cfg: Config) -> np.ndarray:
    """Period in seconds of every trial (Eq. 2 with N = M*P0: P0 + k/(M-1) samples)."""
    out = []
    for r in plan_rows:
        m = int(r["m_rows"])
        k = np.arange(m, dtype=np.float64)
        scale = cfg.tsamp * max(cfg.downsample0, 1) * (2.0 ** int(r["octave"]))
        out.append((r["p0"] + k / (m - 1)) * scale)
    return np.concatenate(out) if out else np.zeros(0)
