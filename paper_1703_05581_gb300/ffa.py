"""Thin Python binding of the C ABI in include/ffa.h (argument marshalling only).

Every step of the search runs in the CUDA library libffa_gb300.so; PyTorch only
provides device memory and streams.  Importing this module raises if the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffa_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1703_05581_gb300.build_lib.build()")

_lib = C.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_CANCELLED, ERR_UNSUPPORTED, ERR_DEVICE = range(8)
IN_F32, IN_U8, IN_F64 = 0, 1, 2
SCORE_ALG1, SCORE_ALG2 = 0, 1
FOLD_F32, FOLD_I8 = 0, 1
STATS_DOUBLES = 1026
NOALLOC_FOLD_MAX_ELEMS = 8 * 1024 * 1024


class FFAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.ffa_status_string(status).decode()} ({status}): {msg}")
        self.status = status


class SearchConfig(C.Structure):
    _fields_ = [("tsamp_s", C.c_double), ("period_min_s", C.c_double),
                ("period_max_s", C.c_double), ("duty_max", C.c_double),
                ("downsample0", C.c_int32), ("detrend_window", C.c_int32),
                ("min_rows", C.c_int32), ("in_type", C.c_int32), ("precision", C.c_int32),
                ("n_widths_fixed", C.c_int32), ("widths_fixed", C.c_int32 * 16),
                ("scorer", C.c_int32), ("alg2_window", C.c_float), ("clip_sigma", C.c_float),
                ("persist_cutoff", C.c_float), ("persistence", C.c_int32)]


class Record(C.Structure):
    _fields_ = [("snr", C.c_float), ("width", C.c_int32), ("phase", C.c_int32),
                ("flags", C.c_uint32)]


class PlanEntry(C.Structure):
    _fields_ = [("octave", C.c_int32), ("p0", C.c_int32), ("m_data", C.c_int32),
                ("m_rows", C.c_int32), ("n_widths", C.c_int32), ("widths", C.c_int32 * 16),
                ("pad", C.c_int32), ("n_octave", C.c_int64), ("first_trial", C.c_int64)]


class Candidate(C.Structure):
    _fields_ = [("trial", C.c_int64), ("period_s", C.c_double), ("snr", C.c_float),
                ("octave", C.c_int32), ("p0", C.c_int32), ("k", C.c_int32),
                ("width", C.c_int32), ("phase", C.c_int32)]


class BestConfig(C.Structure):
    _fields_ = [("snr_min", C.c_double), ("drop_frac", C.c_double), ("drop_abs", C.c_double),
                ("group", C.c_int32), ("primes_max", C.c_int32), ("harm_tol", C.c_double),
                ("group_margin", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("d_arena", C.c_void_p), ("arena_bytes", C.c_size_t), ("n_slots", C.c_int32),
                ("timeout_ms", C.c_int32)]


RECORD_DTYPE = np.dtype([("snr", "<f4"), ("width", "<i4"), ("phase", "<i4"), ("flags", "<u4")])
ENTRY_DTYPE = np.dtype([("octave", "<i4"), ("p0", "<i4"), ("m_data", "<i4"), ("m_rows", "<i4"),
                        ("n_widths", "<i4"), ("widths", "<i4", (16,)), ("pad", "<i4"),
                        ("n_octave", "<i8"), ("first_trial", "<i8")])
CANDIDATE_DTYPE = np.dtype([("trial", "<i8"), ("period_s", "<f8"), ("snr", "<f4"),
                            ("octave", "<i4"), ("p0", "<i4"), ("k", "<i4"), ("width", "<i4"),
                            ("phase", "<i4")])
assert C.sizeof(Record) == 16 and RECORD_DTYPE.itemsize == 16
assert C.sizeof(PlanEntry) == ENTRY_DTYPE.itemsize
assert C.sizeof(Candidate) == CANDIDATE_DTYPE.itemsize

_P, _i64, _i32 = C.c_void_p, C.c_int64, C.c_int32
_sig = {
    "ffa_plan_create": ([C.POINTER(SearchConfig), _i64, C.POINTER(C.c_void_p)], C.c_int),
    "ffa_plan_destroy": ([_P], None),
    "ffa_plan_info": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "ffa_plan_entries": ([_P, _P, _i64], C.c_int),
    "ffa_plan_periods": ([_P, _i64, _i64, _P], C.c_int),
    "ffa_search_series": ([_P, _P, _i32, _i32, _P, C.c_size_t, _P, _P, _P], C.c_int),
    "ffa_search_plane": ([_P, _P, _i64, _P, C.c_size_t, _P, _P, _P], C.c_int),
    "ffa_search": ([_P, _P, _P, C.c_size_t, _P, _P, _P], C.c_int),
    "ffa_search_entries": ([_P, _P, _i64, _i64, _P, C.c_size_t, _P, _P, _P], C.c_int),
    "ffa_search_persistence": ([_P, _P, _P, C.c_size_t, _P, _P, _P, _P], C.c_int),
    "ffa_autotune": ([_P, _P, C.c_size_t, _P, _P], C.c_int),
    "ffa_search_batch": ([_P, _P, _i32, _P, C.c_size_t, _P, _P, _P], C.c_int),
    "ffa_batch_workspace_bytes": ([_P, _i32, _P], C.c_int),
    "ffa_candidates": ([_P, _P, C.c_double, _i32, _P, C.c_size_t, _P, _P, _P, _P, _P, _i32],
                       C.c_int),
    "ffa_candidates_entries": ([_P, _i64, _i64, _P, C.c_double, _i32, _P, C.c_size_t, _P, _P, _P, _P,
                                _P, _i32], C.c_int),
    "ffa2best": ([_P, _P, C.POINTER(BestConfig), _P, C.c_size_t, _P, _i32, _P, _P, _P, _P, _i32],
                 C.c_int),
    "ffa_snr_histogram": ([_P, _i64, _P, _i32, _P, _P], C.c_int),
    "ffa_sigma_gauss": ([_P, _i32, _P], C.c_int),
    "ffa_server_request_bytes": ([C.POINTER(SearchConfig), _i64, _P], C.c_int),
    "ffa_server_create": ([C.POINTER(ServerConfig), C.POINTER(C.c_void_p)], C.c_int),
    "ffa_server_submit": ([_P, C.POINTER(SearchConfig), _P, _i64, C.c_double, _i32, _P, _P], C.c_int),
    "ffa_server_wait": ([_P, _i64, _i32, _P, _i32, _P, _P, _P], C.c_int),
    "ffa_server_stats": ([_P, _P, _P, _P], C.c_int),
    "ffa_server_destroy": ([_P], None),
    "ffa_wait": ([_P, _P, _i32], C.c_int),
    "ffa_downsample": ([_P, _i32, _i64, _i64, _P, _P], C.c_int),
    "ffa_detrend": ([_P, _i64, _i32, _P, _P, _P], C.c_int),
    "ffa_normalise": ([_P, _i64, _i32, _P, _P, _P], C.c_int),
    "ffa_fold": ([_P, _i32, _i64, _i64, _i64, _P, _P, _P], C.c_int),
    "ffa_fold_noalloc": ([_P, _i32, _i64, _i64, _i64, _P, _P], C.c_int),
    "ffa_score": ([_P, _i32, _i64, _i64, _P, _i32, _P, _P, _P], C.c_int),
    "ffa_score_alg2": ([_P, _i32, _i64, _i64, _P, _i32, C.c_float, _P, _P], C.c_int),
    "ffa_timing_enable": ([_i32], C.c_int),
    "ffa_launch_count": ([], C.c_int64),
    "ffa_timing_read": ([_P, _P, _i32], C.c_int),
    "ffa_status_string": ([C.c_int], C.c_char_p),
    "ffa_last_error": ([], C.c_char_p),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTS = tuple(_sig)


def _check(status: int) -> None:
    if status != OK:
        raise FFAError(status, _lib.ffa_last_error().decode())


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


@dataclass
class Config:
    """Search configuration (periods in seconds), mirrors ffa_search_config."""

    tsamp: float
    period_min: float
    period_max: float
    duty: float = 0.2
    downsample0: int = 1
    detrend_window: int = 0
    min_rows: int = 2
    in_type: int = IN_F32
    precision: int = FOLD_F32
    widths: tuple = field(default_factory=tuple)
    scorer: int = SCORE_ALG1
    alg2_window: float = 0.0
    clip_sigma: float = 0.0
    persist_cutoff: float = 0.0
    persistence: bool = False

    def c(self) -> SearchConfig:
        c = SearchConfig()
        c.tsamp_s, c.period_min_s, c.period_max_s, c.duty_max = (
            self.tsamp, self.period_min, self.period_max, self.duty)
        c.downsample0, c.detrend_window, c.min_rows = (self.downsample0, self.detrend_window,
                                                       self.min_rows)
        c.in_type, c.precision = self.in_type, self.precision
        c.n_widths_fixed = len(self.widths)
        for i, w in enumerate(self.widths):
            c.widths_fixed[i] = int(w)
        c.scorer, c.alg2_window = self.scorer, self.alg2_window
        c.clip_sigma, c.persist_cutoff = self.clip_sigma, self.persist_cutoff
        c.persistence = int(bool(self.persistence))
        return c


class Plan:
    """ffa_plan for a series of n input samples."""

    def __init__(self, cfg: Config, n: int):
        self.cfg = cfg
        self.n = int(n)
        h = C.c_void_p()
        self._c = cfg.c()
        _check(_lib.ffa_plan_create(C.byref(self._c), self.n, C.byref(h)))
        self._h = h
        npd, nt, no = C.c_int64(), C.c_int64(), C.c_int32()
        win, ws = C.c_int32(), C.c_size_t()
        _check(_lib.ffa_plan_info(h, C.byref(npd), C.byref(nt), C.byref(no), C.byref(win),
                                  C.byref(ws)))
        self.n_periods, self.n_trials, self.n_octaves = npd.value, nt.value, no.value
        self.window, self.workspace_bytes = win.value, ws.value
        self.entries = np.zeros(self.n_periods, ENTRY_DTYPE)
        if self.n_periods:
            _check(_lib.ffa_plan_entries(h, self.entries.ctypes.data_as(C.c_void_p),
                                         self.n_periods))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ffa_plan_destroy(h)
            self._h = None

    def periods(self, trial_begin: int = 0, count: int | None = None) -> np.ndarray:
        """Trial periods in seconds (ffa_plan_periods: Eq. 2, computed by the library)."""
        count = self.n_trials - trial_begin if count is None else int(count)
        out = np.zeros(max(count, 0), np.float64)
        _check(_lib.ffa_plan_periods(self._h, int(trial_begin), count, out.ctypes.data_as(C.c_void_p)))
        return out

    def workspace(self, device=None) -> torch.Tensor:
        dev = device or torch.device("cuda", torch.cuda.current_device())
        return torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=dev)

    def records(self, device=None) -> torch.Tensor:
        dev = device or torch.device("cuda", torch.cuda.current_device())
        return torch.empty((max(self.n_trials, 1), 4), dtype=torch.int32, device=dev)


def status_word(device=None) -> torch.Tensor:
    dev = device or torch.device("cuda", torch.cuda.current_device())
    return torch.zeros(1, dtype=torch.int32, device=dev)


def search(plan: Plan, series: torch.Tensor, workspace: torch.Tensor | None = None,
           records: torch.Tensor | None = None, status: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """Enqueue the whole search; returns the (n_trials, 4) int32 view of the records."""
    assert series.is_cuda and series.is_contiguous() and series.numel() == plan.n
    workspace = plan.workspace(series.device) if workspace is None else workspace
    records = plan.records(series.device) if records is None else records
    status = status_word(series.device) if status is None else status
    _check(_lib.ffa_search(plan._h, _ptr(series), _ptr(workspace), workspace.numel(),
                           _ptr(records), _ptr(status), _stream(stream)))
    return records


def search_persistence(plan: Plan, series: torch.Tensor, workspace: torch.Tensor | None = None,
                       records: torch.Tensor | None = None, persist: torch.Tensor | None = None,
                       status: torch.Tensor | None = None, stream=None):
    """ffa_search plus the per-trial persistence score: (records, persist)."""
    dev = series.device
    workspace = plan.workspace(dev) if workspace is None else workspace
    records = plan.records(dev) if records is None else records
    if persist is None:
        persist = torch.zeros(max(plan.n_trials, 1), dtype=torch.int32, device=dev)
    status = status_word(dev) if status is None else status
    _check(_lib.ffa_search_persistence(plan._h, _ptr(series), _ptr(workspace), workspace.numel(),
                                       _ptr(records), _ptr(persist), _ptr(status), _stream(stream)))
    return records, persist


def autotune(plan: Plan, workspace: torch.Tensor, stream=None) -> int:
    """Tune the fold's stages per pass for the plan's shapes; returns their count."""
    n = C.c_int32()
    _check(_lib.ffa_autotune(plan._h, _ptr(workspace), workspace.numel(), _stream(stream), C.byref(n)))
    return n.value


def search_entries(plan: Plan, series: torch.Tensor, entry_begin: int, entry_end: int,
                   workspace: torch.Tensor | None = None, records: torch.Tensor | None = None,
                   status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Search only plan entries [entry_begin, entry_end); records of other trials untouched."""
    assert series.is_cuda and series.is_contiguous() and series.numel() == plan.n
    workspace = plan.workspace(series.device) if workspace is None else workspace
    records = plan.records(series.device) if records is None else records
    status = status_word(series.device) if status is None else status
    _check(_lib.ffa_search_entries(plan._h, _ptr(series), int(entry_begin), int(entry_end),
                                   _ptr(workspace), workspace.numel(), _ptr(records), _ptr(status),
                                   _stream(stream)))
    return records


DUMP_RESID, DUMP_Z = 0, 1


def search_series(plan: Plan, series: torch.Tensor, octave: int, what: int = DUMP_Z,
                  workspace: torch.Tensor | None = None, status: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Octave `octave`'s dereddened series (DUMP_RESID, float64) or fold input
    (DUMP_Z: float32 z, or the int8 code), as the search prepares it."""
    assert series.is_cuda and series.is_contiguous() and series.numel() == plan.n
    dev = series.device
    workspace = plan.workspace(dev) if workspace is None else workspace
    status = status_word(dev) if status is None else status
    n_o = int(plan.entries["n_octave"][plan.entries["octave"] == octave][0])
    dt = torch.float64 if what == DUMP_RESID else (
        torch.float32 if plan.cfg.precision == FOLD_F32 else torch.int8)
    out = torch.empty(max(n_o, 1), dtype=dt, device=dev)
    _check(_lib.ffa_search_series(plan._h, _ptr(series), int(octave), int(what), _ptr(workspace),
                                  workspace.numel(), _ptr(out), _ptr(status), _stream(stream)))
    return out[:n_o]


def search_plane(plan: Plan, series: torch.Tensor, entry: int, workspace: torch.Tensor | None = None,
                 status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Every folded profile of plan entry `entry`: an (M, P0) tensor, row k = trial k."""
    assert series.is_cuda and series.is_contiguous() and series.numel() == plan.n
    dev = series.device
    workspace = plan.workspace(dev) if workspace is None else workspace
    status = status_word(dev) if status is None else status
    e = plan.entries[int(entry)]
    dt = torch.float32 if plan.cfg.precision == FOLD_F32 else torch.int32
    plane = torch.empty((int(e["m_rows"]), int(e["p0"])), dtype=dt, device=dev)
    _check(_lib.ffa_search_plane(plan._h, _ptr(series), int(entry), _ptr(workspace), workspace.numel(),
                                 _ptr(plane), _ptr(status), _stream(stream)))
    return plane


def batch_workspace_bytes(plans) -> int:
    """Workspace bytes ffa_search_batch needs for this batch of plans."""
    n = len(plans)
    hp = (C.c_void_p * n)(*[p._h.value for p in plans])
    b = C.c_size_t()
    _check(_lib.ffa_batch_workspace_bytes(hp, n, C.byref(b)))
    return b.value


def search_batch(plans, series, workspace: torch.Tensor | None = None, records=None,
                 status: torch.Tensor | None = None, stream=None):
    """Search a batch of series (uneven lengths, one configuration), base periods
    of all series folded and scored together; returns the record tensors."""
    assert len(plans) == len(series)
    dev = series[0].device
    need = batch_workspace_bytes(plans)
    workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev) if workspace is None else workspace
    records = [p.records(dev) for p in plans] if records is None else records
    status = status_word(dev) if status is None else status
    n = len(plans)
    hp = (C.c_void_p * n)(*[p._h.value for p in plans])
    hs = (C.c_void_p * n)(*[t.data_ptr() for t in series])
    hr = (C.c_void_p * n)(*[r.data_ptr() for r in records])
    _check(_lib.ffa_search_batch(hp, hs, n, _ptr(workspace), workspace.numel(), hr, _ptr(status),
                                 _stream(stream)))
    return records


def records_numpy(records: torch.Tensor, n: int) -> np.ndarray:
    return records[:n].cpu().numpy().view(RECORD_DTYPE).reshape(-1)


def candidates(plan: Plan, records: torch.Tensor, workspace: torch.Tensor, snr_min: float,
               top_k: int = 64, status: torch.Tensor | None = None, stream=None,
               timeout_ms: int = 600000):
    """Return (candidates structured array, best trial index)."""
    status = status_word(records.device) if status is None else status
    out = np.zeros(max(top_k, 1), CANDIDATE_DTYPE)
    n_out, best = C.c_int32(), C.c_int64()
    _check(_lib.ffa_candidates(plan._h, _ptr(records), float(snr_min), int(top_k),
                               _ptr(workspace), workspace.numel(),
                               out.ctypes.data_as(C.c_void_p), C.byref(n_out), C.byref(best),
                               _ptr(status), _stream(stream), int(timeout_ms)))
    return out[: n_out.value], best.value


def candidates_entries(plan: Plan, entry_begin: int, entry_end: int, records: torch.Tensor,
                       workspace: torch.Tensor, snr_min: float, top_k: int = 64,
                       status: torch.Tensor | None = None, stream=None, timeout_ms: int = 600000):
    """Candidates among the trials of plan entries [entry_begin, entry_end)."""
    status = status_word(records.device) if status is None else status
    out = np.zeros(max(top_k, 1), CANDIDATE_DTYPE)
    n_out, best = C.c_int32(), C.c_int64()
    _check(_lib.ffa_candidates_entries(plan._h, int(entry_begin), int(entry_end), _ptr(records),
                                       float(snr_min), int(top_k), _ptr(workspace), workspace.numel(),
                                       out.ctypes.data_as(C.c_void_p), C.byref(n_out), C.byref(best),
                                       _ptr(status), _stream(stream), int(timeout_ms)))
    return out[: n_out.value], best.value


def ffa2best(plan: Plan, records: torch.Tensor, workspace: torch.Tensor, snr_min: float,
             drop_frac: float = 0.1, drop_abs: float = 0.5, group: bool = True,
             primes_max: int = 31, harm_tol: float = 1e-5, group_margin: float = 0.16,
             cap: int = 256, status: torch.Tensor | None = None, stream=None,
             timeout_ms: int = 600000):
    """Candidate selection of Section 2.3.3 on the device periodogram: returns
    (kept candidates strongest first, number of periodogram peaks found)."""
    status = status_word(records.device) if status is None else status
    cfg = BestConfig(float(snr_min), float(drop_frac), float(drop_abs), int(bool(group)),
                     int(primes_max), float(harm_tol), float(group_margin))
    out = np.zeros(max(cap, 1), CANDIDATE_DTYPE)
    n_out, n_peaks = C.c_int32(), C.c_int64()
    _check(_lib.ffa2best(plan._h, _ptr(records), C.byref(cfg), _ptr(workspace), workspace.numel(),
                         out.ctypes.data_as(C.c_void_p), int(cap), C.byref(n_out), C.byref(n_peaks),
                         _ptr(status), _stream(stream), int(timeout_ms)))
    return out[: n_out.value], n_peaks.value


def snr_histogram(records: torch.Tensor, n: int, edges, counts: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Add the S/N histogram of the first n records to `counts` (int64 device
    tensor of len(edges) + 1 counters: below, each bin, at/above the top)."""
    e = np.ascontiguousarray(edges, dtype=np.float32)
    if counts is None:
        counts = torch.zeros(e.size + 1, dtype=torch.int64, device=records.device)
    _check(_lib.ffa_snr_histogram(_ptr(records), int(n), e.ctypes.data_as(C.c_void_p), e.size - 1,
                                  _ptr(counts), _stream(stream)))
    return counts


def sigma_gauss(counts) -> np.ndarray:
    """Gaussian-equivalent sigma at each histogram edge (host counts)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    out = np.zeros(c.size - 1)
    _check(_lib.ffa_sigma_gauss(c.ctypes.data_as(C.c_void_p), c.size - 2,
                                out.ctypes.data_as(C.c_void_p)))
    return out


def request_bytes(cfg: Config, n: int) -> int:
    b = C.c_size_t()
    c = cfg.c()
    _check(_lib.ffa_server_request_bytes(C.byref(c), int(n), C.byref(b)))
    return b.value


class Server:
    """Continuous-batching request loop (ffa_server_*): `arena_bytes` of device
    memory is the admission budget, `n_slots` searches run at once."""

    def __init__(self, arena_bytes: int, n_slots: int = 4, device=None, timeout_ms: int = 600000):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        cfg = ServerConfig(C.c_void_p(self.arena.data_ptr()), int(arena_bytes), int(n_slots),
                           int(timeout_ms))
        h = C.c_void_p()
        with torch.cuda.device(dev):
            _check(_lib.ffa_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep = {}  # ticket -> host buffers that must outlive the request

    def submit(self, cfg: Config, series: np.ndarray, snr_min: float = 6.0, top_k: int = 16,
               records: bool = False) -> int:
        x = np.ascontiguousarray(series)
        c = cfg.c()
        rec = None
        if records:
            rec = np.zeros(max(Plan(cfg, x.size).n_trials, 1), RECORD_DTYPE)
        t = C.c_int64()
        _check(_lib.ffa_server_submit(self._h, C.byref(c), x.ctypes.data_as(C.c_void_p), x.size,
                                      float(snr_min), int(top_k),
                                      None if rec is None else rec.ctypes.data_as(C.c_void_p),
                                      C.byref(t)))
        self._keep[t.value] = (x, c, rec, top_k)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Return (candidates, best, records or None, times_ms [queued, running, total])."""
        x, c, rec, top_k = self._keep[ticket]
        out = np.zeros(max(top_k, 1), CANDIDATE_DTYPE)
        n_out, best = C.c_int32(), C.c_int64()
        times = np.zeros(3)
        try:
            _check(_lib.ffa_server_wait(self._h, int(ticket), int(timeout_ms),
                                        out.ctypes.data_as(C.c_void_p), int(top_k), C.byref(n_out),
                                        C.byref(best), times.ctypes.data_as(C.c_void_p)))
        except FFAError as e:
            if e.status != ERR_TIMEOUT:
                self._keep.pop(ticket, None)
            raise
        self._keep.pop(ticket, None)
        return out[: n_out.value], best.value, rec, times

    def stats(self):
        q, f, u = C.c_int64(), C.c_int64(), C.c_size_t()
        _check(_lib.ffa_server_stats(self._h, C.byref(q), C.byref(f), C.byref(u)))
        return q.value, f.value, u.value

    def close(self) -> None:
        if self._h:
            _lib.ffa_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wait(status: torch.Tensor | None = None, stream=None, timeout_ms: int = 600000) -> None:
    _check(_lib.ffa_wait(_stream(stream), _ptr(status), int(timeout_ms)))


def timing_enable(on: bool) -> None:
    _check(_lib.ffa_timing_enable(1 if on else 0))


def launch_count() -> int:
    return int(_lib.ffa_launch_count())


TIMING_SAMPLE = 64  # phases 2/3 time every 64th base period of each octave


def timing_read():
    """Return (ms[6, 64], counts[6, 64]) summed per (phase, octave); clears the record.

    Phases: 0 preparation, 1 fold + score, 2 fold launches and 3 scoring launch
    of every TIMING_SAMPLE-th base period of the octave, 4 and 5 the same for
    the groups of short base periods holding one of them."""
    ms = np.zeros(384, np.float64)
    cnt = np.zeros(384, np.int32)
    _check(_lib.ffa_timing_read(ms.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p), 384))
    return ms.reshape(6, 64), cnt.reshape(6, 64)


# ---- individual steps --------------------------------------------------------

_IN_TYPES = {torch.float32: IN_F32, torch.uint8: IN_U8, torch.float64: IN_F64}


def downsample(x: torch.Tensor, factor: int, stream=None) -> torch.Tensor:
    out = torch.empty(x.numel() // factor, dtype=torch.float64, device=x.device)
    _check(_lib.ffa_downsample(_ptr(x), _IN_TYPES[x.dtype], x.numel(), int(factor), _ptr(out),
                               _stream(stream)))
    return out


def detrend(raw: torch.Tensor, window: int, status: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    assert raw.dtype == torch.float64
    out = torch.empty_like(raw)
    _check(_lib.ffa_detrend(_ptr(raw), raw.numel(), int(window), _ptr(out), _ptr(status),
                            _stream(stream)))
    return out


def normalise(resid: torch.Tensor, precision: int = FOLD_F32, stream=None):
    """Return (z or q, stats tensor whose first two entries are mean and std)."""
    dt = torch.float32 if precision == FOLD_F32 else torch.int8
    out = torch.empty(resid.numel(), dtype=dt, device=resid.device)
    stats = torch.zeros(STATS_DOUBLES, dtype=torch.float64, device=resid.device)
    _check(_lib.ffa_normalise(_ptr(resid), resid.numel(), precision, _ptr(out), _ptr(stats),
                              _stream(stream)))
    return out, stats


def fold(z: torch.Tensor, p0: int, m_data: int, m_rows: int, stream=None) -> torch.Tensor:
    prec = FOLD_F32 if z.dtype == torch.float32 else FOLD_I8
    dt = torch.float32 if prec == FOLD_F32 else torch.int32
    plane = torch.empty((m_rows, p0), dtype=dt, device=z.device)
    tmp = torch.empty_like(plane)
    _check(_lib.ffa_fold(_ptr(z), prec, int(p0), int(m_data), int(m_rows), _ptr(plane), _ptr(tmp),
                         _stream(stream)))
    return plane


def score(profiles: torch.Tensor, widths, status: torch.Tensor | None = None,
          stream=None) -> torch.Tensor:
    prec = FOLD_F32 if profiles.dtype == torch.float32 else FOLD_I8
    count, p0 = profiles.shape
    w = np.ascontiguousarray(widths, np.int32)
    rec = torch.empty((max(count, 1), 4), dtype=torch.int32, device=profiles.device)
    _check(_lib.ffa_score(_ptr(profiles), prec, count, p0, w.ctypes.data_as(C.c_void_p), w.size,
                          _ptr(rec), _ptr(status), _stream(stream)))
    return rec


def score_alg2(profiles: torch.Tensor, widths, excl_frac: float = 0.2, stream=None) -> torch.Tensor:
    """Algorithm 2 (Section 2.2.2) on (count, p0) profiles; returns (count, 4) int32 records."""
    prec = FOLD_F32 if profiles.dtype == torch.float32 else FOLD_I8
    count, p0 = profiles.shape
    w = np.ascontiguousarray(widths, np.int32)
    rec = torch.empty((max(count, 1), 4), dtype=torch.int32, device=profiles.device)
    _check(_lib.ffa_score_alg2(_ptr(profiles), prec, count, p0, w.ctypes.data_as(C.c_void_p), w.size,
                               float(excl_frac), _ptr(rec), _stream(stream)))
    return rec
