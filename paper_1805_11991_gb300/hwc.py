"""Thin ctypes binding of libhwc (include/hwc.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Names follow the C ABI without the ``hwc_`` prefix.  If the
library cannot be loaded this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_RANGE, ERR_TOO_LARGE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_STATE = range(-1, -9, -1)
MAX_Q = 262144

FAM_ALL_DEG, FAM_MONIC_NOSUB, FAM_MONIC_NOSUB_SAMPLED, FAM_REDUCED = 0, 1, 2, 3
FAM_MONIC_NOSUB_SAMPLED_WINDOW = 4
FLAG_PLAIN, FLAG_GRAPH, FLAG_HORNER, FLAG_NO_TUNE, FLAG_TIMING, FLAG_FAN1 = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20
FLAG_ALL_POINTS = 0x40
FLAG_LAMBDA = 0x80


class HwcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hwc error {code}: {msg}")
        self.code = code


class Family(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("degree", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("sample_count", ctypes.c_uint64)]


class Job(ctypes.Structure):
    _fields_ = [("g", ctypes.c_uint32), ("q", ctypes.c_uint32), ("family", Family),
                ("first", ctypes.c_uint64), ("count", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_uint64), ("max_active", ctypes.c_uint32),
                ("step_items", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhwc.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise OSError(f"libhwc.so not built at {path}")
        lib = ctypes.CDLL(path)
        c_int, u32, u64, vp, sz = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
        P = ctypes.POINTER
        sigs = {
            "hwc_last_error": (ctypes.c_char_p, []),
            "hwc_version": (ctypes.c_char_p, []),
            "hwc_field_tables": (c_int, [u32, u32, P(vp)]),
            "hwc_tables_info": (c_int, [vp, P(u32), u32]),
            "hwc_tables_read": (c_int, [vp, P(u32), P(u32), P(u32), P(u32)]),
            "hwc_tables_free": (None, [vp]),
            "hwc_family_size": (c_int, [u32, P(Family), P(u64)]),
            "hwc_count": (c_int, [u32, u32, P(Family), u64, u64, u32, vp, P(vp)]),
            "hwc_count_members": (c_int, [u32, u32, P(Family), u64, u64, c_int, u32, vp,
                                          P(ctypes.c_int32), P(ctypes.c_uint8)]),
            "hwc_hist_size": (c_int, [vp, P(u64), P(u64), P(u64)]),
            "hwc_hist_genus": (c_int, [vp, P(u32)]),
            "hwc_hist_read": (c_int, [vp, P(ctypes.c_int32), P(u64)]),
            "hwc_hist_lambda": (c_int, [vp, P(u64)]),
            "hwc_hist_save": (c_int, [vp, P(Job), ctypes.c_char_p]),
            "hwc_hist_load": (c_int, [ctypes.c_char_p, P(vp), P(Job)]),
            "hwc_hist_merge": (c_int, [vp, vp]),
            "hwc_hist_from_arrays": (c_int, [u32, u64, P(ctypes.c_int32), P(u64), u64, P(vp)]),
            "hwc_hist_free": (None, [vp]),
            "hwc_batch_create": (c_int, [P(Job), sz, u32, P(vp)]),
            "hwc_batch_launch": (c_int, [vp, vp]),
            "hwc_batch_result": (c_int, [vp, sz, P(vp)]),
            "hwc_batch_kernel_launches": (c_int, [vp, P(u32)]),
            "hwc_batch_job_method": (c_int, [vp, ctypes.c_size_t, P(u32)]),
            "hwc_batch_io_bytes": (c_int, [vp, P(u64), P(u64)]),
            "hwc_batch_kernel_ms": (c_int, [vp, P(ctypes.c_float)]),
            "hwc_batch_free": (None, [vp]),
            "hwc_batch_run": (c_int, [P(Job), sz, u32, vp, P(vp)]),
            "hwc_serve_open": (c_int, [P(ServerConfig), P(vp)]),
            "hwc_serve_submit": (c_int, [vp, P(Job), P(u64)]),
            "hwc_serve_poll": (c_int, [vp, u64, u32, P(vp)]),
            "hwc_serve_latency": (c_int, [vp, u64, P(ctypes.c_double), P(ctypes.c_double)]),
            "hwc_serve_close": (c_int, [vp]),
            "hwc_probe_smem_gather": (c_int, [u32, u32, P(ctypes.c_double)]),
            "hwc_count_noalloc": (c_int, [u32, u32, P(Family), u64, u64, P(vp), u64, vp, vp, vp, vp]),
            "hwc_curve_count": (c_int, [u32, u32, u32, u64, P(u32), P(ctypes.c_int64), vp, P(ctypes.c_float)]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc < 0:
        msg = _lib.hwc_last_error().decode(errors="replace")
        raise HwcError(rc, msg)
    return rc


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


def make_family(kind: int, degree: int, seed: int = 0, sample_count: int = 0) -> Family:
    return Family(kind, degree, seed, sample_count)


def make_job(g: int, q: int, kind: int, degree: int, first: int = 0, count: int | None = None,
             seed: int = 0, sample_count: int = 0) -> Job:
    fam = make_family(kind, degree, seed, sample_count)
    if count is None:
        count = family_size(q, fam) - first
    return Job(g, q, fam, first, count)


# ---------------------------------------------------------------------------
# tables

class Tables:
    """Device-resident Zech tables of F_{q^k} (hwc_field_tables)."""

    def __init__(self, q: int, k: int):
        lib = load()
        self._h = ctypes.c_void_p()
        _check(lib.hwc_field_tables(q, k, ctypes.byref(self._h)))
        info = (ctypes.c_uint32 * 64)()
        n = _check(lib.hwc_tables_info(self._h, info, 64))
        v = list(info[:n])
        self.q, self.k, self.p, self.e, self.Q, self.L, self.n = v[:7]
        self.M = v[7:7 + self.n + 1]
        self.mq = v[7 + self.n + 1:7 + self.n + 1 + self.e + 1]

    def read(self):
        """(antilog[L], log[Q], zech[L], coef_log[q]) as numpy uint32 arrays."""
        a = np.zeros(self.L, np.uint32)
        lg = np.zeros(self.Q, np.uint32)
        z = np.zeros(self.L, np.uint32)
        c = np.zeros(self.q, np.uint32)
        P = ctypes.POINTER(ctypes.c_uint32)
        _check(_lib.hwc_tables_read(self._h, a.ctypes.data_as(P), lg.ctypes.data_as(P),
                                    z.ctypes.data_as(P), c.ctypes.data_as(P)))
        return a, lg, z, c

    def close(self):
        if getattr(self, "_h", None):
            _lib.hwc_tables_free(self._h)
            self._h = None

    __del__ = close


# ---------------------------------------------------------------------------
# histograms

@dataclass
class Histogram:
    g: int
    counts: np.ndarray      # int32 [n, g]: (#C_1..#C_g), sorted lexicographically
    mult: np.ndarray        # uint64 [n]
    n_squarefree: int
    n_total: int
    lam: np.ndarray | None = None   # uint64 [n]: factorisation pattern codes (HWC_FLAG_LAMBDA)

    def as_dict(self):
        return {tuple(int(v) for v in row): int(m) for row, m in zip(self.counts, self.mult)}


def _take_hist(h: ctypes.c_void_p) -> Histogram:
    try:
        n, nsq, ntot = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.hwc_hist_size(h, ctypes.byref(n), ctypes.byref(nsq), ctypes.byref(ntot)))
        g = ctypes.c_uint32()
        _check(_lib.hwc_hist_genus(h, ctypes.byref(g)))
        counts = np.zeros((n.value, g.value), np.int32)
        mult = np.zeros(n.value, np.uint64)
        _check(_lib.hwc_hist_read(h, counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  mult.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        lam = np.zeros(n.value, np.uint64)
        if _lib.hwc_hist_lambda(h, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))) != OK:
            lam = None
        return Histogram(g.value, counts, mult, nsq.value, ntot.value, lam)
    finally:
        _lib.hwc_hist_free(h)


def family_size(q: int, fam: Family) -> int:
    load()
    n = ctypes.c_uint64()
    _check(_lib.hwc_family_size(q, ctypes.byref(fam), ctypes.byref(n)))
    return n.value


def count(g: int, q: int, fam: Family, first: int, n: int, flags: int = 0, stream=None) -> Histogram:
    """hwc_count: histogram of (#C_1..#C_g) over square-free members."""
    load()
    h = ctypes.c_void_p()
    _check(_lib.hwc_count(g, q, ctypes.byref(fam), first, n, flags, _stream_ptr(stream), ctypes.byref(h)))
    return _take_hist(h)


def count_members(g: int, q: int, fam: Family, first: int, n: int, unfiltered: bool = False,
                  flags: int = 0, stream=None):
    """hwc_count_members: (counts int32[n, g], sqf uint8[n])."""
    load()
    counts = np.zeros((n, g), np.int32)
    sqf = np.zeros(n, np.uint8)
    _check(_lib.hwc_count_members(g, q, ctypes.byref(fam), first, n, 1 if unfiltered else 0, flags,
                                  _stream_ptr(stream),
                                  counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  sqf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return counts, sqf


def _to_handle(src: Histogram) -> ctypes.c_void_p:
    """A library histogram with the contents of `src` (without patterns)."""
    h = ctypes.c_void_p()
    c = np.ascontiguousarray(src.counts, np.int32)
    m = np.ascontiguousarray(src.mult, np.uint64)
    _check(_lib.hwc_hist_from_arrays(src.g, len(m), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), src.n_total,
                                     ctypes.byref(h)))
    return h


def hist_save(h: Histogram, path: str, job: Job | None = None) -> None:
    """hwc_hist_save: a checkpoint file of the histogram and the job range it counts."""
    load()
    if h.lam is not None:
        raise ValueError("checkpoints of pattern-keyed histograms are written by the C API")
    hh = _to_handle(h)
    try:
        _check(_lib.hwc_hist_save(hh, ctypes.byref(job) if job is not None else None, path.encode()))
    finally:
        _lib.hwc_hist_free(hh)


def hist_load(path: str):
    """hwc_hist_load: (histogram, job or None)."""
    load()
    h = ctypes.c_void_p()
    jb = Job()
    _check(_lib.hwc_hist_load(path.encode(), ctypes.byref(h), ctypes.byref(jb)))
    hist = _take_hist(h)
    return hist, (jb if jb.g else None)


def hist_merge(a: Histogram, b: Histogram) -> Histogram:
    load()
    ha, hb = ctypes.c_void_p(), ctypes.c_void_p()
    for src, h in ((a, ha), (b, hb)):
        c = np.ascontiguousarray(src.counts, np.int32)
        m = np.ascontiguousarray(src.mult, np.uint64)
        _check(_lib.hwc_hist_from_arrays(src.g, len(m), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), src.n_total,
                                         ctypes.byref(h)))
    try:
        _check(_lib.hwc_hist_merge(ha, hb))
    finally:
        _lib.hwc_hist_free(hb)
    return _take_hist(ha)


# ---------------------------------------------------------------------------
# batches

class Batch:
    """hwc_batch_*: many jobs, one persistent launch (or one launch per job)."""

    def __init__(self, jobs, flags: int = 0):
        lib = load()
        self.n = len(jobs)
        self._jobs = (Job * self.n)(*jobs)
        self._h = ctypes.c_void_p()
        _check(lib.hwc_batch_create(self._jobs, self.n, flags, ctypes.byref(self._h)))

    def launch(self, stream=None):
        _check(_lib.hwc_batch_launch(self._h, _stream_ptr(stream)))

    def result(self, i: int) -> Histogram:
        h = ctypes.c_void_p()
        _check(_lib.hwc_batch_result(self._h, i, ctypes.byref(h)))
        return _take_hist(h)

    def kernel_launches(self) -> int:
        n = ctypes.c_uint32()
        _check(_lib.hwc_batch_kernel_launches(self._h, ctypes.byref(n)))
        return n.value

    def job_method(self, i: int) -> int:
        """Count kernel of job i: 0 Horner, 1 fan-out over c_0, 2 over (c_1, c_0)."""
        m = ctypes.c_uint32()
        _check(_lib.hwc_batch_job_method(self._h, i, ctypes.byref(m)))
        return m.value

    def io_bytes(self):
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.hwc_batch_io_bytes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def kernel_ms(self) -> float:
        ms = ctypes.c_float()
        _check(_lib.hwc_batch_kernel_ms(self._h, ctypes.byref(ms)))
        return ms.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.hwc_batch_free(self._h)
            self._h = None

    __del__ = close


def batch_run(jobs, flags: int = 0, stream=None):
    lib = load()
    arr = (Job * len(jobs))(*jobs)
    outs = (ctypes.c_void_p * len(jobs))()
    _check(lib.hwc_batch_run(arr, len(jobs), flags, _stream_ptr(stream), outs))
    return [_take_hist(ctypes.c_void_p(o)) for o in outs]


def count_noalloc(g: int, q: int, fam: Family, first: int, n: int, tables, max_entries: int,
                  d_counts: int, d_mult: int, d_n_out: int, stream=None) -> None:
    """hwc_count_noalloc: the library allocates nothing; `tables` are the g
    Tables objects of F_{q^k}, k = 1..g, and d_counts / d_mult / d_n_out are
    DEVICE pointers (int32 [max_entries*g], uint64 [max_entries], uint64 [3])
    the caller owns."""
    load()
    handles = (ctypes.c_void_p * len(tables))(*[t._h.value for t in tables])
    _check(_lib.hwc_count_noalloc(g, q, ctypes.byref(fam), first, n, handles, max_entries,
                                  d_counts, d_mult, d_n_out, _stream_ptr(stream)))


def curve_count(q: int, k: int, coeffs, stream=None):
    """hwc_curve_count: #C(F_{q^k}) of explicit curves; coeffs int [n, d+1]
    (c_0..c_d digits).  Returns (counts int64 [n], device ms of the count)."""
    load()
    c = np.ascontiguousarray(np.atleast_2d(coeffs), dtype=np.uint32)
    n, d1 = c.shape
    counts = np.zeros(n, np.int64)
    ms = ctypes.c_float()
    _check(_lib.hwc_curve_count(q, k, d1 - 1, n, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _stream_ptr(stream),
                                ctypes.byref(ms)))
    return counts, ms.value


def probe_smem_gather(entries: int, iters: int = 4096) -> float:
    """Random 16-bit shared-memory reads per second (roofline denominator)."""
    load()
    r = ctypes.c_double()
    _check(_lib.hwc_probe_smem_gather(entries, iters, ctypes.byref(r)))
    return r.value


# ---------------------------------------------------------------------------
# serving

class Server:
    """hwc_serve_*: request loop with continuous batching."""

    def __init__(self, device_bytes: int = 8 << 30, max_active: int = 64, step_items: int = 0):
        lib = load()
        cfg = ServerConfig(device_bytes, max_active, step_items)
        self._h = ctypes.c_void_p()
        _check(lib.hwc_serve_open(ctypes.byref(cfg), ctypes.byref(self._h)))

    def submit(self, job: Job) -> int:
        t = ctypes.c_uint64()
        _check(_lib.hwc_serve_submit(self._h, ctypes.byref(job), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """Histogram if finished, else None."""
        h = ctypes.c_void_p()
        rc = _lib.hwc_serve_poll(self._h, ticket, timeout_ms, ctypes.byref(h))
        if rc == ERR_STATE and not h.value:
            msg = _lib.hwc_last_error().decode()
            if "not finished" in msg:
                return None
        _check(rc)
        return _take_hist(h)

    def latency(self, ticket: int):
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(_lib.hwc_serve_latency(self._h, ticket, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.hwc_serve_close(self._h)
            self._h = None

    __del__ = close
