"""CPU oracle for hyperelliptic point counts (ctypes wrapper of hwc_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library never imports it and shares no code with it.

The oracle computes the plain definition of Sec. 1.1 (point count from r^0,
r^sq and the points at infinity) with polynomial-basis field arithmetic
(Sec. 2.2) and no Zech logarithms; see the header of hwc_oracle.c.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hwc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

ALL, MZ, MZ_SAMPLED = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hwc_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_uint64
        P32 = ctypes.POINTER(ctypes.c_int32)
        P8 = ctypes.POINTER(ctypes.c_uint8)
        lib.orc_field_new.restype = vp
        lib.orc_field_new.argtypes = [i32, i32, i32, i32]
        lib.orc_field_free.restype = None
        lib.orc_field_free.argtypes = [vp]
        lib.orc_field_info.restype = i32
        lib.orc_field_info.argtypes = [vp, P32]
        for name in ("orc_fq_add", "orc_fq_mul"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [vp, i32, i32]
        for name in ("orc_fQ_add", "orc_fQ_mul"):
            f = getattr(lib, name)
            f.restype = i64
            f.argtypes = [vp, i64, i64]
        for name in ("orc_chi", "orc_chi_euler"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [vp, i64]
        lib.orc_eval.restype = i64
        lib.orc_eval.argtypes = [vp, i32, P32, i64]
        lib.orc_squarefree.restype = i32
        lib.orc_squarefree.argtypes = [vp, i32, P32]
        lib.orc_family_size.restype = u64
        lib.orc_family_size.argtypes = [i32, i32, i32, u64]
        lib.orc_decode.restype = i32
        lib.orc_decode.argtypes = [i32, i32, i32, u64, u64, P32]
        lib.orc_count_polys.restype = i32
        lib.orc_count_polys.argtypes = [i32, i32, i32, i32, u64, u64, u64, u64,
                                        i32, i32, i32, i32, P32, P8]
        u32 = ctypes.c_uint32
        P64 = ctypes.POINTER(ctypes.c_uint64)
        lib.hwc_cpu_count.restype = i32
        lib.hwc_cpu_count.argtypes = [u32, u32, u32, u32, u64, u64, u64, u64, i32, u64, P32, P64, P64, P64]
        _lib = lib
        return lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class Field:
    """F_{q^k} of the oracle (tower F_p[T]/m -> F_q[U]/h), for element tests."""

    def __init__(self, q: int, k: int = 1, m_choice: int = 0, h_choice: int = 0):
        self._lib = _load()
        self._h = self._lib.orc_field_new(q, k, m_choice, h_choice)
        if not self._h:
            raise ValueError(f"oracle cannot build F_{q}^{k}")
        info = np.zeros(64, dtype=np.int32)
        self._lib.orc_field_info(self._h, _p32(info))
        self.p, self.e, self.q, self.k, self.Q = (int(v) for v in info[:5])
        self.m = [int(v) for v in info[5:5 + self.e + 1]]
        self.h = [int(v) for v in info[5 + self.e + 1:5 + self.e + 1 + self.k + 1]]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_field_free(h)
            self._h = None

    # F_q (subfield) arithmetic on canonical digits
    def fq_add(self, a, b):
        return self._lib.orc_fq_add(self._h, a, b)

    def fq_mul(self, a, b):
        return self._lib.orc_fq_mul(self._h, a, b)

    # F_Q arithmetic on element integers
    def add(self, y, z):
        return self._lib.orc_fQ_add(self._h, y, z)

    def mul(self, y, z):
        return self._lib.orc_fQ_mul(self._h, y, z)

    def chi(self, y):
        return self._lib.orc_chi(self._h, y)

    def chi_euler(self, y):
        return self._lib.orc_chi_euler(self._h, y)

    def eval(self, coeffs, x):
        c = np.ascontiguousarray(coeffs, dtype=np.int32)
        return self._lib.orc_eval(self._h, len(c) - 1, _p32(c), x)

    def squarefree(self, coeffs):
        c = np.ascontiguousarray(coeffs, dtype=np.int32)
        return bool(self._lib.orc_squarefree(self._h, len(c) - 1, _p32(c)))


def family_size(q: int, kind: int, degree: int, sample_count: int = 0) -> int:
    return int(_load().orc_family_size(q, kind, degree, sample_count))


def decode(q: int, kind: int, degree: int, idx: int, seed: int = 0):
    c = np.zeros(degree + 1, dtype=np.int32)
    if _load().orc_decode(q, kind, degree, seed, idx, _p32(c)) != 0:
        raise ValueError("bad family")
    return [int(v) for v in c]


def count_polys(g: int, q: int, kind: int, degree: int, first: int, count: int, *,
                seed: int = 0, sample_count: int = 0, filter: bool = True,
                m_choice: int = 0, h_choice: int = 0, threads: int | None = None):
    """Per-member point counts.

    Returns (counts int32[count, g] with counts[i, k-1] = #C(F_{q^k}),
    sqf uint8[count]).  With filter=True non-square-free members are not
    evaluated and get counts 0.
    """
    lib = _load()
    if threads is None:
        threads = os.cpu_count() or 1
    counts = np.zeros((count, g), dtype=np.int32)
    sqf = np.zeros(count, dtype=np.uint8)
    rc = lib.orc_count_polys(g, q, kind, degree, seed, sample_count, first, count,
                             1 if filter else 0, m_choice, h_choice, threads,
                             _p32(counts), sqf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError(f"oracle count failed rc={rc}")
    return counts, sqf


def histogram(counts: np.ndarray, sqf: np.ndarray):
    """Multiset of #C tuples over the square-free members: (tuples int32[n, g]
    sorted lexicographically, multiplicities uint64[n])."""
    sel = counts[sqf.astype(bool)]
    if sel.shape[0] == 0:
        return np.zeros((0, counts.shape[1]), np.int32), np.zeros(0, np.uint64)
    tuples, mult = np.unique(sel, axis=0, return_counts=True)
    return tuples.astype(np.int32), mult.astype(np.uint64)


def count_histogram(g: int, q: int, kind: int, degree: int, first: int, count: int, **kw):
    counts, sqf = count_polys(g, q, kind, degree, first, count, **kw)
    return histogram(counts, sqf)


def cpu_count(g: int, q: int, kind: int, degree: int, first: int, count: int, *,
              seed: int = 0, sample_count: int = 0, threads: int | None = None):
    """hwc_cpu_count: the oracle's histogram in one call.  Returns (tuples
    int32[n, g] sorted lexicographically, multiplicities uint64[n],
    number of square-free members)."""
    lib = _load()
    if threads is None:
        threads = os.cpu_count() or 1
    n_e, n_sq = ctypes.c_uint64(), ctypes.c_uint64()
    P64 = ctypes.POINTER(ctypes.c_uint64)
    # distinct tuples: at most the members, and at most the Hasse-Weil box
    # |q^k + 1 - #C_k| <= 2 g q^(k/2) of square-free members
    box = 1
    for k in range(1, g + 1):
        box *= 2 * math.isqrt(4 * g * g * q ** k) + 1
    cap = max(1, min(count, box))
    counts = np.zeros((cap, g), np.int32)
    mult = np.zeros(cap, np.uint64)
    rc = lib.hwc_cpu_count(g, q, kind, degree, seed, sample_count, first, count, threads, cap,
                           _p32(counts), mult.ctypes.data_as(P64), ctypes.byref(n_e), ctypes.byref(n_sq))
    if rc != 0:
        raise ValueError(f"hwc_cpu_count failed rc={rc}")
    n = n_e.value
    return counts[:n].copy(), mult[:n].copy(), n_sq.value
