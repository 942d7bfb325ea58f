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
        lib.orc_count_list.restype = i32
        lib.orc_count_list.argtypes = [i32, i32, i32, u64, P32, i32, P32, P8, ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_lambda_codes.restype = i32
        lib.orc_lambda_codes.argtypes = [i32, i32, i32, i32, u64, u64, u64, u64, i32, ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_factor_degrees.restype = i32
        lib.orc_factor_degrees.argtypes = [vp, i32, P32, P32]
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

    def factor_degrees(self, coeffs):
        """n[m] = number of irreducible factors of degree m (m = 0..d) of the
        square-free coeffs (c_0..c_d) over F_q, by distinct-degree
        factorisation; None if not square-free of degree d."""
        c = np.ascontiguousarray(coeffs, dtype=np.int32)
        n = np.zeros(len(c), dtype=np.int32)
        if self._lib.orc_factor_degrees(self._h, len(c) - 1, _p32(c), _p32(n)) != 0:
            return None
        return [int(v) for v in n]


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


def lambda_codes(g: int, q: int, kind: int, degree: int, first: int, count: int, *,
                 seed: int = 0, sample_count: int = 0, threads: int | None = None):
    """lambda(f) of eq. 1.2 per member (uint64 codes sum_m n_m 16^(m-1), n_m the
    parts equal to m of the partition of 2g+2; an extra part 1 for degree
    2g+1; 0 for members that are not square-free)."""
    lib = _load()
    if threads is None:
        threads = os.cpu_count() or 1
    codes = np.zeros(count, dtype=np.uint64)
    rc = lib.orc_lambda_codes(g, q, kind, degree, seed, sample_count, first, count, threads,
                              codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc != 0:
        raise ValueError(f"oracle lambda failed rc={rc}")
    return codes


def lambda_histogram(g: int, q: int, kind: int, degree: int, first: int, count: int, **kw):
    """N_{g,q} of eq. 1.2 restricted to members [first, first+count) of a
    family, weight 1: rows (#C_1..#C_g, lambda code) sorted by lambda code then
    tuple, and their multiplicities."""
    counts, sqf = count_polys(g, q, kind, degree, first, count, **kw)
    codes = lambda_codes(g, q, kind, degree, first, count, seed=kw.get("seed", 0),
                         sample_count=kw.get("sample_count", 0), threads=kw.get("threads"))
    sel = sqf.astype(bool)
    rows = np.concatenate([codes[sel].astype(np.int64)[:, None], counts[sel].astype(np.int64)], axis=1)
    if rows.shape[0] == 0:
        return np.zeros((0, g), np.int32), np.zeros(0, np.uint64), np.zeros(0, np.uint64)
    uniq, mult = np.unique(rows, axis=0, return_counts=True)
    return uniq[:, 1:].astype(np.int32), uniq[:, 0].astype(np.uint64), mult.astype(np.uint64)


def count_list(g: int, q: int, coeffs: np.ndarray, threads: int | None = None):
    """Point counts, square-freeness and lambda codes of explicit polynomials:
    coeffs int32 [n, d+1] (c_0..c_d, digits).  Returns (counts int32 [n, g],
    sqf uint8 [n], codes uint64 [n])."""
    lib = _load()
    if threads is None:
        threads = os.cpu_count() or 1
    c = np.ascontiguousarray(coeffs, dtype=np.int32)
    n, d1 = c.shape
    counts = np.zeros((n, g), np.int32)
    sqf = np.zeros(n, np.uint8)
    codes = np.zeros(n, np.uint64)
    rc = lib.orc_count_list(g, q, d1 - 1, n, _p32(c), threads, _p32(counts),
                            sqf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                            codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc != 0:
        raise ValueError(f"oracle count_list failed rc={rc}")
    return counts, sqf, codes


# ---------------------------------------------------------------------------
# Reduced families (Sec. 1.2-1.3) and N_{g,q} (eq. 1.2)

def _fq(q: int):
    return Field(q, 1)


def generator_digit(q: int) -> int:
    """The smallest F_q digit whose powers give all of F_q^x (oracle arithmetic)."""
    F = _fq(q)
    for w in range(2, q):
        x, order = w, 1
        while x != 1:
            x = F.fq_mul(x, w)
            order += 1
        if order == q - 1:
            return w
    return 1   # q = 3: F_3^x = {1, 2}, generated by 2 (reached above); q = 2 not used


def reduced_patterns(q: int, d: int):
    """The support patterns of P'_d for p not dividing d, in index order:
    ('A',) c_d X^d + 1;  ('B',) c_d X^d + X;  (i, j) for 1 <= i <= d-2,
    0 <= j < i: c_d X^d + X^i + c_j X^j + c_{j-1} X^(j-1) + ... + c_0 with
    c_j in R_{i-j} (the coset representatives w^t, t < gcd(q-1, i-j)).
    Returns [(pattern, members, mult)]: mult = the number of polynomials of
    degree d whose reduction has the member's pattern, over the members of the
    pattern counted with their twists: q translations times the free nonzero
    coefficients, so q (q-1)^2 / (2 (q-1)) = q(q-1)/2 for A and B, and
    q (q-1)^3 q^j / (2 (q-1) gcd(q-1, i-j) q^j) = q(q-1)^2 / (2 gcd(q-1, i-j))
    for (i, j).  (The paper lists A and the (i, j) patterns; B, the f whose
    only coefficients are c_d and c_1 after translation, is missing there.)"""
    from math import gcd
    out = [(("A",), q - 1, q * (q - 1) // 2), (("B",), q - 1, q * (q - 1) // 2)]
    for i in range(1, d - 1):
        for j in range(i):
            gg = gcd(q - 1, i - j)
            out.append(((i, j), (q - 1) * gg * q ** j, q * (q - 1) ** 2 // (2 * gg)))
    return out


def reduced_family(q: int, d: int):
    """Every member of P'_d (twist folded: the coefficient after the lead is 1)
    in index order: (coeffs int32 [n, d+1], mult uint64 [n]).  Within a
    pattern, member index = low digits (c_0 + c_1 q + ... + c_{j-1} q^(j-1))
    + q^j (t + gcd (c_d - 1)).  Pure Python: small q only."""
    F = _fq(q)
    w = generator_digit(q)
    pw = [1]
    for _ in range(q):
        pw.append(F.fq_mul(pw[-1], w))
    rows, mult = [], []
    for pat, n, m in reduced_patterns(q, d):
        for idx in range(n):
            c = [0] * (d + 1)
            if pat == ("A",):
                c[d], c[0] = 1 + idx, 1
            elif pat == ("B",):
                c[d], c[1] = 1 + idx, 1
            else:
                i, j = pat
                low = idx % q ** j
                rest = idx // q ** j
                from math import gcd
                gg = gcd(q - 1, i - j)
                t, cd = rest % gg, 1 + rest // gg
                for k in range(j):
                    c[k] = low % q
                    low //= q
                c[d], c[i], c[j] = cd, 1, pw[t]
            rows.append(c)
            mult.append(m)
    return np.asarray(rows, np.int32), np.asarray(mult, np.uint64)


def n_gq(g: int, q: int, d: int, reduced: bool):
    """N_{g,q} of eq. 1.2 restricted to degree d, as {(lambda code, a_1..a_g): count}
    with a_k = q^k + 1 - #C_k (eq. 1.1).
    reduced=False: every square-free f of degree d (the definition).
    reduced=True: the members f of P'_d with weight mult(f), each counted for f
    and for its quadratic twist e f (e a non-square), whose a_k is (-1)^k a_k."""
    qk = np.array([q ** (k + 1) + 1 for k in range(g)], np.int64)
    if reduced:
        coeffs, mult = reduced_family(q, d)
        counts, sqf, codes = count_list(g, q, coeffs)
        sel = sqf.astype(bool)
        a = qk[None, :] - counts[sel].astype(np.int64)
        sign = np.array([-1 if (k + 1) % 2 else 1 for k in range(g)], np.int64)
        rows = np.concatenate([np.concatenate([codes[sel].astype(np.int64)[:, None], a], axis=1),
                               np.concatenate([codes[sel].astype(np.int64)[:, None], a * sign], axis=1)])
        w = np.concatenate([mult[sel], mult[sel]]).astype(np.int64)
    else:
        size = (q - 1) * q ** d
        counts, sqf = count_polys(g, q, ALL, d, 0, size)
        codes = lambda_codes(g, q, ALL, d, 0, size)
        sel = sqf.astype(bool)
        rows = np.concatenate([codes[sel].astype(np.int64)[:, None], qk[None, :] - counts[sel].astype(np.int64)],
                              axis=1)
        w = np.ones(rows.shape[0], np.int64)
    if rows.shape[0] == 0:
        return {}
    uniq, inv = np.unique(rows, axis=0, return_inverse=True)
    tot = np.bincount(inv.reshape(-1), weights=w.astype(np.float64), minlength=len(uniq))
    return {tuple(int(v) for v in r): int(round(t)) for r, t in zip(uniq, tot)}
    size = (q - 1) * q ** d
    counts, sqf = count_polys(g, q, ALL, d, 0, size)
    codes = lambda_codes(g, q, ALL, d, 0, size)
    for row, s, code in zip(counts, sqf, codes):
        if not s:
            continue
        key = (int(code),) + tuple(q ** (k + 1) + 1 - int(row[k]) for k in range(g))
        out[key] = out.get(key, 0) + 1
    return out


def curve_count(q: int, k: int, coeffs) -> np.ndarray:
    """#C(F_{q^k}) of explicit curves y^2 = f(x) (coeffs [n, d+1], digits),
    square-free or not: the count of Sec. 1.1 over every x of F_{q^k}."""
    c = np.ascontiguousarray(np.atleast_2d(coeffs), dtype=np.int32)
    counts, _, _ = count_list_unfiltered(k, q, c)
    return counts[:, k - 1].astype(np.int64)


def count_list_unfiltered(g: int, q: int, coeffs: np.ndarray, threads: int | None = None):
    """count_list with every polynomial evaluated (square-free or not)."""
    lib = _load()
    if threads is None:
        threads = os.cpu_count() or 1
    c = np.ascontiguousarray(coeffs, dtype=np.int32)
    n, d1 = c.shape
    counts = np.zeros((n, g), np.int32)
    sqf = np.zeros(n, np.uint8)
    codes = np.zeros(n, np.uint64)
    rc = lib.orc_count_list(g, q, d1 - 1, n, _p32(c), -threads, _p32(counts),
                            sqf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                            codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc != 0:
        raise ValueError(f"oracle count_list failed rc={rc}")
    return counts, sqf, codes
