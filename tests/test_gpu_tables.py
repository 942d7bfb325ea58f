"""Device-built Zech tables (Sec. 2.3, eq. 3.1-3.2) checked with independent
polynomial arithmetic over F_p written here."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

CASES = [(3, 1), (3, 2), (5, 2), (9, 2), (27, 1), (27, 2), (31, 2), (25, 3), (27, 3), (13, 4),
         (9, 4), (61, 2), (293, 1), (293, 2)]


def _digits(v, p, n):
    v = np.asarray(v, dtype=np.int64)
    return np.stack([(v // p ** i) % p for i in range(n)], axis=-1)


def _value(d, p):
    n = d.shape[-1]
    return sum(d[..., i].astype(np.int64) * p ** i for i in range(n))


def _mul_by_x(d, M, p):
    n = d.shape[-1]
    top = d[..., n - 1:n]
    out = np.concatenate([np.zeros_like(top), d[..., :n - 1]], axis=-1)
    return (out - top * np.asarray(M[:n], dtype=np.int64)) % p


def _pmulmod(a, b, M, p):
    n = len(M) - 1
    r = [0] * (2 * n)
    for i in range(n):
        for j in range(n):
            r[i + j] = (r[i + j] + a[i] * b[j]) % p
    for t in range(2 * n - 2, n - 1, -1):
        c = r[t]
        if c:
            r[t] = 0
            for i in range(n):
                r[t - n + i] = (r[t - n + i] - c * M[i]) % p
    return r[:n]


@pytest.mark.parametrize("q,k", CASES)
def test_tables(orc, q, k):
    t = hwc.Tables(q, k)
    antilog, log, zech, coef = t.read()
    p, n, Q, L = t.p, t.n, t.Q, t.L
    assert Q == q ** k and L == Q - 1 and p ** n == Q
    # antilog is the walk X^i: starts at 1, each step multiplies by X mod M
    assert antilog[0] == 1
    d = _digits(antilog, p, n)
    nxt = _value(_mul_by_x(d, t.M, p), p)
    np.testing.assert_array_equal(nxt[:-1], antilog[1:])
    assert nxt[-1] == 1
    # ... visiting every nonzero element once: X is primitive, log inverts it
    assert len(np.unique(antilog)) == L and antilog.min() >= 1
    np.testing.assert_array_equal(log[antilog], np.arange(L))
    assert log[0] == L                                  # eq. 3.1: 0 -> q-1
    # Zech: alpha^Z(n) = 1 + alpha^n; Z(L/2) = L (eq. 3.2)
    plus1 = d.copy()
    plus1[:, 0] = (plus1[:, 0] + 1) % p
    plus1v = _value(plus1, p)
    assert zech[L // 2] == L and plus1v[L // 2] == 0
    mask = np.arange(L) != L // 2
    np.testing.assert_array_equal(antilog[zech[mask]], plus1v[mask])
    # symmetry Z(-n) = Z(n) - n (mod L)
    nn = np.arange(1, L)
    nn = nn[nn != L // 2]
    np.testing.assert_array_equal(zech[(L - nn) % L], (zech[nn].astype(np.int64) - nn) % L)
    # digit convention: same modulus as the oracle's F_q
    assert t.mq == orc.Field(q).m
    # coefficient logs: digit c = sum b_i p^i -> sum b_i theta^i, m(theta) = 0
    assert coef[0] == L
    for c in range(1, min(q, p)):
        assert antilog[coef[c]] == c
    e = t.e
    if e > 1:
        theta = [int(v) for v in _digits(antilog[coef[p]], p, n)]
        pw = [[1] + [0] * (n - 1)]
        for _ in range(e):
            pw.append(_pmulmod(pw[-1], theta, t.M, p))
        acc = [0] * n
        for i, mi in enumerate(t.mq):
            acc = [(a + mi * b) % p for a, b in zip(acc, pw[i])]
        assert all(v == 0 for v in acc)
        for c in range(q):
            b = [(c // p ** i) % p for i in range(e)]
            want = [0] * n
            for i in range(e):
                want = [(a + b[i] * x) % p for a, x in zip(want, pw[i])]
            wv = sum(v * p ** i for i, v in enumerate(want))
            got = 0 if coef[c] == L else int(antilog[coef[c]])
            assert got == wv, c
    t.close()


def test_table_errors():
    with pytest.raises(hwc.HwcError) as e:
        hwc.Tables(21, 1)
    assert e.value.code == hwc.ERR_ARG
    with pytest.raises(hwc.HwcError) as e:
        hwc.Tables(31, 4)      # 31^4 > HWC_MAX_Q
    assert e.value.code == hwc.ERR_TOO_LARGE
