"""The oracle's factorisation pattern lambda(f) (Sec. 1.1, eq. 1.2: the
degrees of the irreducible factors of f, with an extra part 1 for odd degree)
against two other methods:
  - trial division by every monic irreducible polynomial of degree <= d/2,
    in a polynomial arithmetic written here on the oracle's F_q tables;
  - roots: a square-free f has exactly m * n_m roots of exact degree m over
    F_q (one orbit of m conjugates per irreducible factor of degree m), so the
    oracle's F_{q^m} gives n_m for m <= g by counting zeros of f."""
import itertools
import random

import pytest


def _poly_divmod(F, a, b):
    """(quotient, remainder) of a by monic b over F_q (coefficient lists, low first)."""
    a = list(a)
    db = len(b) - 1
    quo = [0] * max(1, len(a) - db)
    for t in range(len(a) - 1, db - 1, -1):
        c = a[t]
        if c == 0:
            continue
        quo[t - db] = c
        for i in range(db + 1):
            a[t - db + i] = F.fq_add(a[t - db + i], F.fq_mul(_neg(F, c), b[i]))
    return quo, a[:db]


def _neg(F, c):
    for x in range(F.q):
        if F.fq_add(c, x) == 0:
            return x
    raise AssertionError


def _monic_irreducibles(F, deg):
    """Every monic irreducible of degree deg over F_q, by trial division by the
    monic polynomials of lower positive degree."""
    q = F.q
    out = []
    lower = [list(t) + [1] for e in range(1, deg // 2 + 1) for t in itertools.product(range(q), repeat=e)]
    for t in itertools.product(range(q), repeat=deg):
        cand = list(t) + [1]
        if all(any(_poly_divmod(F, cand, b)[1]) for b in lower):
            out.append(cand)
    return out


def _pattern_by_division(F, c):
    d = len(c) - 1
    n = [0] * (d + 1)
    rest = list(c)
    for deg in range(1, d // 2 + 1):
        for b in _monic_irreducibles(F, deg):
            quo, rem = _poly_divmod(F, rest, b)
            if not any(rem):
                n[deg] += 1
                rest = quo
    while len(rest) > 1 and rest[-1] == 0:
        rest.pop()
    if len(rest) - 1 >= 1:
        n[len(rest) - 1] += 1
    return n


@pytest.mark.parametrize("q,d", [(3, 5), (3, 6), (3, 8), (5, 5), (5, 6), (7, 6), (9, 6)])
def test_factor_degrees_against_trial_division(orc, q, d):
    F = orc.Field(q, 1)
    rnd = random.Random(q * 31 + d)
    seen = 0
    for _ in range(400):
        c = [rnd.randrange(q) for _ in range(d)] + [rnd.randrange(1, q)]
        if not F.squarefree(c):
            continue
        got = F.factor_degrees(c)
        # trial division needs a monic polynomial: divide by the lead
        lead = c[-1]
        inv = next(x for x in range(1, q) if F.fq_mul(lead, x) == 1)
        monic = [F.fq_mul(v, inv) for v in c]
        assert got == _pattern_by_division(F, monic), (q, c)
        assert sum(m * k for m, k in enumerate(got)) == d
        seen += 1
    assert seen > 50


@pytest.mark.parametrize("q,g", [(3, 4), (5, 3), (7, 2), (9, 2)])
def test_factor_degrees_against_root_counts(orc, q, g):
    """n_m for m <= g from the zeros of f of exact degree m in the oracle's F_{q^m}."""
    fields = {m: orc.Field(q, m) for m in range(1, g + 1)}
    rnd = random.Random(q * 7 + g)
    for d in (2 * g + 1, 2 * g + 2):
        done = 0
        while done < 25:
            c = [rnd.randrange(q) for _ in range(d)] + [rnd.randrange(1, q)]
            if not fields[1].squarefree(c):
                continue
            n = fields[1].factor_degrees(c)
            roots = {m: [x for x in range(q ** m) if fields[m].eval(c, x) == 0] for m in fields}
            for m in fields:   # roots in F_{q^m} = sum over e | m of e * n_e
                assert len(roots[m]) == sum(e * n[e] for e in range(1, m + 1) if m % e == 0), (c, m)
            done += 1


def _n_irreducible(q, m):
    """Monic irreducible polynomials of degree m over F_q (Gauss)."""
    def mu(n):
        r, k, p = 1, n, 2
        while p * p <= k:
            if k % p == 0:
                k //= p
                if k % p == 0:
                    return 0
                r = -r
            p += 1
        return -r if k > 1 else r
    return sum(mu(m // e) * q ** e for e in range(1, m + 1) if m % e == 0) // m


@pytest.mark.parametrize("q,g", [(3, 1), (3, 2), (5, 1), (5, 2), (7, 1), (9, 1)])
def test_lambda_counts_over_whole_family_closed_form(orc, q, g):
    """Over every f of exact degree d (any lead), the square-free f with n_m
    irreducible factors of degree m number (q - 1) prod_m binom(N_m, n_m),
    N_m the monic irreducibles of degree m: a factorisation picks distinct
    monic irreducibles and a lead."""
    from math import comb
    for d in (2 * g + 1, 2 * g + 2):
        size = orc.family_size(q, 0, d)
        codes = orc.lambda_codes(g, q, 0, d, 0, size)
        got = {}
        for v in codes.tolist():
            if v:
                got[v] = got.get(v, 0) + 1
        want = {}

        def parts(rest, mmax, acc):
            if rest == 0:
                yield dict(acc)
                return
            for m in range(min(rest, mmax), 0, -1):
                for k in range(1, rest // m + 1):
                    acc[m] = k
                    yield from parts(rest - m * k, m - 1, acc)
                    del acc[m]

        for n in parts(d, d, {}):
            ways = (q - 1)
            for m, k in n.items():
                ways *= comb(_n_irreducible(q, m), k)
            if ways:
                nn = dict(n)
                if d == 2 * g + 1:
                    nn[1] = nn.get(1, 0) + 1
                code = sum(k << (4 * (m - 1)) for m, k in nn.items())
                want[code] = ways
        assert got == want, (q, g, d)
