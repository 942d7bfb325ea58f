"""The fact behind the two-level kernel's direct zero-digit count for g <= 2,
checked in an independently built F_{q^2} (tests/pyfield.py).

Write F_{q^2} = F_q + F_q alpha.  For x outside F_q and any u, the line
{u + b x : b in F_q} meets F_q in exactly one point.  That happens at
b = -u1/x1 (coordinates in the basis {1, alpha}), with c = -(u0 + b x0) the
digit for which u + b x + c = 0.  For x in F_q, u + b x lies in F_q for every b
when u does, and for no b otherwise.  So z(b, c) = #{x != 0 : f_{b,c}(x) = 0}
over F_{q^2} is one event per point outside F_q, plus q events per point of
F_q^x (where u(x) is in F_q).  The tests check that recipe against brute force.
"""
import random

import pytest

from pyfield import GF, prime_power


def _field(q):
    p, e = prime_power(q)
    F = GF(p, 2 * e)
    emb = F.subfield_embedding(q)           # digit -> element of F_{q^2}
    dig = {v: c for c, v in enumerate(emb)}  # element of F_q -> digit
    m1 = _minus_one(F, emb)
    return F, emb, dig, (lambda a: F.mul(a, m1))


def _minus_one(F, emb):
    for v in emb:
        if F.add(v, 1) == 0:
            return v
    raise AssertionError


def _primitive(F, q):
    order = q * q - 1
    for a in range(2, F.size):
        x, k = a, 1
        while x != 1:
            x = F.mul(x, a)
            k += 1
        if k == order:
            return a
    raise AssertionError


def _coords(F, emb, dig, alpha, y):
    """(y0, y1) digits with y = e_y0 + e_y1 alpha, by search."""
    for y1 in range(len(emb)):
        t = F.mul(emb[y1], alpha)
        for y0 in range(len(emb)):
            if F.add(emb[y0], t) == y:
                return y0, y1
    raise AssertionError


@pytest.mark.parametrize("q", [3, 5, 7, 9])
def test_line_meets_fq_once(q):
    F, emb, dig, neg = _field(q)
    alpha = _primitive(F, q)
    fq = set(emb)
    inv = {a: b for a in emb for b in emb if F.mul(a, b) == 1}
    rnd = random.Random(q)
    xs = [x for x in range(1, F.size) if x not in fq]
    for x in rnd.sample(xs, min(len(xs), 12)):
        x0, x1 = _coords(F, emb, dig, alpha, x)
        assert x1 != 0
        for u in range(F.size):
            hits = [b for b in range(q) if F.add(u, F.mul(emb[b], x)) in fq]
            assert len(hits) == 1
            u0, u1 = _coords(F, emb, dig, alpha, u)
            b = dig[neg(F.mul(emb[u1], inv[emb[x1]]))] if u1 else 0
            assert hits == [b]
            y = F.add(u, F.mul(emb[b], x))
            c = dig[neg(F.add(emb[u0], F.mul(emb[b], emb[x0])))]
            assert F.add(y, emb[c]) == 0


@pytest.mark.parametrize("q,d", [(3, 5), (5, 5), (5, 6), (7, 6), (9, 5)])
def test_direct_zero_digit_recipe_equals_brute_force(q, d):
    """z(b, c) for every (c_1, c_0) = (b, c) of one group, two ways."""
    F, emb, dig, neg = _field(q)
    alpha = _primitive(F, q)
    fq = set(emb)
    rnd = random.Random(100 * q + d)
    cu = [0, 0] + [rnd.randrange(q) for _ in range(d - 2)] + [1]   # u = sum_{i>=2} c_i x^i, monic
    cu[d - 1] = 0

    def u_of(x):
        acc = 0
        for coef in reversed(cu):
            acc = F.add(F.mul(acc, x), emb[coef])
        return acc

    brute = {}
    for b in range(q):
        for c in range(q):
            brute[(b, c)] = sum(1 for x in range(1, F.size)
                                if F.add(F.add(u_of(x), F.mul(emb[b], x)), emb[c]) == 0)
    inv = {a: bb for a in emb for bb in emb if F.mul(a, bb) == 1}
    recipe = {(b, c): 0 for b in range(q) for c in range(q)}
    for x in range(1, F.size):
        u = u_of(x)
        if x in fq:                       # every b: c = -(u + b x), u in F_q
            assert u in fq
            for b in range(q):
                recipe[(b, dig[neg(F.add(u, F.mul(emb[b], x)))])] += 1
        else:                             # one b from the coordinates
            x0, x1 = _coords(F, emb, dig, alpha, x)
            u0, u1 = _coords(F, emb, dig, alpha, u)
            b = dig[neg(F.mul(emb[u1], inv[emb[x1]]))]
            c = dig[neg(F.add(emb[u0], F.mul(emb[b], emb[x0])))]
            recipe[(b, c)] += 1
    assert recipe == brute
