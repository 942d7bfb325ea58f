"""Tiny finite fields in pure Python, built independently of the oracle.

Used only by the tests to pin the oracle by brute force.  F_{p^n} is built
directly as F_p[X]/M(X) with M the monic irreducible of degree n of LARGEST
index sum_i M_i p^i (the oracle uses a tower with the smallest ones), so the
two share neither code nor basis.  The subfield F_q (q = p^e) is reached
through a root theta of the digit-convention modulus m (first monic
irreducible of degree e over F_p by index), found here by search.
"""
from __future__ import annotations

import itertools


def _poly_divides(a, b, p):
    """True iff monic b divides a over F_p (lists, low degree first)."""
    a = list(a)
    db = len(b) - 1
    for t in range(len(a) - 1, db - 1, -1):
        c = a[t] % p
        if c:
            for i in range(db + 1):
                a[t - db + i] = (a[t - db + i] - c * b[i]) % p
    return all(v % p == 0 for v in a[:db])


def irreducible_over_fp(a, p):
    n = len(a) - 1
    for t in range(1, n // 2 + 1):
        for low in itertools.product(range(p), repeat=t):
            if _poly_divides(a, list(low) + [1], p):
                return False
    return True


def prime_power(q):
    for p in range(2, q + 1):
        if q % p == 0:
            e, x = 0, q
            while x % p == 0:
                x //= p
                e += 1
            if x != 1:
                raise ValueError("not a prime power")
            return p, e
    raise ValueError(q)


def digit_modulus(p, e):
    """First monic irreducible of degree e over F_p in index order (the
    digit convention of the library and the oracle)."""
    for idx in range(p ** e):
        low = [(idx // p ** i) % p for i in range(e)]
        if irreducible_over_fp(low + [1], p):
            return low + [1]
    raise AssertionError


class GF:
    """F_{p^n} = F_p[X]/M, elements are ints sum a_i p^i."""

    def __init__(self, p, n):
        self.p, self.n, self.size = p, n, p ** n
        M = None
        for idx in range(p ** n - 1, -1, -1):
            low = [(idx // p ** i) % p for i in range(n)]
            if low[0] and irreducible_over_fp(low + [1], p):
                M = low + [1]
                break
        self.M = M
        N = self.size
        self._add = [[self._add_def(a, b) for b in range(N)] for a in range(N)]
        self._mul = [[self._mul_def(a, b) for b in range(N)] for a in range(N)]

    def _dig(self, a):
        return [(a // self.p ** i) % self.p for i in range(self.n)]

    def _val(self, d):
        return sum(v * self.p ** i for i, v in enumerate(d))

    def _add_def(self, a, b):
        return self._val([(x + y) % self.p for x, y in zip(self._dig(a), self._dig(b))])

    def _mul_def(self, a, b):
        p, n = self.p, self.n
        da, db = self._dig(a), self._dig(b)
        r = [0] * (2 * n)
        for i in range(n):
            for j in range(n):
                r[i + j] = (r[i + j] + da[i] * db[j]) % p
        for t in range(2 * n - 2, n - 1, -1):
            c = r[t]
            if c:
                r[t] = 0
                for i in range(n):
                    r[t - n + i] = (r[t - n + i] - c * self.M[i]) % p
        return self._val(r[:n])

    def add(self, a, b):
        return self._add[a][b]

    def mul(self, a, b):
        return self._mul[a][b]

    def pow(self, a, e):
        r = 1
        for _ in range(e):
            r = self.mul(r, a)
        return r

    def subfield_embedding(self, q):
        """Map from the canonical digit c of F_q (c = sum b_i p^i <-> sum b_i T^i,
        T a root of the digit-convention modulus) into this field."""
        p, e = prime_power(q)
        assert p == self.p and self.n % e == 0
        m = digit_modulus(p, e)
        theta = None
        for t in range(self.size):
            acc = 0
            for coef in reversed(m):     # Horner for m(t)
                acc = self.add(self.mul(acc, t), coef)
            if acc == 0:
                theta = t
                break
        assert theta is not None
        powers = [1]
        for _ in range(e - 1):
            powers.append(self.mul(powers[-1], theta))
        emb = []
        for c in range(q):
            b = [(c // p ** i) % p for i in range(e)]
            v = 0
            for bi, th in zip(b, powers):
                for _ in range(bi):
                    v = self.add(v, th)
            emb.append(v)
        return emb


def brute_force_count(F: GF, emb, coeffs, g):
    """#C_f(F) by counting pairs (x, y) with y^2 = f(x), plus the points at
    infinity: 1 when deg f = 2g+1, and the number of square roots of the lead
    coefficient in F when deg f = 2g+2 (textbook smooth model)."""
    d = len(coeffs) - 1
    c = [emb[v] for v in coeffs]
    sq_count = [0] * F.size
    for y in range(F.size):
        sq_count[F.mul(y, y)] += 1
    total = 0
    for x in range(F.size):
        acc = 0
        for coef in reversed(c):
            acc = F.add(F.mul(acc, x), coef)
        total += sq_count[acc]
    if d == 2 * g + 2:
        total += sq_count[c[d]]
    else:
        total += 1
    return total


def squarefree_by_square_divisors(q, coeffs):
    """f is NOT square-free iff u^2 | f for some monic u of degree 1..d/2
    (second method, no derivative), over F_q built as F_p[T]/m."""
    p, e = prime_power(q)
    Fq = GF.__new__(GF)
    Fq.p, Fq.n, Fq.size = p, e, q
    Fq.M = digit_modulus(p, e)
    Fq._add = [[Fq._add_def(a, b) for b in range(q)] for a in range(q)]
    Fq._mul = [[Fq._mul_def(a, b) for b in range(q)] for a in range(q)]
    neg = [next(b for b in range(q) if Fq.add(a, b) == 0) for a in range(q)]
    inv = [None] + [next(b for b in range(q) if Fq.mul(a, b) == 1) for a in range(1, q)]

    def pmul(a, b):
        r = [0] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            for j, y in enumerate(b):
                r[i + j] = Fq.add(r[i + j], Fq.mul(x, y))
        return r

    def divides(b, a):
        a = list(a)
        db = len(b) - 1
        il = inv[b[-1]]
        for t in range(len(a) - 1, db - 1, -1):
            cf = Fq.mul(a[t], il)
            if cf:
                for i in range(db + 1):
                    a[t - db + i] = Fq.add(a[t - db + i], neg[Fq.mul(cf, b[i])])
        return all(v == 0 for v in a[:db])

    d = len(coeffs) - 1
    for t in range(1, d // 2 + 1):
        for low in itertools.product(range(q), repeat=t):
            u = list(low) + [1]
            if divides(pmul(u, u), coeffs):
                return False
    return True
