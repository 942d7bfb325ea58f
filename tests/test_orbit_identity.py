"""The Frobenius-orbit form of the character sums, pinned on the oracle's
own field arithmetic (polynomial basis, no Zech tables).

For f with coefficients in F_q and x in F_{q^k}, f(x^q) = f(x)^q, so chi(f(x))
is constant on the orbit {x, x^q, x^(q^2), ...} of x.  An x of exact degree m
over F_q (m | k) has an orbit of m elements, all in F_{q^m}, and for y in
F_{q^m} chi_{q^k}(y) = chi_{q^m}(y)^(k/m).  Hence, with R_m one representative
of each orbit of elements of exact degree m (x = 0 counted in R_1),
    E_m = sum_{x in R_m} chi_{q^m}(f(x)),   Z_m = #{x in R_m : f(x) = 0},
    S_k = sum_{x in F_{q^k}} chi_{q^k}(f(x))
        = sum_{m | k} m * (E_m if k/m is odd else |R_m| - Z_m).
This is the sum the count kernels evaluate (one point per orbit); here it is
computed from the oracle's F_{q^m} and compared with the oracle's own point
counts #C_k = q^k + S_k + (points at infinity)."""
import random

import pytest


def _pow(F, x, e):
    r, b = 1, x
    while e:
        if e & 1:
            r = F.mul(r, b)
        b = F.mul(b, b)
        e >>= 1
    return r


def _reps(F, q, m):
    """One element per Frobenius orbit of the elements of F_{q^m} of exact
    degree m (for m = 1: every element, 0 included)."""
    Q = q ** m
    seen = set()
    out = []
    for x in range(Q):
        if x in seen:
            continue
        orbit = [x]
        y = _pow(F, x, q)
        while y != x:
            orbit.append(y)
            y = _pow(F, y, q)
        seen.update(orbit)
        if len(orbit) == m:
            out.append(x)
    return out


def _mobius(n):
    r, k, p = 1, n, 2
    while p * p <= k:
        if k % p == 0:
            k //= p
            if k % p == 0:
                return 0
            r = -r
        p += 1
    return -r if k > 1 else r


@pytest.mark.parametrize("q,g", [(3, 4), (5, 3), (5, 4), (7, 3), (9, 2), (9, 3)])
def test_orbit_sums_reproduce_oracle_counts(orc, q, g):
    fields = {m: orc.Field(q, m) for m in range(1, g + 1)}
    reps = {m: _reps(fields[m], q, m) for m in range(1, g + 1)}
    # |R_m| is the number of monic irreducibles of degree m (Gauss; x - 0 among them for m = 1)
    for m in range(1, g + 1):
        n_irr = sum(_mobius(m // d) * q ** d for d in range(1, m + 1) if m % d == 0) // m
        assert len(reps[m]) == n_irr
    rnd = random.Random(q * 100 + g)
    for kind, d in [(1, 2 * g + 1), (0, 2 * g + 2), (0, 2 * g + 1)]:
        size = orc.family_size(q, kind, d)
        for idx in rnd.sample(range(size), 6):
            c = orc.decode(q, kind, d, idx)
            counts, sqf = orc.count_polys(g, q, kind, d, idx, 1, filter=False, threads=1)
            E, Z = {}, {}
            for m in range(1, g + 1):
                F = fields[m]
                vals = [F.eval(c, x) for x in reps[m]]
                E[m] = sum(F.chi(v) for v in vals)
                Z[m] = sum(1 for v in vals if v == 0)
            for k in range(1, g + 1):
                S = sum(m * (E[m] if (k // m) % 2 else len(reps[m]) - Z[m])
                        for m in range(1, k + 1) if k % m == 0)
                Fk = fields[k]
                inf = 1 + (Fk.chi(c[d]) if d == 2 * g + 2 else 0)
                assert q ** k + S + inf == int(counts[0, k - 1]), (q, g, kind, d, idx, k)
