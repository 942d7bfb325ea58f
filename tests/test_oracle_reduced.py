"""N_{g,q} of eq. 1.2 through the reduced families (Sec. 1.2-1.3): each
member f of P'_d (the coefficient after the lead set to 1, the quadratic
twist folded in) counted with weight mult(f), once with its own (a_1..a_g)
and once with its twist's, must give exactly the histogram of (a_1..a_g,
lambda) over every square-free f of degree d (the definition, p not
dividing d).  This pins the readings the paper's garbled formulas need:
  - i, j are the two largest indices below d-1 with nonzero coefficients;
  - the pattern c_d X^d + c_1 X (missing in the paper) is added;
  - mult = q(q-1)/2 for c_d X^d + c_0 and c_d X^d + c_1 X, and
    q(q-1)^2 / (2 gcd(q-1, i-j)) for the (i, j) patterns;
  - the twist e f (e a non-square) has a_k(e f) = (-1)^k a_k(f), since
    chi_{q^k}(e) = (-1)^k."""
import itertools
from math import comb

import pytest


@pytest.mark.parametrize("g,q,d", [(2, 3, 5), (2, 5, 6), (2, 7, 5), (2, 7, 6), (3, 3, 7), (2, 9, 5), (3, 5, 7)])
def test_reduced_families_reproduce_the_definition(orc, g, q, d):
    assert orc.n_gq(g, q, d, reduced=True) == orc.n_gq(g, q, d, reduced=False)


def test_reduced_family_sizes(orc):
    from math import gcd
    for q, d in [(3, 5), (5, 6), (7, 5), (9, 7)]:
        pats = orc.reduced_patterns(q, d)
        coeffs, mult = orc.reduced_family(q, d)
        assert len(coeffs) == sum(n for _, n, _ in pats)
        want = 2 * (q - 1) + sum((q - 1) * gcd(q - 1, i - j) * q ** j for i in range(1, d - 1) for j in range(i))
        assert len(coeffs) == want
        # every member is monic-free in the lead, has c_{d-1} = 0 and the next coefficient 1
        for c in coeffs.tolist():
            assert c[d] != 0 and c[d - 1] == 0
            top = max(i for i in range(d - 1) if c[i])
            assert c[top] == 1


@pytest.mark.parametrize("p,d", [(3, 5), (5, 6)])
def test_multiplicities_by_orbit_enumeration(orc, p, d):
    """Brute force over every square-free f of degree d over F_p (p prime):
    the orbits of f -> f(aX + b) / e^2; mult(f) of each reduced member (and
    of its twist) is the size of its orbit over the members in that orbit."""
    F = orc.Field(p, 1)

    def act(c, a, b, e):
        out = [0] * (d + 1)
        for n, cn in enumerate(c):
            if cn:
                for k in range(n + 1):
                    out[k] = (out[k] + cn * comb(n, k) * pow(a, k, p) * pow(b, n - k, p)) % p
        inv = pow(e * e % p, p - 2, p)
        return tuple(v * inv % p for v in out)

    allf = [c for c in itertools.product(range(p), repeat=d + 1) if c[d] and F.squarefree(list(c))]
    orbit_of, sizes = {}, []
    for c in allf:
        if c in orbit_of:
            continue
        orb = {act(c, a, b, e) for a in range(1, p) for b in range(p) for e in range(1, p)}
        for x in orb:
            orbit_of[x] = len(sizes)
        sizes.append(len(orb))
    eps = next(x for x in range(1, p) if pow(x, (p - 1) // 2, p) == p - 1)
    coeffs, mult = orc.reduced_family(p, d)
    members = []
    for c, m in zip(coeffs.tolist(), mult.tolist()):
        for s in (1, eps):
            cc = tuple(v * s % p for v in c)
            if F.squarefree(list(cc)):
                members.append((cc, m))
    per = {}
    for c, _ in members:
        per[orbit_of[c]] = per.get(orbit_of[c], 0) + 1
    assert len(per) == len(sizes)   # every orbit has a reduced member
    for c, m in members:
        o = orbit_of[c]
        assert sizes[o] == m * per[o]
