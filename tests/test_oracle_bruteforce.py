"""Oracle pinned to brute force on tiny fields (pairs (x, y) with y^2 = f(x)).

The brute force lives in tests/pyfield.py: another field construction
(F_p[X]/M of degree e*k directly, largest-index modulus), no quadratic
character, and points at infinity counted as square roots of the lead.
"""
import random

import numpy as np
import pytest

from pyfield import GF, brute_force_count, prime_power, squarefree_by_square_divisors


def _bf_counts(q, g, coeffs_list):
    p, e = prime_power(q)
    fields = []
    for k in range(1, g + 1):
        F = GF(p, e * k)
        fields.append((F, F.subfield_embedding(q)))
    return np.array([[brute_force_count(F, emb, c, g) for (F, emb) in fields]
                     for c in coeffs_list], dtype=np.int32)


def test_config1_full_bruteforce(orc):
    """g=2, q=3, every f of exact degree 5 and 6, counts over F_3 and F_9."""
    for d in (5, 6):
        n = orc.family_size(3, orc.ALL, d)
        counts, sqf = orc.count_polys(2, 3, orc.ALL, d, 0, n, filter=False)
        coeffs = [orc.decode(3, orc.ALL, d, i) for i in range(n)]
        bf = _bf_counts(3, 2, coeffs)
        np.testing.assert_array_equal(counts, bf)


@pytest.mark.parametrize("q,g,kind,d,n", [
    (5, 2, 1, 5, 60), (5, 2, 1, 6, 60), (7, 2, 0, 5, 40), (9, 2, 1, 5, 24),
    (9, 2, 0, 6, 16), (3, 3, 1, 7, 50), (3, 3, 1, 8, 40), (5, 3, 1, 7, 8), (3, 4, 1, 9, 10),
])
def test_random_slices_bruteforce(orc, q, g, kind, d, n):
    size = orc.family_size(q, kind, d)
    rnd = random.Random(q * 1000 + d)
    idx = sorted(rnd.sample(range(size), min(n, size)))
    coeffs = [orc.decode(q, kind, d, i) for i in idx]
    bf = _bf_counts(q, g, coeffs)
    for row, i in zip(bf, idx):
        counts, _ = orc.count_polys(g, q, kind, d, i, 1, filter=False)
        np.testing.assert_array_equal(counts[0], row)


@pytest.mark.parametrize("q,d", [(5, 3), (5, 4), (7, 3), (9, 3)])
def test_genus_one_bruteforce(orc, q, d):
    """g = 1 (elliptic, degree 3 or 4), every member of the ALL family."""
    n = orc.family_size(q, orc.ALL, d)
    rnd = random.Random(d)
    idx = sorted(rnd.sample(range(n), min(n, 150)))
    coeffs = [orc.decode(q, orc.ALL, d, i) for i in idx]
    bf = _bf_counts(q, 1, coeffs)
    got = np.concatenate([orc.count_polys(1, q, orc.ALL, d, i, 1, filter=False)[0] for i in idx])
    np.testing.assert_array_equal(got, bf)


def test_textbook_elliptic_curve(orc):
    # y^2 = x^3 + x + 1 over F_5 has 9 points (affine 8 + infinity); hand count:
    # x=0,2,3,4 give nonzero squares (2 points each), x=1 gives 3, a non-square.
    idx = 1 + 5 * 1  # c0=1, c1=1, c2=0, lead 1
    assert orc.decode(5, orc.ALL, 3, idx) == [1, 1, 0, 1]
    counts, sqf = orc.count_polys(1, 5, orc.ALL, 3, idx, 1)
    assert counts[0, 0] == 9 and sqf[0] == 1


@pytest.mark.parametrize("q,kind,d", [(3, 0, 5), (3, 0, 6), (5, 1, 5), (3, 1, 6), (9, 1, 6), (5, 1, 10), (3, 1, 9)])
def test_squarefree_second_method(orc, q, kind, d):
    """gcd(f, f') test against 'no u^2 divides f' on tiny fields, including
    p | d families (q=3, d=6, 9; q=5, d=10) where f' can vanish."""
    F = orc.Field(q, 1)
    n = orc.family_size(q, kind, d)
    rnd = random.Random(q + d)
    idx = sorted(rnd.sample(range(n), min(n, 120)))
    for i in idx:
        c = orc.decode(q, kind, d, i)
        assert F.squarefree(c) == squarefree_by_square_divisors(q, c), (q, d, c)
