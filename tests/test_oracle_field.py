"""Pins of the oracle's field arithmetic (Sec. 2.2) against mathematics.

Each check would fail for a plausible slip in the polynomial-basis code: a
wrong reduction sign or index breaks the field axioms or the cyclicity of
F_Q^x; a wrong square bitmap disagrees with Euler's criterion.
"""
import random

import pytest


@pytest.mark.parametrize("q", [3, 5, 7, 9, 25, 27, 49, 121, 125])
def test_fq_is_a_field(orc, q):
    F = orc.Field(q, 1)
    rnd = random.Random(q)
    for _ in range(400):
        a, b, c = (rnd.randrange(q) for _ in range(3))
        assert F.fq_add(a, b) == F.fq_add(b, a)
        assert F.fq_mul(a, b) == F.fq_mul(b, a)
        assert F.fq_mul(a, F.fq_mul(b, c)) == F.fq_mul(F.fq_mul(a, b), c)
        assert F.fq_mul(a, F.fq_add(b, c)) == F.fq_add(F.fq_mul(a, b), F.fq_mul(a, c))
    for a in range(q):
        assert F.fq_add(a, 0) == a and F.fq_mul(a, 1) == a
        if a:
            assert any(F.fq_mul(a, b) == 1 for b in range(q))
    # characteristic p: adding 1 to itself p times gives 0
    acc = 0
    for _ in range(F.p):
        acc = F.fq_add(acc, 1)
    assert acc == 0


def test_digit_moduli_match_hand_derivation(orc):
    # First monic irreducible by index sum m_i p^i, derived by hand:
    # q=9:  T^2+1   (-1 is not a square mod 3)
    # q=25: T^2+2   (T^2+1 splits since -1 = 2^2 mod 5; -2 = 3 is a non-square)
    # q=27: T^3+2T+1 (candidates of index 1,2,4,5 have a root in F_3)
    # q=49: T^2+1   (-1 = 6 is a non-square mod 7)
    assert orc.Field(9).m == [1, 0, 1]
    assert orc.Field(25).m == [2, 0, 1]
    assert orc.Field(27).m == [1, 2, 0, 1]
    assert orc.Field(49).m == [1, 0, 1]
    assert orc.Field(31).m == [0, 1]


def _order(F, y):
    n, acc = 1, y
    while acc != 1:
        acc = F.mul(acc, y)
        n += 1
    return n


@pytest.mark.parametrize("q,k", [(3, 2), (3, 4), (5, 2), (9, 2), (7, 3), (25, 2), (27, 2), (13, 2)])
def test_fQ_multiplicative_group_is_cyclic(orc, q, k):
    F = orc.Field(q, k)
    Q = F.Q
    # some element has order exactly Q-1, so F_Q^x is cyclic of order Q-1
    assert any(_order(F, y) == Q - 1 for y in range(2, min(Q, 60)))
    # Frobenius fixes F_Q: y^Q = y for all y (spot check)
    rnd = random.Random(Q)
    for y in [rnd.randrange(Q) for _ in range(40)]:
        acc = 1
        for _ in range(Q):
            acc = F.mul(acc, y)
        assert acc == y


@pytest.mark.parametrize("q,k", [(3, 1), (3, 2), (5, 2), (9, 2), (27, 2), (31, 2), (13, 3), (7, 4)])
def test_chi_bitmap_equals_euler_criterion(orc, q, k):
    F = orc.Field(q, k)
    Q = F.Q
    step = max(1, Q // 3000)
    for y in range(0, Q, step):
        assert F.chi(y) == F.chi_euler(y)
    # exactly (Q-1)/2 nonzero squares
    assert sum(1 for y in range(1, Q) if F.chi(y) == 1) == (Q - 1) // 2


@pytest.mark.parametrize("q,k", [(3, 2), (9, 2), (5, 3), (27, 2)])
def test_subfield_character_is_power(orc, q, k):
    # For c in F_q: chi_{q^k}(c) = chi_q(c)^k (used for the points at infinity)
    Fq, FQ = orc.Field(q, 1), orc.Field(q, k)
    for c in range(1, q):
        assert FQ.chi(c) == Fq.chi(c) ** k


def test_alternative_tower_modulus_is_a_field(orc):
    F = orc.Field(9, 2, h_choice=1)
    assert F.h != orc.Field(9, 2).h
    assert any(_order(F, y) == 80 for y in range(2, 40))
