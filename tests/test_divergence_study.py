"""Branch divergence of the Zech-logarithm Horner evaluation (Sec. 4, the
discussion after Table 1).  In the log encoding an element of F_Q is either 0
or alpha^l, so a Zech addition a + b needs a special case when an addend is
zero: in Horner's rule s <- s x + c_i that is c_i = 0 or s x = 0.  The paper
assumes each happens with probability 1/q^e and bounds the share of such
additions by 2d/q^e.

Measured here on the oracle's polynomial-basis arithmetic, for members drawn
at random from the benchmark families (monic, c_{d-1} = 0: the additions of
c_{d-2}, ..., c_0) and every x in F_{q^e}^x:
- a zero coefficient occurs in about 1/q of the additions, not 1/q^e, since
  c_i lies in F_q; it is the same for every x of one f, so lanes that share
  f (the paper's work items; the lanes of every kernel here) take the same
  path and do not diverge;
- a vanishing partial sum, the case that does split lanes sharing f, stays
  below the paper's bound: about (number of subfields of F_{q^e})/q^e of
  the additions.
The kernels here keep the common path branch-free (the poison entry of the
Zech table marks a vanishing sum) and send only the rare lanes to a branchy
step."""
import math

import numpy as np
import pytest

import oracle

# (q, e, degree, members): fields of the benchmark configurations
CASES = [
    (31, 2, 6, 60),      # configuration 2: F_{31^2}
    (13, 3, 7, 30),      # configuration 4: F_{13^3}
    (7, 4, 9, 25),       # configuration 5: F_{7^4}
    (293, 2, 5, 2),      # configuration 3: F_{293^2}
]


@pytest.fixture(scope="module")
def orc():
    oracle.build()
    return oracle


def _rates(orc, q, e, d, members, seed=5):
    F = orc.Field(q, e)
    for a in range(q):   # the constant digits of F_q are the elements 0..q-1 of F_{q^e}
        assert F.add(a, 1) == F.fq_add(a, 1)
    rng = np.random.default_rng(seed)
    adds = zero_coef = zero_sum = 0
    for _ in range(members):
        c = [int(v) for v in rng.integers(0, q, size=d - 1)] + [0, 1]   # c_0..c_{d-2}, c_{d-1} = 0, c_d = 1
        for x in range(1, F.Q):
            s = x                               # c_d x + c_{d-1} (= 0: nothing to add)
            for i in range(d - 2, -1, -1):
                s = F.mul(s, x)
                zero_coef += c[i] == 0
                zero_sum += s == 0
                s = F.add(s, c[i])
                adds += 1
    return adds, zero_coef / adds, zero_sum / adds


@pytest.mark.parametrize("case", CASES, ids=lambda c: "q%de%d" % c[:2])
def test_divergent_additions_stay_below_the_papers_bound(orc, case):
    q, e, d, members = case
    adds, r_coef, r_sum = _rates(orc, q, e, d, members)
    Q = q ** e
    # zero coefficients: about 1/q of the additions (binomial over the
    # members' d - 1 coefficients, each counted once per x; five sigma)
    p = 1 / q
    assert abs(r_coef - p) < 5 * math.sqrt(p * (1 - p) / (members * (d - 1)))
    # vanishing partial sums: below the paper's 2d/q^e, and of the order of
    # (subfields of F_{q^e}) / q^e
    subfields = sum(1 for m in range(1, e + 1) if e % m == 0)
    assert r_sum < 2 * d / Q
    assert r_sum < 3 * subfields / Q
