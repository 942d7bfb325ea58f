"""N_{g,q} of eq. 1.2 from the reduced families P'_d (HWC_FAM_REDUCED, Sec.
1.2-1.3) on the GPU: each member weighted by mult(f) and counted also for its
quadratic twist.  The histogram must equal the oracle's N_{g,q} over every
square-free f of degree d (the definition), with and without the
factorisation patterns; per-member counts equal the oracle's on the same
reduced polynomials."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

CASES = [(2, 3, 5), (2, 5, 6), (2, 7, 5), (2, 7, 6), (2, 9, 5), (3, 3, 7), (3, 5, 7), (3, 5, 8),
         (4, 3, 10)]


def _ids(c):
    return "g%dq%dd%d" % c


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_reduced_members_match_oracle(orc, case):
    g, q, d = case
    coeffs, mult = orc.reduced_family(q, d)
    oc, os_, _ = orc.count_list(g, q, coeffs)
    fam = hwc.make_family(hwc.FAM_REDUCED, d)
    assert hwc.family_size(q, fam) == len(coeffs)
    gc, gs = hwc.count_members(g, q, fam, 0, len(coeffs))
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gc, oc)


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_reduced_histogram_is_n_gq(orc, case):
    g, q, d = case
    want = orc.n_gq(g, q, d, reduced=False)   # every square-free f of degree d
    fam = hwc.make_family(hwc.FAM_REDUCED, d)
    n = hwc.family_size(q, fam)
    h = hwc.count(g, q, fam, 0, n, hwc.FLAG_LAMBDA)
    got = {}
    for row, code, m in zip(h.counts, h.lam, h.mult):
        key = (int(code),) + tuple(q ** (k + 1) + 1 - int(row[k]) for k in range(g))
        got[key] = got.get(key, 0) + int(m)
    assert got == want
    assert h.n_squarefree == sum(want.values())
    # without the patterns: the plain histogram of every f of degree d
    plain = hwc.count(g, q, fam, 0, n)
    full = hwc.count(g, q, hwc.make_family(hwc.FAM_ALL_DEG, d), 0, (q - 1) * q ** d)
    np.testing.assert_array_equal(plain.counts, full.counts)
    np.testing.assert_array_equal(plain.mult, full.mult)


def test_reduced_family_refuses_p_dividing_d():
    with pytest.raises(hwc.HwcError) as e:
        hwc.family_size(3, hwc.make_family(hwc.FAM_REDUCED, 6))
    assert e.value.code == hwc.ERR_ARG
