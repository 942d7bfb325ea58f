"""Single curves over large fields (hwc_curve_count): the curve of Sec. 4,
Table 1, y^2 = 12x^6 + 13x^5 + 10x^4 + 11x^3 + 16x^2 + 12x + 17, counted over
F_{p^2} for every p of the table (Q up to 9.0e6, Zech tables in L2), and
random curves of every degree over F_{q^k}, against the oracle's count over
every point (polynomial basis, no Zech tables)."""
import random

import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

TABLE1_P = [101, 211, 307, 401, 503, 1009, 1511, 2003, 3001]
TABLE1_CURVE = [17, 12, 16, 11, 10, 13, 12]   # c_0..c_6


@pytest.mark.parametrize("p", TABLE1_P)
def test_table1_curve_over_fp2(orc, p):
    c = np.array([TABLE1_CURVE])
    got, ms = hwc.curve_count(p, 2, c)
    want = orc.curve_count(p, 2, c)
    assert int(got[0]) == int(want[0])
    # Hasse-Weil: |p^2 + 1 - #C| <= 2 g p with g = 2
    assert abs(p * p + 1 - int(got[0])) <= 4 * p
    assert ms > 0


@pytest.mark.parametrize("q,k", [(3, 1), (3, 4), (5, 3), (9, 2), (27, 2), (31, 2), (7, 4), (13, 3), (293, 2)])
def test_random_curves_match_oracle(orc, q, k):
    rnd = random.Random(q * 10 + k)
    for d in range(3, 11):
        rows = []
        for _ in range(5):
            c = [rnd.randrange(q) for _ in range(d)] + [rnd.randrange(1, q)]
            rows.append(c)
        rows.append([0] * d + [1])                      # x^d: a single root of multiplicity d
        rows.append([0, 1] + [0] * (d - 2) + [1])      # x^d + x
        c = np.array(rows)
        got, _ = hwc.curve_count(q, k, c)
        want = orc.curve_count(q, k, c)
        np.testing.assert_array_equal(got, want, err_msg=f"q={q} k={k} d={d}")


def test_curve_limits():
    with pytest.raises(hwc.HwcError) as e:
        hwc.curve_count(4099, 2, np.array([TABLE1_CURVE]))   # 4099^2 > 2^24
    assert e.value.code == hwc.ERR_TOO_LARGE
    with pytest.raises(hwc.HwcError) as e:
        hwc.curve_count(31, 2, np.array([[1, 2, 3, 0]]))     # c_d = 0
    assert e.value.code == hwc.ERR_ARG
