"""hwc_cpu_count, the oracle's histogram in one C call, against the per-member
oracle counts reduced in numpy (which the other oracle tests pin)."""
import numpy as np
import pytest


@pytest.mark.parametrize("g,q,kind,d,first,count", [
    (2, 3, 0, 5, 0, 486), (2, 3, 0, 6, 0, 1458), (2, 9, 1, 5, 100, 5000), (2, 31, 1, 6, 31 ** 4, 7000),
    (3, 5, 1, 7, 123, 3000), (1, 13, 0, 3, 0, 12 * 13 ** 3), (2, 7, 1, 5, 0, 0),
])
def test_cpu_count_equals_per_member_reduction(orc, g, q, kind, d, first, count):
    t, m, nsq = orc.cpu_count(g, q, kind, d, first, count)
    counts, sqf = orc.count_polys(g, q, kind, d, first, count)
    t2, m2 = orc.histogram(counts, sqf)
    np.testing.assert_array_equal(t, t2)
    np.testing.assert_array_equal(m, m2)
    assert nsq == int(sqf.sum()) == int(m.sum())


def test_cpu_count_across_slices(orc):
    """More members than one internal slice (2^20): slice histograms merge."""
    g, q, kind, d = 1, 19, 0, 4
    count = (1 << 20) + 54321
    t, m, nsq = orc.cpu_count(g, q, kind, d, 7, count)
    counts, sqf = orc.count_polys(g, q, kind, d, 7, count)
    t2, m2 = orc.histogram(counts, sqf)
    np.testing.assert_array_equal(t, t2)
    np.testing.assert_array_equal(m, m2)
    assert nsq == int(sqf.sum())


def test_cpu_count_sampled_family(orc):
    t, m, nsq = orc.cpu_count(2, 293, 2, 5, 0, 40, seed=7, sample_count=1 << 24)
    counts, sqf = orc.count_polys(2, 293, 2, 5, 0, 40, seed=7, sample_count=1 << 24)
    t2, m2 = orc.histogram(counts, sqf)
    np.testing.assert_array_equal(t, t2)
    np.testing.assert_array_equal(m, m2)


def test_cpu_count_rejects_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.cpu_count(2, 6, 1, 5, 0, 10)            # q not a prime power
    with pytest.raises(ValueError):
        orc.cpu_count(2, 5, 1, 5, 0, 5 ** 4 + 1)    # beyond the family
