"""Genus 4 over F_13 on the two-level kernel.  The fan-out rows of F_{13^4}
(28,561 elements) take 114 KB as u32 words, which with the doubled Zech table
leaves no room for the kernel's warps; the layout then stages the rows of the
orbit-point fields as int16 (13 digit bits and the flag in bit 15, sign
extended on the read).  Checked against the oracle member by member on ragged
slices from the middle of the degree-9 and degree-10 families, as a histogram
on a larger slice, and, for a densely drawn sample (the weighted form of the
kernel over all 13^8 members), against the per-member kernel over the same
draws."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

MZ = hwc.FAM_MONIC_NOSUB
SAMPLED = hwc.FAM_MONIC_NOSUB_SAMPLED
Q = 13


@pytest.mark.parametrize("d", [9, 10])
def test_members_match_oracle(orc, d):
    n_fam = Q ** (d - 1)
    first = n_fam // 2 + 17          # not on a group boundary (groups of 169)
    n = 169 * 6 + 50                 # several groups and a ragged tail
    b = hwc.Batch([hwc.make_job(4, Q, MZ, d, first, n)], hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 2
    b.close()
    fam = hwc.make_family(MZ, d)
    gc, gs = hwc.count_members(4, Q, fam, first, n)
    oc, os_ = orc.count_polys(4, Q, MZ, d, first, n)
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gc, oc)


def test_histogram_matches_oracle(orc):
    first, n = 3 * Q ** 8 // 7 + 5, 12_000
    h = hwc.count(4, Q, hwc.make_family(MZ, 9), first, n, hwc.FLAG_NO_TUNE)
    tup, mult, nsq = orc.cpu_count(4, Q, MZ, 9, first, n)
    np.testing.assert_array_equal(h.counts, tup)
    np.testing.assert_array_equal(h.mult, mult)
    assert (h.n_squarefree, h.n_total) == (nsq, n)


def test_weighted_sample_matches_per_member():
    sc = 1 << 26                     # the genus-4 serving workload's q = 13 draws
    first, n = 12_345, (1 << 25) + 6789   # one sample per 24 members: dense
    assert n * 32 >= Q ** 8
    job = hwc.make_job(4, Q, SAMPLED, 9, first, n, 11, sc)
    b = hwc.Batch([job], hwc.FLAG_GRAPH | hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 2
    b.launch()
    got = b.result(0)
    b.close()
    want = hwc.count(4, Q, hwc.make_family(SAMPLED, 9, 11, sc), first, n, hwc.FLAG_HORNER)
    np.testing.assert_array_equal(got.counts, want.counts)
    np.testing.assert_array_equal(got.mult, want.mult)
    assert (got.n_squarefree, got.n_total) == (want.n_squarefree, n)
