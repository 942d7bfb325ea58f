"""Sampled families whose samples share their high digits (c_2..c_{d-2})
often enough run on the class-sharing kernel (classes.cuh, job method 3): the
samples are sorted by class on the device and the members of a class share
the chain for u = sum_{i>=2} c_i x^i.  Histograms against the oracle over the
same samples (several q, degrees 3..6, a prime power, every point and one
point per Frobenius orbit), against the per-member kernel on the 2^24 samples
over F_{293^2} of the mixed-q workload, and over graph replays (the sort runs
again inside the graph)."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

SAMPLED = hwc.FAM_MONIC_NOSUB_SAMPLED

# (g, q, degree, seed, samples, first, count): sparse draws (no whole-family
# kernel) with at least 16 samples per class on average
CASES = [
    (1, 37, 3, 5, 500, 0, 500),               # one class: u = x^3
    (1, 41, 4, 6, 2000, 3, 1990),             # classes c_2
    (2, 37, 5, 7, 30000, 0, 30000),           # classes (c_2, c_3)
    (2, 61, 5, 8, 70000, 1234, 65000),
    (2, 25, 5, 9, 11000, 0, 11000),           # F_25: q <= 31 but fewer than one draw per 32 members
    (2, 37, 6, 10, 820000, 0, 820000),        # classes (c_2, c_3, c_4)
]


def _ids(c):
    return "g%dq%dd%d_n%d" % (c[0], c[1], c[2], c[6])


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_class_kernel_matches_oracle(orc, case):
    g, q, d, seed, sc, first, n = case
    b = hwc.Batch([hwc.make_job(g, q, SAMPLED, d, first, n, seed, sc)], hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 3
    b.launch()
    got = b.result(0)
    b.close()
    tup, mult, nsq = orc.cpu_count(g, q, SAMPLED, d, first, n, seed=seed, sample_count=sc)
    np.testing.assert_array_equal(got.counts, tup)
    np.testing.assert_array_equal(got.mult, mult)
    assert (got.n_squarefree, got.n_total) == (nsq, n)


def test_class_kernel_every_point(orc):
    g, q, d, seed, sc, first, n = CASES[2]
    fam = hwc.make_family(SAMPLED, d, seed, sc)
    got = hwc.count(g, q, fam, first, n, hwc.FLAG_ALL_POINTS | hwc.FLAG_NO_TUNE)
    tup, mult, nsq = orc.cpu_count(g, q, SAMPLED, d, first, n, seed=seed, sample_count=sc)
    np.testing.assert_array_equal(got.counts, tup)
    np.testing.assert_array_equal(got.mult, mult)


def test_q293_samples_match_per_member_kernel():
    g, q, d, seed, sc = 2, 293, 5, 7, 1 << 24   # the mixed-q workload's sampled job
    job = hwc.make_job(g, q, SAMPLED, d, 0, sc, seed, sc)
    b = hwc.Batch([job], hwc.FLAG_GRAPH | hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 3
    outs = []
    for _ in range(2):   # a replay sorts the samples again
        b.launch()
        outs.append(b.result(0))
    b.close()
    want = hwc.count(g, q, hwc.make_family(SAMPLED, d, seed, sc), 0, sc, hwc.FLAG_HORNER)
    for got in outs:
        np.testing.assert_array_equal(got.counts, want.counts)
        np.testing.assert_array_equal(got.mult, want.mult)
        assert (got.n_squarefree, got.n_total) == (want.n_squarefree, sc)


def test_too_few_samples_per_class_stay_per_member():
    b = hwc.Batch([hwc.make_job(2, 61, SAMPLED, 5, 0, 1000, 3, 1 << 20)], hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 0
    b.close()
