"""Sampled families drawn densely (at least one sample per 32 members, q <= 31)
run on the two-level kernel over the whole family, each member counted with
its multiplicity among the samples (the samples are drawn with replacement,
hwc.h).  The histogram must equal the oracle's over the decoded samples, the
per-member kernel's (HWC_FLAG_HORNER), and the server's; per-sample counts
(hwc_count_members) stay in sample order."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

SAMPLED = hwc.FAM_MONIC_NOSUB_SAMPLED

# (g, q, degree, seed, sample_count, first, count): dense draws, repeated
# members (q = 3: 81 members, 6000 draws), ragged sub-ranges of the samples
CASES = [
    (1, 5, 3, 3, 400, 0, 400),
    (2, 3, 5, 5, 6000, 0, 6000),
    (2, 5, 5, 7, 3000, 0, 3000),
    (2, 7, 6, 9, 4000, 1234, 2345),
    (2, 13, 5, 11, 20000, 0, 20000),
    (3, 5, 7, 13, 4000, 0, 4000),
    (3, 9, 8, 17, 200000, 777, 150001),
    (4, 3, 9, 19, 5000, 0, 5000),
    (4, 3, 10, 23, 20000, 11, 19000),
]


def _ids(c):
    return "g%dq%dd%d_n%d" % (c[0], c[1], c[2], c[6])


def _same(a, b):
    np.testing.assert_array_equal(a.counts, b.counts)
    np.testing.assert_array_equal(a.mult, b.mult)
    assert a.n_squarefree == b.n_squarefree


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_weighted_matches_oracle_and_per_member(orc, case):
    g, q, d, seed, sc, first, n = case
    fam = hwc.make_family(SAMPLED, d, seed, sc)
    # dense enough for the whole-family kernel
    assert n * 32 >= q ** (d - 1)
    b = hwc.Batch([hwc.make_job(g, q, SAMPLED, d, first, n, seed, sc)], hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 2
    b.launch()
    got = b.result(0)
    b.close()
    tup, mult, nsq = orc.cpu_count(g, q, SAMPLED, d, first, n, seed=seed, sample_count=sc)
    np.testing.assert_array_equal(got.counts, tup)
    np.testing.assert_array_equal(got.mult, mult)
    assert got.n_squarefree == nsq
    assert got.n_total == n   # every sample examined once, repeats included
    per_member = hwc.count(g, q, fam, first, n, hwc.FLAG_HORNER)
    _same(got, per_member)
    _same(hwc.count(g, q, fam, first, n), got)


def test_weighted_under_graph_repeats():
    g, q, d, seed, sc, first, n = CASES[4]
    job = hwc.make_job(g, q, SAMPLED, d, first, n, seed, sc)
    b = hwc.Batch([job], hwc.FLAG_GRAPH | hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 2
    outs = []
    for _ in range(3):   # the multiplicities are cleared and drawn again every run
        b.launch()
        outs.append(b.result(0))
    b.close()
    for h in outs[1:]:
        _same(h, outs[0])
    _same(outs[0], hwc.count(g, q, hwc.make_family(SAMPLED, d, seed, sc), first, n, hwc.FLAG_HORNER))


def test_sparse_draws_stay_per_member():
    # fewer than one sample per 32 members: the per-member kernel over the samples
    b = hwc.Batch([hwc.make_job(2, 13, SAMPLED, 5, 0, 500, 3, 1 << 20)], hwc.FLAG_NO_TUNE)
    assert b.job_method(0) == 0
    b.close()


def test_member_counts_keep_sample_order(orc):
    g, q, d, seed, sc, first, n = CASES[3]
    fam = hwc.make_family(SAMPLED, d, seed, sc)
    gc, gs = hwc.count_members(g, q, fam, first, n)
    oc, os_ = orc.count_polys(g, q, SAMPLED, d, first, n, seed=seed, sample_count=sc)
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gc, oc)


def test_server_weighted_request_equals_batched():
    g, q, d, seed, sc, first, n = CASES[6]
    job = hwc.make_job(g, q, SAMPLED, d, first, n, seed, sc)
    want = hwc.count(g, q, hwc.make_family(SAMPLED, d, seed, sc), first, n)
    srv = hwc.Server(device_bytes=2 << 30, max_active=4, step_items=64)
    t = srv.submit(job)
    h = srv.poll(t, timeout_ms=120_000)
    srv.close()
    _same(h, want)
