"""Windows of a densely drawn sampled family (HWC_FAM_MONIC_NOSUB_SAMPLED_WINDOW):
the draws of samples 0..sample_count-1 whose member index lies in
[first, first + count), counted by the whole-family kernel with their
multiplicities.  Checked against the oracle's counts of the samples that land
in the window (small families), against the whole sampled family when
windows cover it (the genus-4 q = 13 draws of the serving workload), through
the server, and for the refusals."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

SAMPLED = hwc.FAM_MONIC_NOSUB_SAMPLED
WINDOW = hwc.FAM_MONIC_NOSUB_SAMPLED_WINDOW


def _members_drawn(orc, q, d, seed, sc):
    """Member index of every sample, from the oracle's decoding of the sample
    into digits (c_0..c_{d-2}, base q little endian)."""
    out = np.zeros(sc, np.int64)
    for j in range(sc):
        c = orc.decode(q, SAMPLED, d, j, seed)
        out[j] = sum(int(c[i]) * q ** i for i in range(d - 1))
    return out


def _oracle_window(orc, g, q, d, seed, sc, a, b):
    counts, sqf = orc.count_polys(g, q, SAMPLED, d, 0, sc, seed=seed, sample_count=sc)
    idx = _members_drawn(orc, q, d, seed, sc)
    inw = (idx >= a) & (idx < b)
    tup, mult = orc.histogram(counts[inw], sqf[inw])
    return tup, mult, int(sqf[inw].sum()), int(inw.sum())


# (g, q, degree, seed, samples, windows (first, count)): ragged, not on group boundaries
CASES = [
    (2, 5, 5, 7, 3000, [(0, 313), (313, 312), (17, 18)]),
    (2, 13, 5, 11, 20000, [(0, 28561), (5000, 17000), (28000, 561)]),
    (3, 5, 7, 13, 4000, [(100, 9000), (9100, 6525)]),
    (4, 3, 10, 23, 20000, [(11, 19000)]),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "g%dq%dd%d" % c[:3])
def test_window_matches_oracle(orc, case):
    g, q, d, seed, sc, windows = case
    for a, n in windows:
        h = hwc.count(g, q, hwc.make_family(WINDOW, d, seed, sc), a, n, hwc.FLAG_NO_TUNE)
        tup, mult, nsq, ntot = _oracle_window(orc, g, q, d, seed, sc, a, a + n)
        np.testing.assert_array_equal(h.counts, tup)
        np.testing.assert_array_equal(h.mult, mult)
        assert (h.n_squarefree, h.n_total) == (nsq, ntot)


def test_windows_cover_the_sampled_family_g4_q13():
    q, d, seed, sc = 13, 9, 11, 1 << 26      # the genus-4 serving workload's q = 13 draws
    fam = q ** (d - 1)
    cuts = [0, fam // 3 + 5, 2 * fam // 3 - 7, fam]
    acc = None
    for a, b in zip(cuts, cuts[1:]):
        h = hwc.count(4, q, hwc.make_family(WINDOW, d, seed, sc), a, b - a)
        acc = h if acc is None else hwc.hist_merge(acc, h)
    whole = hwc.count(4, q, hwc.make_family(SAMPLED, d, seed, sc), 0, sc)
    np.testing.assert_array_equal(acc.counts, whole.counts)
    np.testing.assert_array_equal(acc.mult, whole.mult)
    assert (acc.n_squarefree, acc.n_total) == (whole.n_squarefree, sc)


def test_window_requests_through_the_server():
    g, q, d, seed, sc = 2, 13, 5, 11, 20000
    fam = q ** (d - 1)
    cuts = [0, 4000, 4001, 15000, fam]
    srv = hwc.Server(device_bytes=2 << 30, max_active=4, step_items=64)
    tickets = [srv.submit(hwc.make_job(g, q, WINDOW, d, a, b - a, seed, sc)) for a, b in zip(cuts, cuts[1:])]
    acc = None
    for t in tickets:
        h = srv.poll(t, timeout_ms=120_000)
        acc = h if acc is None else hwc.hist_merge(acc, h)
    srv.close()
    whole = hwc.count(g, q, hwc.make_family(SAMPLED, d, seed, sc), 0, sc, hwc.FLAG_HORNER)
    np.testing.assert_array_equal(acc.counts, whole.counts)
    np.testing.assert_array_equal(acc.mult, whole.mult)
    assert acc.n_total == sc


@pytest.mark.parametrize("g,q,d,sc,flags", [
    (2, 37, 5, 1 << 20, 0),               # q > 31: no whole-family kernel
    (2, 13, 5, 500, 0),                   # fewer than one draw per 32 members
    (2, 13, 5, 20000, hwc.FLAG_HORNER),   # the per-member kernel asked for
])
def test_window_refusals(g, q, d, sc, flags):
    with pytest.raises(hwc.HwcError) as e:
        hwc.count(g, q, hwc.make_family(WINDOW, d, 3, sc), 0, 100, flags)
    assert e.value.code == hwc.ERR_ARG
    with pytest.raises(hwc.HwcError) as e:
        hwc.count_members(2, 13, hwc.make_family(WINDOW, 5, 3, 20000), 0, 100)
    assert e.value.code == hwc.ERR_ARG
