"""GPU point counts against the oracle, element by element (bit-exact).

Per-member comparisons span several 32-member tiles and a ragged tail; full
histograms are compared exactly where the oracle finishes in seconds."""
import numpy as np
import pytest

from hwc_helpers import assert_hist_equal, gpu_hist, gpu_members, oracle_hist, oracle_members
from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import ALL_DEG, MONIC_NOSUB, MONIC_NOSUB_SAMPLED, JobSpec, config1

pytestmark = pytest.mark.gpu


def test_config1_full_histograms(orc):
    """g=2, q=3: all 486 + 1458 polynomials of degree 5 and 6 (square-free
    totals 324 and 972)."""
    totals = []
    for spec in config1():
        h = gpu_hist(spec)
        assert_hist_equal(h, oracle_hist(orc, spec))
        assert h.n_total == spec.n()
        totals.append(h.n_squarefree)
    assert totals == [324, 972]


MEMBER_CASES = [
    JobSpec(2, 3, ALL_DEG, 6, 0, 1458),
    JobSpec(2, 31, MONIC_NOSUB, 5, 12345, 32 * 7 + 19),
    JobSpec(2, 31, MONIC_NOSUB, 6, 9_000_001, 32 * 5 + 3),
    JobSpec(2, 27, MONIC_NOSUB, 5, 100, 32 * 6 + 1),
    JobSpec(2, 27, MONIC_NOSUB, 6, 14_000_000, 32 * 4 + 31),
    JobSpec(2, 9, MONIC_NOSUB, 5, 0, 6561),
    JobSpec(2, 25, MONIC_NOSUB, 6, 777, 200),
    JobSpec(2, 5, ALL_DEG, 5, 0, 4 * 5 ** 5),
    JobSpec(2, 61, MONIC_NOSUB, 5, 5_000_000, 100),
    JobSpec(2, 49, MONIC_NOSUB, 5, 0, 97),
    JobSpec(3, 13, MONIC_NOSUB, 7, 1_000_000, 150),
    JobSpec(3, 27, MONIC_NOSUB, 7, 200_000_000, 40),
    JobSpec(3, 5, MONIC_NOSUB, 8, 0, 500),
    JobSpec(4, 7, MONIC_NOSUB, 9, 3_000_000, 70),
    JobSpec(4, 3, MONIC_NOSUB, 10, 0, 3 ** 9),
    JobSpec(1, 7, ALL_DEG, 3, 0, 6 * 7 ** 3),
    JobSpec(1, 9, ALL_DEG, 4, 0, 8 * 9 ** 4),
    JobSpec(4, 13, MONIC_NOSUB_SAMPLED, 9, 0, 24, seed=11, sample_count=1 << 26),
    JobSpec(4, 13, MONIC_NOSUB_SAMPLED, 9, (1 << 26) - 9, 9, seed=11, sample_count=1 << 26),
    JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 40, seed=7, sample_count=1 << 24),
    JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, (1 << 24) - 5, 5, seed=7, sample_count=1 << 24),
]


@pytest.mark.parametrize("spec", MEMBER_CASES, ids=lambda s: f"g{s.g}q{s.q}k{s.kind}d{s.degree}@{s.first}+{s.n()}")
@pytest.mark.parametrize("unfiltered", [False, True])
@pytest.mark.parametrize("kernel", ["auto", "fan1", "horner"])
def test_members_match_oracle(orc, spec, unfiltered, kernel):
    """'auto' takes the two-level fan-out kernel for enumerated families with
    q <= 31, the one-level c_0 fan-out up to q = 63 and the per-member Horner
    kernel otherwise; 'fan1' and 'horner' force the other two."""
    if unfiltered and spec.q > 100:
        pytest.skip("one mode is enough for the slow oracle field")
    enumerated = spec.kind != MONIC_NOSUB_SAMPLED
    if kernel == "horner" and (not enumerated or spec.q > 63):
        pytest.skip("same kernel as 'auto'")
    if kernel == "fan1" and (not enumerated or spec.q > 31):
        pytest.skip("same kernel as 'auto'")
    flags = {"auto": 0, "fan1": hwc.FLAG_FAN1, "horner": hwc.FLAG_HORNER}[kernel]
    gc, gs = gpu_members(spec, unfiltered=unfiltered, flags=flags)
    oc, os_ = oracle_members(orc, spec, filter=not unfiltered)
    np.testing.assert_array_equal(gs, os_)
    np.testing.assert_array_equal(gc, oc)


@pytest.mark.parametrize("spec", [
    JobSpec(2, 27, MONIC_NOSUB, 5), JobSpec(2, 31, MONIC_NOSUB, 5), JobSpec(2, 13, MONIC_NOSUB, 6),
    JobSpec(3, 7, MONIC_NOSUB, 7), JobSpec(2, 9, ALL_DEG, 5), JobSpec(4, 3, MONIC_NOSUB, 9),
    JobSpec(2, 31, MONIC_NOSUB, 6, 20_000_000, 300_001),
], ids=lambda s: f"g{s.g}q{s.q}d{s.degree}@{s.first}")
@pytest.mark.parametrize("flags", [0, hwc.FLAG_FAN1, hwc.FLAG_HORNER], ids=["auto", "fan1", "horner"])
def test_full_histograms_match_oracle(orc, spec, flags):
    h = gpu_hist(spec, flags)
    assert_hist_equal(h, oracle_hist(orc, spec))
    assert h.n_total == spec.n()


def test_empty_range():
    h = gpu_hist(JobSpec(2, 31, MONIC_NOSUB, 5, 100, 0))
    assert h.n_total == 0 and h.n_squarefree == 0 and len(h.mult) == 0


@pytest.mark.parametrize("flags", [0, hwc.FLAG_FAN1, hwc.FLAG_HORNER], ids=["auto", "fan1", "horner"])
def test_edge_ranges(orc, flags):
    """Last member, single members, and ranges that start and end inside a
    group of q members sharing c_1..c_d (partial fan-out groups)."""
    for spec in (JobSpec(2, 31, MONIC_NOSUB, 5, 31 ** 4 - 1, 1), JobSpec(2, 3, ALL_DEG, 5, 0, 1),
                 JobSpec(2, 31, MONIC_NOSUB, 5, 31 * 100 + 7, 31 * 3 + 11),
                 JobSpec(2, 61, MONIC_NOSUB, 5, 61 * 7 + 40, 61 * 2 + 5),
                 JobSpec(2, 37, MONIC_NOSUB, 6, 37 ** 4 + 30, 20),
                 JobSpec(3, 13, MONIC_NOSUB, 7, 13 ** 5 + 12, 2),
                 JobSpec(2, 31, MONIC_NOSUB, 5, 31 * 31 * 5 + 17, 31 * 31 * 2 + 40),
                 JobSpec(2, 3, ALL_DEG, 6, 5, 1000), JobSpec(2, 5, MONIC_NOSUB, 6, 24, 3000)):
        gc, gs = gpu_members(spec, unfiltered=True, flags=flags)
        oc, os_ = oracle_members(orc, spec, filter=False)
        np.testing.assert_array_equal(gc, oc)
        np.testing.assert_array_equal(gs, os_)


@pytest.mark.parametrize("g,q,d", [(2, 5, 5), (2, 3, 6), (3, 3, 7), (2, 7, 6)])
@pytest.mark.parametrize("flags", [0, hwc.FLAG_FAN1, hwc.FLAG_HORNER], ids=["auto", "fan1", "horner"])
def test_character_sum_identity_on_gpu(g, q, d, flags):
    """Unfiltered whole MZ_d family: sum_f sum_x chi(f(x)) = sum over m | k with
    k/m even of N_m q^(d-1-m) (q^m - 1) (N_m = elements of degree exactly m)."""
    from test_oracle_invariants import _mobius
    spec = JobSpec(g, q, MONIC_NOSUB, d)
    counts, _ = gpu_members(spec, unfiltered=True, flags=flags)
    for k in range(1, g + 1):
        Q = q ** k
        inf = 1 if d == 2 * g + 1 else 2
        got = int((counts[:, k - 1].astype(np.int64) - Q - inf).sum())
        want = 0
        for m in range(1, k + 1):
            if k % m or (k // m) % 2:
                continue
            Nm = sum(_mobius(m // j) * q ** j for j in range(1, m + 1) if m % j == 0)
            want += Nm * q ** (d - 1 - m) * (q ** m - 1)
        assert got == want
