"""N_{g,q} of eq. 1.2 (HWC_FLAG_LAMBDA): histograms keyed by the point
counts and the factorisation pattern lambda(f), against the oracle, which
factors f by distinct-degree factorisation (no point counts involved)."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import ALL_DEG, MONIC_NOSUB, MONIC_NOSUB_SAMPLED, JobSpec

pytestmark = pytest.mark.gpu

CASES = [
    JobSpec(1, 5, ALL_DEG, 3),
    JobSpec(1, 7, ALL_DEG, 4),
    JobSpec(2, 3, ALL_DEG, 5),
    JobSpec(2, 3, ALL_DEG, 6),
    JobSpec(2, 5, ALL_DEG, 6, 7, 40000),
    JobSpec(2, 9, ALL_DEG, 5, 100, 30000),
    JobSpec(2, 31, MONIC_NOSUB, 6, 12345, 20000),
    JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 400, seed=7, sample_count=1 << 24),
    JobSpec(3, 3, ALL_DEG, 7),
    JobSpec(3, 3, ALL_DEG, 8),
    JobSpec(3, 7, MONIC_NOSUB, 8, 5000, 8000),
    JobSpec(4, 3, ALL_DEG, 10, 1000, 6000),
    JobSpec(4, 5, MONIC_NOSUB, 9, 0, 3000),
]


def _ids(s):
    return f"g{s.g}q{s.q}d{s.degree}k{s.kind}-{s.first}+{s.n()}"


@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_lambda_histogram_matches_oracle(orc, spec):
    fam = hwc.make_family(spec.kind, spec.degree, spec.seed, spec.sample_count)
    h = hwc.count(spec.g, spec.q, fam, spec.first, spec.n(), hwc.FLAG_LAMBDA)
    tuples, codes, mult = orc.lambda_histogram(spec.g, spec.q, spec.kind, spec.degree, spec.first, spec.n(),
                                               seed=spec.seed, sample_count=spec.sample_count)
    assert h.lam is not None
    np.testing.assert_array_equal(h.lam, codes)
    np.testing.assert_array_equal(h.counts, tuples)
    np.testing.assert_array_equal(h.mult, mult)
    # summed over the patterns it is the plain histogram
    plain = hwc.count(spec.g, spec.q, fam, spec.first, spec.n())
    assert plain.lam is None
    agg = {}
    for row, m in zip(h.counts, h.mult):
        agg[tuple(int(v) for v in row)] = agg.get(tuple(int(v) for v in row), 0) + int(m)
    assert agg == plain.as_dict()


def test_lambda_refuses_all_points():
    fam = hwc.make_family(ALL_DEG, 5)
    with pytest.raises(hwc.HwcError) as e:
        hwc.count(2, 3, fam, 0, 100, hwc.FLAG_LAMBDA | hwc.FLAG_ALL_POINTS)
    assert e.value.code == hwc.ERR_ARG
