"""One point per Frobenius orbit (the default) against every point of every
field (HWC_FLAG_ALL_POINTS) and against the oracle, member by member, on each
count kernel: the per-member Horner kernel, the c_0 fan-out and the (c_1, c_0)
fan-out, for g = 1..4.  The orbit form of the sums is pinned on the oracle's
arithmetic in test_orbit_identity.py."""
import numpy as np
import pytest

from hwc_helpers import gpu_members, oracle_members
from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import ALL_DEG, MONIC_NOSUB, MONIC_NOSUB_SAMPLED, JobSpec

pytestmark = pytest.mark.gpu

CASES = [
    JobSpec(1, 7, ALL_DEG, 4, 0, 2000),
    JobSpec(2, 5, ALL_DEG, 6, 1000, 9000),
    JobSpec(2, 31, MONIC_NOSUB, 5, 5000, 3000),
    JobSpec(2, 27, MONIC_NOSUB, 6, 123456, 2500),
    JobSpec(2, 43, MONIC_NOSUB, 5, 77, 1500),
    JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 300, seed=7, sample_count=1 << 24),
    JobSpec(3, 9, MONIC_NOSUB, 7, 4000, 2000),
    JobSpec(3, 13, MONIC_NOSUB, 8, 99999, 1200),
    JobSpec(3, 17, MONIC_NOSUB, 7, 1000000, 600),
    JobSpec(4, 5, MONIC_NOSUB, 9, 2000, 1400),
    JobSpec(4, 7, MONIC_NOSUB, 10, 0, 700),
    JobSpec(4, 13, MONIC_NOSUB_SAMPLED, 9, 0, 200, seed=11, sample_count=1 << 26),
]

KERNELS = {"auto": 0, "horner": hwc.FLAG_HORNER, "fan1": hwc.FLAG_FAN1}


def _ids(s):
    return f"g{s.g}q{s.q}d{s.degree}k{s.kind}"


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_orbit_points_equal_all_points_and_oracle(orc, spec, kernel):
    flags = KERNELS[kernel]
    for unfiltered in (False, True):
        oc, os_ = orc.count_polys(spec.g, spec.q, spec.kind, spec.degree, spec.first, spec.n(),
                                  seed=spec.seed, sample_count=spec.sample_count, filter=not unfiltered)
        gc, gs = gpu_members(spec, unfiltered=unfiltered, flags=flags)
        ac, as_ = gpu_members(spec, unfiltered=unfiltered, flags=flags | hwc.FLAG_ALL_POINTS)
        np.testing.assert_array_equal(gs, os_)
        np.testing.assert_array_equal(as_, os_)
        np.testing.assert_array_equal(gc, oc, err_msg=f"orbit points, unfiltered={unfiltered}")
        np.testing.assert_array_equal(ac, oc, err_msg=f"all points, unfiltered={unfiltered}")


@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_orbit_histogram_equals_all_points(spec):
    from hwc_helpers import to_job
    j = to_job(spec)
    h1 = hwc.count(spec.g, spec.q, j.family, spec.first, spec.n())
    h2 = hwc.count(spec.g, spec.q, j.family, spec.first, spec.n(), hwc.FLAG_ALL_POINTS)
    np.testing.assert_array_equal(h1.counts, h2.counts)
    np.testing.assert_array_equal(h1.mult, h2.mult)
