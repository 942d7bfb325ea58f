"""The benchmark workload at full size, in the launch configuration bench.py
times (one persistent launch in a CUDA graph): properties that hold at any size
plus sampled members recomputed one by one by the oracle."""
import math
import random

import numpy as np
import pytest

from hwc_helpers import gpu_members, oracle_members, to_job
from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import JobSpec, config2

pytestmark = pytest.mark.gpu


def _weil_ok(h, q):
    """(a_1, a_2) of a genus-2 curve: a_1^2 = a_2 mod 2 (e_2 integral),
    |a_1| <= 4 sqrt(q), |e_2| <= 6 q."""
    for row in h.counts:
        a1 = q + 1 - int(row[0])
        a2 = q * q + 1 - int(row[1])
        if (a1 * a1 - a2) % 2:
            return False
        e2 = (a1 * a1 - a2) // 2
        if a1 * a1 > 16 * q or abs(e2) > 6 * q:
            return False
    return True


def test_config2_full_size():
    jobs = config2()
    b = hwc.Batch([to_job(s) for s in jobs], flags=hwc.FLAG_GRAPH)
    b.launch()
    for i, s in enumerate(jobs):
        h = b.result(i)
        assert h.n_total == s.n()
        assert h.n_squarefree == int(h.mult.sum())
        p = 3 if s.q == 27 else 31
        if s.degree % p:
            # translation X -> X + b: q^(d-1) - q^(d-2) square-free members
            assert h.n_squarefree == s.q ** (s.degree - 1) - s.q ** (s.degree - 2)
        assert _weil_ok(h, s.q)
    b.close()


@pytest.mark.parametrize("spec", config2(), ids=lambda s: f"q{s.q}d{s.degree}")
def test_config2_sampled_members(orc, spec):
    rnd = random.Random(spec.q * 10 + spec.degree)
    for first in sorted(rnd.sample(range(spec.n() - 40), 6)):
        sl = spec.with_range(first, 40)
        gc, gs = gpu_members(sl)
        oc, os_ = oracle_members(orc, sl)
        np.testing.assert_array_equal(gs, os_)
        np.testing.assert_array_equal(gc, oc)
