"""Test helpers: run the same job spec through the GPU library and the oracle."""
from __future__ import annotations

import numpy as np

from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import JobSpec


def to_job(spec: JobSpec) -> hwc.Job:
    return hwc.make_job(spec.g, spec.q, spec.kind, spec.degree, spec.first, spec.n(),
                        spec.seed, spec.sample_count)


def gpu_hist(spec: JobSpec, flags: int = 0):
    j = to_job(spec)
    return hwc.count(spec.g, spec.q, j.family, spec.first, spec.n(), flags)


def gpu_members(spec: JobSpec, unfiltered: bool = False, flags: int = 0):
    j = to_job(spec)
    return hwc.count_members(spec.g, spec.q, j.family, spec.first, spec.n(), unfiltered, flags)


def oracle_members(orc, spec: JobSpec, filter: bool = True):
    return orc.count_polys(spec.g, spec.q, spec.kind, spec.degree, spec.first, spec.n(),
                           seed=spec.seed, sample_count=spec.sample_count, filter=filter)


def oracle_hist(orc, spec: JobSpec):
    counts, sqf = oracle_members(orc, spec)
    return orc.histogram(counts, sqf)


def assert_hist_equal(h, ref):
    tuples, mult = ref
    np.testing.assert_array_equal(h.counts, tuples)
    np.testing.assert_array_equal(h.mult, mult)
    assert h.n_squarefree == int(mult.sum())
