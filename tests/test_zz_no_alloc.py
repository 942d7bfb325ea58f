"""The allocation-free histogram entry point (hwc_count_noalloc) against the
regular one (hwc_count): the same histogram, exactly, on calls in a row.

Some callers cannot allocate device memory when they count (processes whose
device memory is reserved up front, or threads that must not call the
synchronising cudaMalloc); this
entry point keeps its working memory in a fixed device array and writes into
buffers the caller owns.  This file runs last so that a failure here leaves
every other test already run."""
import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import ALL_DEG, MONIC_NOSUB, MONIC_NOSUB_SAMPLED, JobSpec

pytestmark = pytest.mark.gpu

CALLS = [
    JobSpec(2, 31, MONIC_NOSUB, 5, 1000, 50_000),
    JobSpec(2, 13, MONIC_NOSUB, 6),
    JobSpec(2, 31, MONIC_NOSUB, 5, 1000, 50_000),   # same job again: no state left behind
    JobSpec(3, 7, MONIC_NOSUB, 7, 0, 8_000),
    JobSpec(2, 3, ALL_DEG, 6),
    JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 200, seed=7, sample_count=1 << 24),
]


def _noalloc(spec, tables_cache, max_entries=20000, free_bytes=None):
    """Run one call; with free_bytes (a list) append the device's free memory
    just before and just after the call (torch's allocator idle meanwhile)."""
    import torch
    tabs = []
    for k in range(1, spec.g + 1):
        key = (spec.q, k)
        if key not in tables_cache:
            tables_cache[key] = hwc.Tables(spec.q, k)
        tabs.append(tables_cache[key])
    counts = torch.full((max_entries, spec.g), -1, dtype=torch.int32, device="cuda")
    mult = torch.zeros(max_entries, dtype=torch.int64, device="cuda")
    n_out = torch.zeros(3, dtype=torch.int64, device="cuda")
    fam = hwc.make_family(spec.kind, spec.degree, spec.seed, spec.sample_count)
    torch.cuda.synchronize()
    if free_bytes is not None:
        free_bytes.append(torch.cuda.mem_get_info()[0])
    hwc.count_noalloc(spec.g, spec.q, fam, spec.first, spec.n(), tabs, max_entries,
                      counts.data_ptr(), mult.data_ptr(), n_out.data_ptr())
    if free_bytes is not None:
        free_bytes.append(torch.cuda.mem_get_info()[0])
    n, nsq, ntot = (int(v) for v in n_out.cpu())
    c = counts[:n].cpu().numpy()
    m = mult[:n].cpu().numpy().astype(np.uint64)
    order = np.lexsort(c.T[::-1])
    return c[order], m[order], nsq, ntot


def test_noalloc_matches_count_on_calls_in_a_row():
    import torch
    torch.cuda.init()
    cache = {}
    for i, spec in enumerate(CALLS):
        fam = hwc.make_family(spec.kind, spec.degree, spec.seed, spec.sample_count)
        ref = hwc.count(spec.g, spec.q, fam, spec.first, spec.n())
        free = []
        c, m, nsq, ntot = _noalloc(spec, cache, free_bytes=free)
        np.testing.assert_array_equal(c, ref.counts)
        np.testing.assert_array_equal(m, ref.mult)
        assert nsq == ref.n_squarefree and ntot == ref.n_total == spec.n()
        # after the first call (which loads the kernels and looks up the
        # scratch array on this device) a call takes no device memory
        if i > 0:
            assert free[0] == free[1], f"device free memory changed across the call: {free}"


def test_noalloc_rejects_jobs_beyond_its_scratch():
    import torch
    cache = {}
    spec = JobSpec(3, 27, MONIC_NOSUB, 7, 0, 10_000_000)   # up to 4.6e5 distinct tuples
    with pytest.raises(hwc.HwcError) as e:
        _noalloc(spec, cache)
    assert e.value.code == hwc.ERR_TOO_LARGE
    with pytest.raises(hwc.HwcError) as e:                 # output too small
        _noalloc(JobSpec(2, 31, MONIC_NOSUB, 5, 0, 100_000), cache, max_entries=10)
    assert e.value.code == hwc.ERR_TOO_LARGE
