"""Batched execution (one persistent launch, CUDA graph) and the serving loop:
every job's histogram is the same alone and in any mix (exact integers)."""
import time

import numpy as np
import pytest

from hwc_helpers import assert_hist_equal, gpu_hist, oracle_hist, to_job
from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import (ALL_DEG, MONIC_NOSUB, MONIC_NOSUB_SAMPLED, JobSpec,
                                               split_job)

pytestmark = pytest.mark.gpu

MIX = [
    JobSpec(2, 3, MONIC_NOSUB, 5), JobSpec(2, 13, MONIC_NOSUB, 5), JobSpec(2, 31, MONIC_NOSUB, 5, 0, 200_000),
    JobSpec(2, 3, ALL_DEG, 6), JobSpec(3, 5, MONIC_NOSUB, 7), JobSpec(4, 3, MONIC_NOSUB, 9),
    JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 3000, seed=7, sample_count=1 << 24),
    JobSpec(3, 13, MONIC_NOSUB, 8, 0, 50_000), JobSpec(2, 9, MONIC_NOSUB, 6),
]


def _alone():
    return [gpu_hist(s) for s in MIX]


def _same(a, b):
    assert a.g == b.g and a.n_total == b.n_total and a.n_squarefree == b.n_squarefree
    np.testing.assert_array_equal(a.counts, b.counts)
    np.testing.assert_array_equal(a.mult, b.mult)


@pytest.mark.parametrize("flags", [0, hwc.FLAG_GRAPH, hwc.FLAG_PLAIN, hwc.FLAG_PLAIN | hwc.FLAG_GRAPH])
def test_batch_equals_alone(flags):
    alone = _alone()
    b = hwc.Batch([to_job(s) for s in MIX], flags=flags | hwc.FLAG_TIMING)
    for rep in range(2):           # relaunch: histograms are cleared each run
        b.launch()
        for i in range(len(MIX)):
            _same(b.result(i), alone[i])
        assert b.kernel_ms() > 0
    n = b.kernel_launches()
    def key(s):
        fan = s.kind != MONIC_NOSUB_SAMPLED and s.q <= 63
        method = (2 if s.q <= 31 else 1) if fan else 0
        return (s.degree, method, (1 if s.q <= 31 else 2) if fan else 0)
    groups = len({key(s) for s in MIX})
    assert n == 2 + (len(MIX) if flags & hwc.FLAG_PLAIN else groups)
    b.close()


def test_small_jobs_match_oracle(orc):
    for s in MIX:
        if s.n() * s.nominal_evals_per_member() < 5e7 and s.q < 100:
            assert_hist_equal(gpu_hist(s), oracle_hist(orc, s))


def test_shards_merge_to_whole():
    spec = JobSpec(2, 27, MONIC_NOSUB, 6, 0, 1_000_003)
    whole = gpu_hist(spec)
    parts = [gpu_hist(p) for p in split_job(spec, 5)]
    acc = parts[0]
    for p in parts[1:]:
        acc = hwc.hist_merge(acc, p)
    _same(acc, whole)


def test_batch_run_convenience():
    outs = hwc.batch_run([to_job(s) for s in MIX[:3]])
    alone = _alone()
    for a, b in zip(outs, alone[:3]):
        _same(a, b)


def test_server_results_same_alone_and_mixed():
    alone = _alone()
    srv = hwc.Server(device_bytes=2 << 30, max_active=4, step_items=64)
    tickets = []
    for i, s in enumerate(MIX):       # arrivals while earlier requests run
        tickets.append(srv.submit(to_job(s)))
        time.sleep(0.002 * (i % 3))
    for i, t in enumerate(tickets):
        h = srv.poll(t, timeout_ms=120_000)
        assert h is not None
        _same(h, alone[i])
        queued, total = srv.latency(t)
        assert total >= queued >= 0
    with pytest.raises(hwc.HwcError):
        srv.poll(tickets[0])          # already collected
    srv.close()


def test_server_rejects_oversized_request():
    srv = hwc.Server(device_bytes=1 << 20, max_active=2)
    t = srv.submit(to_job(JobSpec(3, 27, MONIC_NOSUB, 7, 0, 10_000_000)))
    with pytest.raises(hwc.HwcError) as e:
        srv.poll(t, timeout_ms=60_000)
    assert e.value.code == hwc.ERR_BUSY
    srv.close()
