"""World-size-2 gloo ranks on CPU: sharded member ranges, gathered and merged
histograms equal the single-process histogram.  Each rank counts its slice
with the oracle (no GPU here); the sharding and the merge are the library's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, spec, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import oracle
    from paper_1805_11991_gb300 import hwc, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, q, kind, d, first, count = spec
    a, n = shard.shard_range(first, count, rank, world)
    counts, sqf = oracle.count_polys(g, q, kind, d, a, n, threads=2)
    tuples, mult = oracle.histogram(counts, sqf)
    h = hwc.Histogram(g, tuples, mult, int(mult.sum()), n)
    merged = shard.gather_merge(h)
    if rank == 0:
        out.put((merged.counts.tolist(), merged.mult.tolist(), merged.n_squarefree, merged.n_total))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("spec", [(2, 7, 1, 5, 0, 7 ** 4), (2, 5, 0, 6, 100, 30001), (3, 3, 1, 7, 11, 700)])
def test_two_gloo_ranks_merge_to_single(orc, spec):
    ctx = mp.get_context("spawn")
    q_out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, spec, q_out)) for r in range(2)]
    for p in procs:
        p.start()
    res = q_out.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, q, kind, d, first, count = spec
    tuples, mult = orc.count_histogram(g, q, kind, d, first, count)
    np.testing.assert_array_equal(np.asarray(res[0], np.int32).reshape(-1, g), tuples)
    np.testing.assert_array_equal(np.asarray(res[1], np.uint64), mult)
    assert res[2] == int(mult.sum()) and res[3] == count


def test_shard_ranges_cover_exactly():
    from paper_1805_11991_gb300 import shard
    for first, count, world in [(0, 10, 3), (5, 1, 4), (7, 0, 2), (3, 1000003, 8)]:
        got = [shard.shard_range(first, count, r, world) for r in range(world)]
        pos = first
        for a, n in got:
            assert a == pos and n >= 0
            pos += n
        assert pos == first + count


def _window_rank_main(rank, world, port, spec, out):
    """Rank `rank` counts its share of a densely drawn sample (a window of
    the family, from the library's sharding rule) with the oracle: the
    oracle's counts of every draw, kept where the drawn member lies in the
    window."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import oracle
    from paper_1805_11991_gb300 import hwc, shard
    from paper_1805_11991_gb300.workloads import MONIC_NOSUB_SAMPLED_WINDOW, JobSpec, shard_job
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    job = JobSpec(*spec)
    part = shard_job(job, rank, world)
    assert part.kind == MONIC_NOSUB_SAMPLED_WINDOW
    g, q, d, seed, sc = job.g, job.q, job.degree, job.seed, job.sample_count
    counts, sqf = oracle.count_polys(g, q, job.kind, d, 0, sc, seed=seed, sample_count=sc, threads=2)
    idx = np.array([sum(int(c) * q ** i for i, c in enumerate(oracle.decode(q, job.kind, d, j, seed)[:d - 1]))
                    for j in range(sc)])
    inw = (idx >= part.first) & (idx < part.first + part.n())
    tuples, mult = oracle.histogram(counts[inw], sqf[inw])
    h = hwc.Histogram(g, tuples, mult, int(mult.sum()), int(inw.sum()))
    merged = shard.gather_merge(h)
    if rank == 0:
        out.put((merged.counts.tolist(), merged.mult.tolist(), merged.n_squarefree, merged.n_total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_windowed_sample_merge_to_single(orc):
    # g=2, q=13, degree 5, 20000 draws (seed 11) of 13^4 members: dense enough
    # for the whole-family kernel, so each rank takes a window of the family
    from paper_1805_11991_gb300.workloads import MONIC_NOSUB_SAMPLED
    spec = (2, 13, MONIC_NOSUB_SAMPLED, 5, 0, 20000, 11, 20000)
    ctx = mp.get_context("spawn")
    q_out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_window_rank_main, args=(r, 2, port, spec, q_out)) for r in range(2)]
    for p in procs:
        p.start()
    res = q_out.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    tuples, mult, nsq = orc.cpu_count(2, 13, MONIC_NOSUB_SAMPLED, 5, 0, 20000, seed=11, sample_count=20000)
    np.testing.assert_array_equal(np.asarray(res[0], np.int32).reshape(-1, 2), tuples)
    np.testing.assert_array_equal(np.asarray(res[1], np.uint64), mult)
    assert res[2] == nsq and res[3] == 20000


def test_shard_job_parts_cover_the_job():
    from paper_1805_11991_gb300.workloads import (MONIC_NOSUB, MONIC_NOSUB_SAMPLED, MONIC_NOSUB_SAMPLED_WINDOW,
                                                  JobSpec, shard_job, split_job)
    dense = JobSpec(4, 13, MONIC_NOSUB_SAMPLED, 9, seed=11, sample_count=1 << 26)
    sparse = JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, seed=7, sample_count=1 << 24)
    plain = JobSpec(3, 27, MONIC_NOSUB, 7, 5, 1000003)
    for job in (dense, sparse, plain):
        for world in (1, 2, 3, 8):
            parts = [shard_job(job, r, world) for r in range(world)]
            windowed = job is dense
            assert all((p.kind == MONIC_NOSUB_SAMPLED_WINDOW) == windowed for p in parts)
            pos = 0 if windowed else job.first
            for p in parts:
                assert p.first == pos
                pos += p.n()
            assert pos == (13 ** 8 if windowed else job.first + job.n())
            assert [p for p in parts if p.n() > 0] == split_job(job, world)
