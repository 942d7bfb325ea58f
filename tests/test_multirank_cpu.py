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
