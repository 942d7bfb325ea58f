"""Every configuration of the benchmark against the oracle's stored histograms
(tests/golden/oracle_histograms.json, written by make_oracle_histograms.py,
which calls only oracle/): whole families where the oracle finishes them in
minutes (configuration 2 in full, configuration 4's q = 13, configuration 5's
q = 7, configurations 1 and 3 up to q = 31), else a slice from the start and a
ragged slice from the middle of the job.  Bit-exact: the tuples and
multiplicities of the GPU histogram hash to the oracle's digest.

Each configuration runs as one batch in a CUDA graph (the launch the benchmark
times), and every job also runs alone through hwc_count with each count kernel
that applies (automatic choice, forced per-member Horner, forced one-level
fan-out)."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "oracle_histograms.json")) as _fh:
    GOLD = json.load(_fh)["jobs"]
CONFIGS = sorted({e["config"] for e in GOLD.values()})


def _digest(counts: np.ndarray, mult: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(counts, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(mult, dtype="<u8").tobytes())
    return h.hexdigest()


def _job(e):
    return hwc.make_job(e["g"], e["q"], e["kind"], e["degree"], e["first"], e["count"], e["seed"],
                        e["sample_count"])


def _check(h, e, what):
    assert h.n_total == e["count"], what
    assert h.n_squarefree == e["n_squarefree"], what
    if "tuples" in e:
        ref = np.asarray(e["tuples"], dtype=np.int64)
        np.testing.assert_array_equal(h.counts, ref[:, :-1], err_msg=what)
        np.testing.assert_array_equal(h.mult.astype(np.int64), ref[:, -1], err_msg=what)
    c = h.counts.astype(object)
    m = h.mult.astype(object)
    m1 = [int(sum(m * c[:, k])) for k in range(e["g"])]
    m2 = [int(sum(m * c[:, k] * c[:, k])) for k in range(e["g"])]
    assert (len(h.mult), m1, m2) == (e["n_entries"], e["moment1"], e["moment2"]), what
    assert _digest(h.counts, h.mult) == e["sha256"], what


@pytest.mark.parametrize("config", CONFIGS)
def test_config_batch_in_graph_matches_oracle(config):
    entries = [e for e in GOLD.values() if e["config"] == config]
    b = hwc.Batch([_job(e) for e in entries], flags=hwc.FLAG_GRAPH)
    try:
        for rep in range(2):   # a replay of the graph gives the same histograms
            b.launch()
            for i, e in enumerate(entries):
                _check(b.result(i), e, f"{config} job {i} replay {rep}")
    finally:
        b.close()


def _ids(k):
    e = GOLD[k]
    return f"{e['config']}-g{e['g']}q{e['q']}d{e['degree']}k{e['kind']}-{e['first']}+{e['count']}"


KERNEL_FLAGS = {"auto": 0, "horner": hwc.FLAG_HORNER, "fan1": hwc.FLAG_FAN1}


@pytest.mark.parametrize("kernel", sorted(KERNEL_FLAGS))
@pytest.mark.parametrize("key", sorted(GOLD), ids=_ids)
def test_job_alone_matches_oracle(key, kernel):
    e = GOLD[key]
    if kernel == "fan1" and (e["kind"] == hwc.FAM_MONIC_NOSUB_SAMPLED or e["q"] > 31):
        pytest.skip("same kernel as 'auto' (the one-level fan-out applies only to enumerated q <= 31 jobs)")
    if kernel == "horner" and e["kind"] == hwc.FAM_MONIC_NOSUB_SAMPLED:
        pytest.skip("same kernel as 'auto' (sampled families run the per-member kernel)")
    fam = hwc.make_family(e["kind"], e["degree"], e["seed"], e["sample_count"])
    h = hwc.count(e["g"], e["q"], fam, e["first"], e["count"], KERNEL_FLAGS[kernel])
    _check(h, e, f"{_ids(key)} {kernel}")
