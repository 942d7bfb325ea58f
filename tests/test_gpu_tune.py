"""The autotuner: every kernel choice it can make gives the same histogram,
and its cache file carries a choice over to a new process."""
import os
import subprocess
import sys

import pytest

from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import JobSpec, MONIC_NOSUB

from hwc_helpers import assert_hist_equal, oracle_hist

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# g = 3, q = 11, monic degree 8 with c_7 = 0: 11^7 members, large enough for
# the tuner's probe (two work items per resident warp)
BIG = JobSpec(3, 11, MONIC_NOSUB, 8)


def _job(spec):
    return hwc.make_job(spec.g, spec.q, spec.kind, spec.degree, spec.first, spec.n(), spec.seed,
                        spec.sample_count)


def test_tuned_equals_untuned_and_forced_kernels():
    j = _job(BIG)
    tuned = hwc.Batch([j], flags=0)
    tuned.launch()
    h_tuned = tuned.result(0)
    method = tuned.job_method(0)
    assert method in (1, 2)
    for flags in (hwc.FLAG_NO_TUNE, hwc.FLAG_NO_TUNE | hwc.FLAG_FAN1):
        other = hwc.Batch([j], flags=flags)
        other.launch()
        assert_hist_equal(other.result(0), (h_tuned.counts, h_tuned.mult))
        other.close()
    tuned.close()


def test_tuned_slice_matches_oracle(orc):
    # a slice of the tuned class (the class choice is cached from the full job)
    hwc.Batch([_job(BIG)], flags=0).close()
    spec = JobSpec(3, 11, MONIC_NOSUB, 8, first=11 ** 6 * 3 + 17, count=20000)
    b = hwc.Batch([_job(spec)], flags=0)
    b.launch()
    assert_hist_equal(b.result(0), oracle_hist(orc, spec))
    b.close()


_CHILD = r"""
import sys
sys.path.insert(0, %r)
from paper_1805_11991_gb300 import hwc
from paper_1805_11991_gb300.workloads import JobSpec, MONIC_NOSUB
s = JobSpec(3, 11, MONIC_NOSUB, 8)
j = hwc.make_job(s.g, s.q, s.kind, s.degree, s.first, s.n(), s.seed, s.sample_count)
b = hwc.Batch([j], flags=0)
b.launch()
h = b.result(0)
print(b.job_method(0), h.n_squarefree)
"""


def test_cache_file_carries_the_choice(tmp_path):
    path = tmp_path / "tune.txt"
    env = dict(os.environ, HWC_TUNE_CACHE=str(path))
    out1 = subprocess.run([sys.executable, "-c", _CHILD % ROOT], env=env, capture_output=True, text=True,
                          timeout=600)
    assert out1.returncode == 0, out1.stderr
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    fields = lines[0].split()
    assert len(fields) == 10 and fields[2:7] == ["3", "11", "8", "1", "0"]
    out2 = subprocess.run([sys.executable, "-c", _CHILD % ROOT], env=env, capture_output=True, text=True,
                          timeout=600)
    assert out2.returncode == 0, out2.stderr
    assert out2.stdout.split() == out1.stdout.split()
    assert out1.stdout.split()[0] == fields[7]            # the kernel the file names
    assert path.read_text().splitlines() == lines       # read back, not measured again
