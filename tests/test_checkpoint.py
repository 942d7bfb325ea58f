"""Histogram checkpoints (hwc_hist_save / hwc_hist_load): a file round trip
keeps the tuples, multiplicities, members examined and the job range (CPU,
no kernels); an interrupted job resumed from its checkpoint equals the job
counted in one go (GPU)."""
import os

import numpy as np
import pytest

from paper_1805_11991_gb300 import hwc


def test_checkpoint_round_trip(tmp_path):
    g = 3
    counts = np.array([[5, 20, 30], [4, 18, 33], [5, 20, 31]], np.int32)
    mult = np.array([7, 1, 2], np.uint64)
    h = hwc.Histogram(g, counts, mult, int(mult.sum()), 40)
    job = hwc.make_job(3, 5, hwc.FAM_MONIC_NOSUB, 7, 100, 40)
    path = str(tmp_path / "h.ckpt")
    hwc.hist_save(h, path, job)
    back, jb = hwc.hist_load(path)
    order = np.lexsort(counts.T[::-1])
    np.testing.assert_array_equal(back.counts, counts[order])
    np.testing.assert_array_equal(back.mult, mult[order])
    assert back.n_total == 40 and back.n_squarefree == 10
    assert (jb.g, jb.q, jb.family.kind, jb.family.degree, jb.first, jb.count) == (3, 5, 1, 7, 100, 40)
    hwc.hist_save(h, path)                 # without a job
    _, jb = hwc.hist_load(path)
    assert jb is None


def test_checkpoint_rejects_bad_files(tmp_path):
    path = str(tmp_path / "bad.ckpt")
    with open(path, "wb") as fh:
        fh.write(b"not a histogram at all")
    with pytest.raises(hwc.HwcError) as e:
        hwc.hist_load(path)
    assert e.value.code == hwc.ERR_ARG
    h = hwc.Histogram(2, np.array([[3, 9]], np.int32), np.array([2], np.uint64), 2, 2)
    good = str(tmp_path / "good.ckpt")
    hwc.hist_save(h, good)
    with open(good, "rb") as fh:
        data = fh.read()
    with open(path, "wb") as fh:
        fh.write(data[:-4])                  # truncated
    with pytest.raises(hwc.HwcError):
        hwc.hist_load(path)
    with pytest.raises(hwc.HwcError):
        hwc.hist_load(str(tmp_path / "missing.ckpt"))


@pytest.mark.gpu
def test_resume_from_checkpoint_equals_one_run(tmp_path):
    g, q, d = 3, 9, 7
    fam = hwc.make_family(hwc.FAM_MONIC_NOSUB, d)
    n = hwc.family_size(q, fam)
    cut = n // 3 + 12345                    # not on a group boundary
    path = str(tmp_path / "part.ckpt")
    first = hwc.count(g, q, fam, 0, cut)
    hwc.hist_save(first, path, hwc.make_job(g, q, hwc.FAM_MONIC_NOSUB, d, 0, cut))
    # a later process: load, count the rest, merge
    done, job = hwc.hist_load(path)
    assert job.first + job.count == cut
    rest = hwc.count(g, q, fam, cut, n - cut)
    merged = hwc.hist_merge(done, rest)
    whole = hwc.count(g, q, fam, 0, n)
    np.testing.assert_array_equal(merged.counts, whole.counts)
    np.testing.assert_array_equal(merged.mult, whole.mult)
    assert merged.n_total == whole.n_total == n
    assert os.path.getsize(path) > 0
