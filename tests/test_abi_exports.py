"""The C ABI library loads on a machine without a GPU and exports every
function include/hwc.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1805_11991_gb300 import build as hbuild
from paper_1805_11991_gb300 import hwc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hwc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hwc_field_tables", "hwc_count", "hwc_hist_read", "hwc_batch_run", "hwc_serve_open"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(hbuild.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", hbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hwc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_the_header():
    lib = hwc.load()
    for n in declared_functions():
        assert getattr(lib, n).argtypes is not None or getattr(lib, n).restype is not None, n


def test_family_sizes_host_only():
    assert hwc.family_size(31, hwc.make_family(hwc.FAM_MONIC_NOSUB, 5)) == 31 ** 4
    assert hwc.family_size(3, hwc.make_family(hwc.FAM_ALL_DEG, 6)) == 2 * 3 ** 6
    assert hwc.family_size(293, hwc.make_family(hwc.FAM_MONIC_NOSUB_SAMPLED, 5, 7, 1 << 24)) == 1 << 24
    # windows of a sampled family name members of the enumerated family
    assert hwc.family_size(13, hwc.make_family(hwc.FAM_MONIC_NOSUB_SAMPLED_WINDOW, 9, 11, 1 << 26)) == 13 ** 8
    with pytest.raises(hwc.HwcError) as e:
        hwc.family_size(13, hwc.make_family(hwc.FAM_MONIC_NOSUB_SAMPLED_WINDOW, 9, 11, 0))
    assert e.value.code == hwc.ERR_ARG
    with pytest.raises(hwc.HwcError) as e:
        hwc.family_size(15, hwc.make_family(hwc.FAM_MONIC_NOSUB, 5))
    assert e.value.code == hwc.ERR_ARG


@pytest.mark.parametrize("g,q,kind,d,first,count,code", [
    (2, 15, 1, 5, 0, 1, hwc.ERR_ARG),          # 15 is not a prime power
    (2, 4, 1, 5, 0, 1, hwc.ERR_ARG),           # even q
    (2, 31, 1, 7, 0, 1, hwc.ERR_ARG),          # degree not 2g+1 / 2g+2
    (5, 3, 1, 11, 0, 1, hwc.ERR_ARG),          # g > 4
    (2, 31, 1, 5, 31 ** 4, 1, hwc.ERR_RANGE),  # past the end
    (2, 31, 9, 5, 0, 1, hwc.ERR_ARG),          # unknown family
    (4, 37, 1, 9, 0, 1, hwc.ERR_TOO_LARGE),    # 37^4 above the largest field
])
def test_argument_errors_before_any_cuda_call(g, q, kind, d, first, count, code):
    fam = hwc.make_family(kind, d)
    with pytest.raises(hwc.HwcError) as e:
        hwc.count(g, q, fam, first, count)
    assert e.value.code == code
    with pytest.raises(hwc.HwcError) as e:
        hwc.count_members(g, q, fam, first, count)
    assert e.value.code == code


def test_histogram_merge_host_only():
    import numpy as np
    a = hwc.Histogram(2, np.array([[4, 10], [5, 9]], np.int32), np.array([3, 1], np.uint64), 4, 10)
    b = hwc.Histogram(2, np.array([[3, 12], [5, 9]], np.int32), np.array([2, 5], np.uint64), 7, 9)
    m = hwc.hist_merge(a, b)
    assert m.as_dict() == {(3, 12): 2, (4, 10): 3, (5, 9): 6}
    assert m.n_squarefree == 11 and m.n_total == 19
