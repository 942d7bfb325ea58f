"""The oracle and the GPU path share no code, the package never reaches the
oracle, and the product path fails loudly when its CUDA library is missing
(there is no CPU fallback)."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1805_11991_gb300")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_imports_the_oracle():
    for path in _files(PKG, (".py",)):
        text = open(path).read()
        assert not re.search(r"^\s*(import oracle|from oracle\b|from \.\.oracle)", text, re.M), path
        assert "liboracle" not in text and "hwc_oracle" not in text, path


def test_sources_share_no_headers():
    for path in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")):
        for inc in re.findall(r'#include\s+"([^"]+)"', open(path).read()):
            assert "oracle" not in inc, (path, inc)
    oracle_c = open(os.path.join(ROOT, "oracle", "hwc_oracle.c")).read()
    for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', oracle_c):
        assert not inc.startswith(("hwc", "../", "include/")) and "csrc" not in inc, inc


def test_missing_library_fails_loudly():
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1805_11991_gb300 import build, hwc\n"
        "build.LIB = '/nonexistent/libhwc.so'\n"
        "try:\n"
        "    hwc.load(build_if_missing=False)\n"
        "except OSError as e:\n"
        "    print('raised', e)\n"
        "else:\n"
        "    print('loaded')\n" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised"), out.stdout
