"""Hand-derived point counts (tests/golden/hand_counts.txt): the oracle on
the CPU and the library on the GPU against values worked out by hand from the
definition of #C (Sec. 1.1)."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    out = []
    with open(os.path.join(HERE, "golden", "hand_counts.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            head, counts, _why = line.split("|", 2)
            q, g, kind, d, *coeffs = (int(v) for v in head.split())
            assert len(coeffs) == d + 1
            out.append((q, g, kind, d, coeffs, [int(v) for v in counts.split()]))
    return out


def _index(q, kind, d, c):
    if kind == 0:
        return sum(c[i] * q ** i for i in range(d)) + (c[d] - 1) * q ** d
    assert c[d] == 1 and c[d - 1] == 0
    return sum(c[i] * q ** i for i in range(d - 1))


CASES = _cases()
IDS = [f"q{q}g{g}k{kind}d{d}" + "".join(map(str, c)) for q, g, kind, d, c, _ in CASES]


@pytest.mark.parametrize("q,g,kind,d,coeffs,want", CASES, ids=IDS)
def test_oracle_hand_counts(orc, q, g, kind, d, coeffs, want):
    i = _index(q, kind, d, coeffs)
    assert list(orc.decode(q, kind, d, i)) == coeffs
    counts, sqf = orc.count_polys(g, q, kind, d, i, 1)
    assert sqf[0] == 1
    assert counts[0].tolist() == want


@pytest.mark.gpu
@pytest.mark.parametrize("flags", ["auto", "fan1", "horner"])
@pytest.mark.parametrize("q,g,kind,d,coeffs,want", CASES, ids=IDS)
def test_library_hand_counts(q, g, kind, d, coeffs, want, flags):
    from paper_1805_11991_gb300 import hwc
    fl = {"auto": 0, "fan1": hwc.FLAG_FAN1, "horner": hwc.FLAG_HORNER}[flags]
    i = _index(q, kind, d, coeffs)
    counts, sqf = hwc.count_members(g, q, hwc.make_family(kind, d), i, 1, flags=fl)
    assert sqf[0] == 1
    assert counts[0].tolist() == want
