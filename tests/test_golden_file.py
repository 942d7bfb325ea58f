"""The stored oracle histograms (tests/golden/oracle_histograms.json) against
facts that do not come from the file: the oracle recomputes the cheap entries
and must give the same digest, square-free totals of whole families equal
their closed forms, and every stored tuple obeys the Hasse-Weil bound."""
import hashlib
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "oracle_histograms.json")) as _fh:
    GOLD = json.load(_fh)["jobs"]


def _digest(counts, mult):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(counts, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(mult, dtype="<u8").tobytes())
    return h.hexdigest()


def _p_of(q):
    for p in range(3, q + 1, 2):
        if q % p == 0:
            return p


def test_every_configuration_is_present():
    assert {e["config"] for e in GOLD.values()} == {f"config{i}" for i in range(1, 6)}
    # the jobs the parity plan names: g=3 q=17 and q=25, g=4 q=9 and q=11, q=293, the q=13 samples
    have = {(e["g"], e["q"]) for e in GOLD.values()}
    assert {(3, 17), (3, 25), (3, 27), (4, 9), (4, 11), (4, 13), (2, 293), (2, 31)} <= have


@pytest.mark.parametrize("key", sorted(k for k, e in GOLD.items() if e["count"] * e["q"] ** e["g"] < 3e7))
def test_cheap_entries_recomputed_by_the_oracle(orc, key):
    e = GOLD[key]
    counts, mult, nsq = orc.cpu_count(e["g"], e["q"], e["kind"], e["degree"], e["first"], e["count"],
                                      seed=e["seed"], sample_count=e["sample_count"])
    assert nsq == e["n_squarefree"]
    assert len(mult) == e["n_entries"]
    assert _digest(counts, mult) == e["sha256"]


def test_whole_family_squarefree_totals():
    """ALL_d: (q-1)(q^d - q^(d-1)) square-free members; MZ_d with p not dividing
    d: q^(d-1) - q^(d-2) (X -> X + b maps the monic square-free polynomials of
    degree d onto those with c_{d-1} = 0, q to one)."""
    checked = 0
    for e in GOLD.values():
        q, d, kind = e["q"], e["degree"], e["kind"]
        if e["first"] != 0:
            continue
        if kind == 0 and e["count"] == (q - 1) * q ** d:
            assert e["n_squarefree"] == (q - 1) * (q ** d - q ** (d - 1))
            checked += 1
        elif kind == 1 and e["count"] == q ** (d - 1) and d % _p_of(q):
            assert e["n_squarefree"] == q ** (d - 1) - q ** (d - 2)
            checked += 1
    assert checked >= 10


def test_stored_tuples_obey_hasse_weil():
    """|q^k + 1 - #C_k| <= 2 g q^(k/2) for every stored tuple (exact integer test)."""
    n = 0
    for e in GOLD.values():
        for row in e.get("tuples", []):
            *cs, m = row
            assert m > 0
            for k, c in enumerate(cs, start=1):
                a = e["q"] ** k + 1 - c
                assert a * a <= 4 * e["g"] ** 2 * e["q"] ** k
            n += 1
        if "tuples" in e:
            assert sum(r[-1] for r in e["tuples"]) == e["n_squarefree"]
    assert n > 0


def test_moments_match_stored_tuples():
    for e in GOLD.values():
        if "tuples" not in e:
            continue
        t = np.asarray(e["tuples"], dtype=object)
        for k in range(e["g"]):
            assert int(sum(t[:, -1] * t[:, k])) == e["moment1"][k]
            assert int(sum(t[:, -1] * t[:, k] * t[:, k])) == e["moment2"][k]
