#!/usr/bin/env python
"""Write tests/golden/oracle_histograms.json: the CPU oracle's histograms of
the benchmark families (whole families where the oracle finishes them in
minutes, else a slice from the start and a ragged slice from the middle).

Calls only oracle/ (polynomial-basis arithmetic, no Zech tables): nothing here
comes from the GPU library.  Each entry records the job (g, q, family kind,
degree, seed, sample count, first member, member count) and the histogram of
(#C(F_q), ..., #C(F_{q^g})) over its square-free members (Algorithm 1, the
histogram increment with weight 1) as
  - n_entries, n_squarefree;
  - sha256 of the canonical bytes: the tuples sorted lexicographically as
    little-endian int32 (row-major), then the multiplicities as little-endian
    uint64;
  - moments sum_i mult_i * #C_k and sum_i mult_i * #C_k^2 per k (to tell a
    wrong tuple from a wrong multiplicity when a digest differs);
  - the full tuple list when it has at most 400 entries.

The run is incremental: entries already in the file with the same job are
kept.  Usage: python tests/golden/make_oracle_histograms.py [--threads N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_histograms.json")
ALL, MZ, MZS = 0, 1, 2


def family_size(q, kind, d, sample_count):
    if kind == ALL:
        return (q - 1) * q ** d
    if kind == MZ:
        return q ** (d - 1)
    return sample_count


def jobs():
    """(config, g, q, kind, degree, seed, sample_count, first, count).  Slices:
    'head' = the first n members, 'mid' = n members from just past the middle
    (an offset that cuts groups of q and q^2 consecutive members)."""
    out = []

    def whole(cfg, g, q, kind, d, seed=0, sc=0):
        out.append((cfg, g, q, kind, d, seed, sc, 0, family_size(q, kind, d, sc)))

    def slices(cfg, g, q, kind, d, n, seed=0, sc=0):
        size = family_size(q, kind, d, sc)
        out.append((cfg, g, q, kind, d, seed, sc, 0, n))
        mid = size // 2 + 12345
        out.append((cfg, g, q, kind, d, seed, sc, mid, n))

    # configuration 1: g=2, q=3, every f of exact degree 5 and 6
    whole("config1", 2, 3, ALL, 5)
    whole("config1", 2, 3, ALL, 6)
    # configuration 3: g=2, monic degree 5 with c_4 = 0 over every odd prime power q < 64,
    # plus q = 293 with 2^24 members drawn by seed 7
    for q in (3, 5, 7, 9, 11, 13, 17, 19, 23, 25, 27, 29, 31):
        whole("config3", 2, q, MZ, 5)
    for q in (37, 41, 43, 47, 49, 53, 59, 61):
        slices("config3", 2, q, MZ, 5, 1 << 17)
    slices("config3", 2, 293, MZS, 5, 1 << 14, seed=7, sc=1 << 24)
    # configuration 4: g=3, monic degree 7 with c_6 = 0, q in {13, 17, 25, 27}
    slices("config4", 3, 17, MZ, 7, 1 << 17)
    slices("config4", 3, 25, MZ, 7, 1 << 16)
    slices("config4", 3, 27, MZ, 7, 1 << 16)
    # configuration 5: g=4, monic degree 9 with c_8 = 0, q in {7, 9, 11}, and
    # q = 13 with 2^26 members drawn by seed 11
    slices("config5", 4, 9, MZ, 9, 1 << 17)
    slices("config5", 4, 11, MZ, 9, 1 << 16)
    slices("config5", 4, 13, MZS, 9, 1 << 15, seed=11, sc=1 << 26)
    # whole families that take minutes on the oracle, last
    whole("config4", 3, 13, MZ, 7)
    whole("config5", 4, 7, MZ, 9)
    # configuration 2: g=2, q = 31 and 27, monic degree 5 and 6 with c_{d-1} = 0
    for q in (27, 31):
        for d in (5, 6):
            whole("config2", 2, q, MZ, d)
    return out


def key(j):
    cfg, g, q, kind, d, seed, sc, first, count = j
    return f"{cfg}:g{g}:q{q}:kind{kind}:d{d}:seed{seed}:sc{sc}:first{first}:count{count}"


def digest(counts: np.ndarray, mult: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(counts, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(mult, dtype="<u8").tobytes())
    return h.hexdigest()


def summarize(counts: np.ndarray, mult: np.ndarray, n_sqf: int) -> dict:
    c = counts.astype(object)
    m = mult.astype(object)
    g = counts.shape[1]
    d = {
        "n_entries": int(counts.shape[0]),
        "n_squarefree": int(n_sqf),
        "sha256": digest(counts, mult),
        "moment1": [int(sum(m * c[:, k])) for k in range(g)],
        "moment2": [int(sum(m * c[:, k] * c[:, k])) for k in range(g)],
    }
    if counts.shape[0] <= 400:
        d["tuples"] = [[int(v) for v in row] + [int(mm)] for row, mm in zip(counts, mult)]
    return d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    oracle.build()
    try:
        with open(OUT) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {"about": __doc__.strip().splitlines()[0], "jobs": {}}
    for j in jobs():
        k = key(j)
        if k in data["jobs"]:
            continue
        cfg, g, q, kind, d, seed, sc, first, count = j
        t0 = time.time()
        counts, mult, n_sqf = oracle.cpu_count(g, q, kind, d, first, count, seed=seed, sample_count=sc,
                                               threads=args.threads)
        entry = {"config": cfg, "g": g, "q": q, "kind": kind, "degree": d, "seed": seed,
                 "sample_count": sc, "first": first, "count": count}
        entry.update(summarize(counts, mult, n_sqf))
        data["jobs"][k] = entry
        with open(OUT + ".tmp", "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(f"{k}: {entry['n_entries']} tuples, {n_sqf} square-free, {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main()
