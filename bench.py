#!/usr/bin/env python
"""Benchmark: point evaluations per second of the GPU point count.

Workload (one "step", default --config config4, the largest workload that
fits one GPU): g=3, q in {13, 17, 25, 27}, the full monic degree-7 families
with zero x^6 coefficient (q^6 members each, 6.6e8 in all), counts over F_q,
F_{q^2} and F_{q^3}, exact histograms -- all four jobs in one persistent
launch replayed from a CUDA graph (clear, count, compact).

value  = point evaluations of square-free members per second, device-timed
         (CUDA events on the launch stream, L2 flushed between steps);
e2e    = the same through the public C ABI with host results (descriptor
         upload from pinned memory, launch, histogram copy-back and sort;
         two batches alternate, the host sorting one step's histograms while
         the GPU runs the next);
plain  = the same jobs with one launch per job (no persistent queue, no graph).
At one GPU the line also carries, each with its own device times:
  config3 = the mixed-q workload (g=2, every odd prime power q < 64 plus
            2^24 sampled members over F_293), batched against plain;
  config2 = g=2, q = 31 and 27, batched;
  served  = configuration 2 as Poisson-timed requests through the server
            (p50/p99 latency, results against the batched histograms);
  config5, served_config5 = the genus-4 served workload (q = 7, 9, 11 and
            2^26 draws over F_13), batched, then as requests (the draws cut
            into windows of members);
  table1  = the paper's Table 1 workload: one curve over F_{p^2}, p = 101..3001
            (hwc_curve_count), beside the paper's times.
Under torchrun (N > 1) every job's member range is split across the ranks
(contiguous shards, no collective on the data path) and the shards'
histograms are gathered and merged after the timed region.

--impl reference times the CPU oracle (oracle/) on bounded samples of the
same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_11991_gb300.workloads import CONFIGS, MONIC_NOSUB_SAMPLED, JobSpec, shard_job  # noqa: E402

METRIC = "point evals/s (square-free members x sum_k q^k), batched persistent launch"
UNIT = "evals/s"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hwc", choices=["hwc", "reference"])
    ap.add_argument("--config", default="config4", choices=sorted(CONFIGS))
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the config3 / config2 / served / config5 / table1 extras of the one-GPU line")
    ap.add_argument("--extra-steps", type=int, default=2,
                    help="timed steps of the config3 extra (batched and plain each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default kernel choices; no probe launches): for profiles")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve", action="store_true",
                    help="also run the served form: the workload cut into requests on a Poisson schedule")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="offered load as a fraction of the measured batched throughput")
    return ap.parse_args()


def evals_per_member(spec: JobSpec) -> int:
    return spec.nominal_evals_per_member()


KERNELS = {0: "k_persistent", 1: "k_fan_persistent", 2: "k_fan2_persistent", 3: "k_cls_persistent"}


def chain_reads(spec: JobSpec, lo: int) -> float:
    """Expected Zech reads of the shared Horner chain over c_lo..c_d per
    point: one per nonzero coefficient c_i, lo <= i <= d-1 (c_{d-1} is 0 in
    the families without the subleading term)."""
    d, q = spec.degree, spec.q
    free = d - lo - (1 if spec.kind != 0 else 0)   # positions lo..d-1 that vary
    return free * (q - 1) / q


def _mobius(n: int) -> int:
    r, k, p = 1, n, 2
    while p * p <= k:
        if k % p == 0:
            k //= p
            if k % p == 0:
                return 0
            r = -r
        p += 1
    return -r if k > 1 else r


def points_per_member(spec: JobSpec) -> int:
    """Points x != 0 the kernels evaluate per member: every x in F_q^x, and one
    x per Frobenius orbit of the elements of exact degree m of F_{q^m},
    m = 2..g (as many as monic irreducibles of degree m)."""
    q = spec.q
    pts = q - 1
    for m in range(2, spec.g + 1):
        pts += sum(_mobius(m // d) * q ** d for d in range(1, m + 1) if m % d == 0) // m
    return pts


def table_reads(spec: JobSpec, n_squarefree: int, method: int) -> float:
    """Shared-memory table reads one launch performs for this job (expected
    value over the family; the points of points_per_member):
      0, per-member Horner: one Zech read per nonzero c_i, i <= d-2, per
        point of a square-free member;
      1, fan-out over c_0 (groups of q members): per group and point, the
        chain over c_1..c_d plus one fan-out row;
      2, fan-out over (c_1, c_0) (groups of q^2 members): per group and
        point, the chain over c_2..c_d, one Zech addition per c_1 != 0 and
        one fan-out row per c_1: chain + 2q - 1.  A sampled family on this
        kernel is counted over every group of its family (the samples'
        multiplicities as weights);
      3, sampled members sorted by class (c_2..c_{d-2}): per tile of up to 32
        samples of a class and point, the chain over c_2..c_d, and per
        square-free member and point one Zech read for c_1 != 0 and one for
        c_0 != 0 (tiles: samples / 32 + classes / 2 expected)."""
    d, q = spec.degree, spec.q
    pts = points_per_member(spec)
    if method == 3:
        tiles = spec.n() / 32 + q ** (d - 3) / 2
        return n_squarefree * pts * 2 * (q - 1) / q + tiles * pts * chain_reads(spec, 2)
    if method == 2:
        members = q ** (d - 1) if spec.kind == MONIC_NOSUB_SAMPLED else spec.n()
        return members / q ** 2 * pts * (chain_reads(spec, 2) + 2 * q - 1)
    if method == 1:
        return spec.n() / q * pts * (chain_reads(spec, 1) + 1)
    return n_squarefree * pts * (d - 1) * (q - 1) / q


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and --impl reference)

def oracle_rate(jobs, seconds: float, offset_frac: float = 0.0, threads: int | None = None):
    """Time the oracle on a bounded sample: the same number of members from
    each job, starting at offset_frac of the family; returns
    (evals/s of square-free members, members/s, threads, sample text).
    threads: OpenMP threads (all host cores by default)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    # calibrate on a tiny slice
    probe = 64 * threads
    t0 = time.perf_counter()
    for s in jobs:
        oracle.count_polys(s.g, s.q, s.kind, s.degree, s.first, min(probe, s.n()),
                           seed=s.seed, sample_count=s.sample_count, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-3)
    per = max(64, int(probe * seconds / dt))
    evals = members = 0
    t0 = time.perf_counter()
    for s in jobs:
        n = min(per, s.n())
        first = s.first + int((s.n() - n) * offset_frac)
        _, sqf = oracle.count_polys(s.g, s.q, s.kind, s.degree, first, n, seed=s.seed,
                                    sample_count=s.sample_count, threads=threads)
        evals += int(sqf.sum()) * evals_per_member(s)
        members += n
    dt = time.perf_counter() - t0
    sample = f"{members} members: up to {per} consecutive members of each of the {len(jobs)} jobs"
    return evals / dt, members / dt, threads, sample


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    jobs = CONFIGS[args.config]()
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        oracle_rate(jobs, per_step / 4, offset_frac=(i + 0.5) / (args.warmup + 1))
    rates = []
    curves = []
    threads = sample = None
    step_s = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        r, c, threads, sample = oracle_rate(jobs, per_step, offset_frac=i / max(1, args.steps))
        step_s.append(time.perf_counter() - t0)
        rates.append(r)
        curves.append(c)
    value = statistics.mean(rates)
    r1, _, _, sample1 = oracle_rate(jobs, 4.0, offset_frac=0.5, threads=1)   # the paper's CPU column is 1 core
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.mean(step_s), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (full families, exact decode)",
        "config": {"workload": args.config, "jobs": [j.__dict__ for j in jobs]},
        "curves_per_s": statistics.mean(curves),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"each step: {sample} (a different slice per step)",
                         "value_1core": r1, "sample_1core": sample1},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-i", str(self.gpu),
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[3][1:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


def _strip_comments(text: str) -> str:
    """C/C++ source without comments and blank space (string literals are
    kept as they are; none of the kernel sources puts comment markers in one)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


# the instantiation files of each profiled kernel; the hash follows their
# local #include lines
KERNEL_SOURCES = {"k_fan2_persistent": ["fan2_a.cu", "fan2_b.cu", "fan2_wa.cu", "fan2_wb.cu"]}


def kernel_source_hash(kernel: str = "k_fan2_persistent") -> str:
    """Hash of a count kernel's device sources (its instantiation files and
    every header they include, transitively) with comments and white space
    removed: a traffic figure stays valid across comment-only edits, host-side
    changes and changes to other kernels, and lapses on any change of this
    kernel's code."""
    import re
    src = os.path.join(ROOT, "paper_1805_11991_gb300", "csrc")
    todo = [os.path.join(src, f) for f in KERNEL_SOURCES[kernel]]
    seen = set()
    while todo:
        path = os.path.normpath(todo.pop())
        if path in seen or not os.path.exists(path):
            continue
        seen.add(path)
        with open(path) as fh:
            for inc in re.findall(r'#include\s+"([^"]+)"', fh.read()):
                todo.append(os.path.join(os.path.dirname(path), inc))
    h = hashlib.sha256()
    for path in sorted(seen):
        with open(path) as fh:
            h.update(os.path.relpath(path, ROOT).encode() + b"\0" + _strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per step of the count kernels from the committed ncu summary
    of this workload, if it was taken on the current kernel source."""
    try:
        with open(PROFILE_TRAFFIC) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    w = d.get(workload)
    if not w or w.get("kernel_source_hash") != kernel_source_hash():
        return None
    return w.get("dram_bytes_per_step")


# ---------------------------------------------------------------------------
# served form

def serve_leg(hwc, jobs, batched_results, batched_evals_per_s, n_requests, load, seed=11):
    """The workload as a stream of requests: every job cut into slices of about
    equal evaluation work, shuffled (seed), submitted at Poisson arrival times
    (seed) whose mean rate offers `load` times the batched throughput.  Returns
    throughput, p50/p99 latency (submit -> result) and whether every job's
    merged slices equal its batched histogram."""
    import numpy as np
    from paper_1805_11991_gb300.workloads import poisson_arrivals, split_job
    work = [s.n() * evals_per_member(s) for s in jobs]
    target = sum(work) / n_requests
    reqs = []
    for j, (spec, w) in enumerate(zip(jobs, work)):
        reqs += [(j, r) for r in split_job(spec, max(1, round(w / target)))]
    order = np.random.default_rng(seed).permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    # a window of a densely drawn sample counts the draws landing in it
    req_evals = [r.drawn() * evals_per_member(r) for _, r in reqs]
    mean_service_s = (sum(req_evals) / len(reqs)) / batched_evals_per_s
    arrivals = poisson_arrivals(len(reqs), load / mean_service_s, seed=seed)
    srv = hwc.Server()
    tickets, submitted = [], []
    t0 = time.perf_counter()
    for (j, r), t_arr in zip(reqs, arrivals):
        delay = t0 + float(t_arr) - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        submitted.append(time.perf_counter())
        tickets.append(srv.submit(hwc.make_job(r.g, r.q, r.kind, r.degree, r.first, r.n(), r.seed,
                                               r.sample_count)))
    hists = []
    for t in tickets:
        h = None
        while h is None:
            h = srv.poll(t, 1000)
        hists.append(h)
    total_ms = [srv.latency(t)[1] / 1e3 for t in tickets]    # submit -> done, from the server's clock
    srv.close()
    # wall time: first submission to the last request done (host-side merging excluded)
    t_end = max(sub + ms / 1e3 for sub, ms in zip(submitted, total_ms))
    sqf = sum(h.n_squarefree * evals_per_member(r) for h, (_, r) in zip(hists, reqs))
    lat = sorted(total_ms)
    merged = [None] * len(jobs)
    for h, (j, _) in zip(hists, reqs):
        merged[j] = h if merged[j] is None else hwc.hist_merge(merged[j], h)
    same = all(m is not None and np.array_equal(m.counts, b.counts) and np.array_equal(m.mult, b.mult)
               for m, b in zip(merged, batched_results))
    p = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
    return {"value": sqf / (t_end - t0), "unit": UNIT, "requests": len(reqs),
            "arrival_rate_per_s": load / mean_service_s, "offered_load": load,
            "p50_ms": p(0.50), "p99_ms": p(0.99), "max_ms": lat[-1], "wall_s": t_end - t0,
            "arrivals": "Poisson, seed %d; requests: every job cut into slices of equal work (a densely drawn "
                        "sample into windows of members with the draws landing in them), shuffled" % seed,
            "matches_batched": bool(same)}


# ---------------------------------------------------------------------------
# GPU arm

def _hjobs(hwc, jobs):
    return [hwc.make_job(s.g, s.q, s.kind, s.degree, s.first, s.n(), s.seed, s.sample_count) for s in jobs]


def _timed(batch, k, stream, flush):
    """k steps of `batch`, each timed by CUDA events on `stream` with an L2
    flush (outside the events) before it; returns (total ms, count-kernel ms
    per step)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    kms = []
    for a, b in ev:
        with torch.cuda.stream(stream):
            flush.zero_()                    # L2 flush, outside the timed events
        a.record(stream)
        batch.launch(stream)
        b.record(stream)
        kms.append(batch.kernel_ms())       # waits for this step
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev), kms


def _workload_units(batch, jobs):
    """(square-free evaluations, members, table reads, kernels, results) of one
    run of a batch whose last launch has finished."""
    results = [batch.result(i) for i in range(len(jobs))]
    sqf = [h.n_squarefree for h in results]
    methods = [batch.job_method(i) for i in range(len(jobs))]
    units = sum(n * evals_per_member(s) for n, s in zip(sqf, jobs))
    members = sum(s.n() for s in jobs)
    reads = sum(table_reads(s, n, m) for n, s, m in zip(sqf, jobs, methods))
    kernels = sorted({KERNELS[m] for m in methods})
    return units, members, reads, kernels, results


def extra_workload(hwc, name, steps, warmup, stream, flush, plain=True):
    """One more workload on this GPU, batched (graph) and optionally plain,
    with its own device times; returns (summary dict, batched results)."""
    jobs = CONFIGS[name]()
    hj = _hjobs(hwc, jobs)
    batched = hwc.Batch(hj, flags=hwc.FLAG_GRAPH | hwc.FLAG_TIMING)
    pl = hwc.Batch(hj, flags=hwc.FLAG_PLAIN | hwc.FLAG_TIMING) if plain else None
    for _ in range(warmup):
        batched.launch(stream)
        if pl:
            pl.launch(stream)
    import torch
    torch.cuda.synchronize()
    units, members, reads, kernels, results = _workload_units(batched, jobs)
    ms, kms = _timed(batched, steps, stream, flush)
    out = {"jobs": len(jobs), "members": members, "steps": steps, "warmup": warmup,
           "batched": {"value": units * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                       "kernel_ms": statistics.mean(kms), "curves_per_s": members * steps / (ms * 1e-3),
                       "launches_per_step": batched.kernel_launches(),
                       "table_reads_per_s": reads / (statistics.mean(kms) * 1e-3), "kernels": kernels}}
    if pl:
        pms, pkms = _timed(pl, steps, stream, flush)
        out["plain"] = {"value": units * steps / (pms * 1e-3), "unit": UNIT, "ms_per_step": pms / steps,
                        "kernel_ms": statistics.mean(pkms), "launches_per_step": pl.kernel_launches()}
        out["batched_over_plain"] = out["batched"]["value"] / out["plain"]["value"]
        pl.close()
    batched.close()
    return out, jobs, results


# Sec. 4, Table 1: the curve y^2 = 12x^6 + 13x^5 + 10x^4 + 11x^3 + 16x^2 + 12x + 17
# over F_{p^2}; the paper's times (ms) on a Tesla K80 and one Xeon E5-2683 core:
# (p, tables, CPU, GPU eval, GPU reduce)
TABLE1 = [(101, 4.70, 0.63, 0.36, 0.10), (211, 23.8, 4.47, 1.47, 0.15), (307, 54.9, 12.1, 3.11, 0.22),
          (401, 99.2, 22.2, 0.95, 0.35), (503, 167, 36.3, 1.25, 0.83), (1009, 892, 148, 2.93, 6.49),
          (1511, 2545, 349, 394, 19.7), (2003, 5093, 789, 11.5, 36.1), (3001, 13474, 3669, 15.4, 82.6)]
TABLE1_CURVE = [17, 12, 16, 11, 10, 13, 12]   # c_0..c_6


def table1_leg(hwc, reps=5):
    """The paper's only timed workload: one curve over F_{p^2} per p of Table 1,
    through hwc_curve_count (tables built on the first call, then cached).
    Reports the table build (wall clock of the first call minus its count),
    the count's device time (best of `reps`, CUDA events) and evals/s = p^2 / t,
    beside the paper's K80 times (context: other hardware, one curve)."""
    import numpy as np
    c = np.array([TABLE1_CURVE])
    hwc.curve_count(3, 2, np.array([[1, 0, 0, 0, 0, 0, 1]]))   # load the kernels
    rows = []
    for p, tab, cpu, ev, red in TABLE1:
        t0 = time.perf_counter()
        cnt, ms0 = hwc.curve_count(p, 2, c)
        first_ms = 1e3 * (time.perf_counter() - t0)
        best = min(hwc.curve_count(p, 2, c)[1] for _ in range(reps))
        rows.append({"p": p, "count": int(cnt[0]), "tables_ms": max(0.0, first_ms - ms0), "count_ms": best,
                     "evals_per_s": p * p / (best * 1e-3), "paper_tables_ms": tab, "paper_cpu_ms": cpu,
                     "paper_gpu_eval_reduce_ms": ev + red,
                     "vs_paper_gpu": (ev + red) / best})
    return rows


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_1805_11991_gb300 import hwc, shard

    full_jobs = CONFIGS[args.config]()
    # each rank takes a contiguous shard of every job's member range (a
    # densely drawn sample: a window of its family with the draws in it)
    jobs = full_jobs if world == 1 else [shard_job(s, rank, world) for s in full_jobs]
    hjobs = _hjobs(hwc, jobs)
    tune = hwc.FLAG_NO_TUNE if args.no_tune else 0
    batched = hwc.Batch(hjobs, flags=hwc.FLAG_GRAPH | hwc.FLAG_TIMING | tune)
    plain = hwc.Batch(hjobs, flags=hwc.FLAG_PLAIN | hwc.FLAG_TIMING | tune)
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (also fixes the square-free counts used as units)
    for _ in range(max(args.warmup, 3)):
        batched.launch(stream)
        plain.launch(stream)
    torch.cuda.synchronize()
    units, members, lookups, kernels, results = _workload_units(batched, jobs)

    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        total_ms, kernel_ms = _timed(batched, args.steps, stream, flush)
    torch.cuda.synchronize()
    barrier()
    plain_ms, plain_kms = _timed(plain, args.steps, stream, flush)

    # e2e through the public API: every step uploads its descriptors, launches,
    # copies every job's histogram back and sorts it on the host.  Two batches
    # of the same jobs alternate, so that the host reads one step's histograms
    # while the GPU runs the next.
    e2e_steps = max(3, args.steps // 2)
    other = hwc.Batch(hjobs, flags=hwc.FLAG_GRAPH | tune)
    other.launch(stream)
    for i in range(len(jobs)):
        other.result(i)
    pair = (batched, other)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    pair[0].launch(stream)
    for step in range(e2e_steps):
        if step + 1 < e2e_steps:
            pair[(step + 1) % 2].launch(stream)   # queued behind this step
        cur = pair[step % 2]
        for i in range(len(jobs)):
            cur.result(i)
    e2e_s = time.perf_counter() - t0
    h2d, d2h = batched.io_bytes()
    other.close()

    all_units, all_members = units, members
    if dist is not None:
        t = torch.tensor([total_ms, plain_ms, e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, plain_ms, e2e_s = (float(v) for v in t.tolist())
        u = torch.tensor([units, members], device="cuda", dtype=torch.float64)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        all_units, all_members = (float(v) for v in u.tolist())

    # roofline of the dominant kernel (the persistent count kernel)
    kern_ms = statistics.mean(kernel_ms)
    achieved = lookups / (kern_ms * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(local_rank)
    sms = props.multi_processor_count
    sm_max = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            sm_max = json.load(fh).get("sm_max_mhz")
    except (OSError, ValueError):
        pass
    sm_max = sm_max or 2070.0
    peak = sms * sm_max * 1e6 * 32 / 1e9          # one 32-lane LDS wavefront per SM per clock
    table_entries = 2 * (27 ** 3 - 1) + 1 if args.config == "config4" else 2 * (31 ** 2 - 1) + 1
    measured = hwc.probe_smem_gather(table_entries, 4096) / 1e9
    traffic = profiled_traffic(args.config)

    value = all_units * args.steps / (total_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic: full coefficient families decoded on the device",
        "config": {"workload": args.config,
                   "jobs": [f"g{s.g} q{s.q} d{s.degree} members {s.n()}" for s in full_jobs],
                   "members": int(all_members), "squarefree_evals_per_step": int(all_units),
                   "l2": "flushed (512 MiB write) between steps",
                   "launch": "persistent kernel in a CUDA graph",
                   "sharding": f"each job's members split into {world} contiguous shards" if world > 1 else None},
        "curves_per_s": all_members * args.steps / (total_ms * 1e-3),
        "plain": {"value": all_units * args.steps / (plain_ms * 1e-3), "unit": UNIT,
                  "ms_per_step": plain_ms / args.steps, "launches_per_step": plain.kernel_launches()},
        "e2e": {"value": all_units * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * batched.kernel_launches(),
        "roofline": {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "Glookup/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "+".join(kernels),
                     "kernel_ms": kern_ms, "table_reads_per_step": lookups,
                     "peak_source": f"{sms} SMs x {sm_max:.0f} MHz x 32 lanes (bank-conflict-free LDS)",
                     "measured_random_gather": measured,
                     "frac_of_measured_random_gather": achieved / measured},
    }
    if world > 1:
        # merge every job's shards (after the timed region) and check them against
        # one GPU counting the whole job
        merged = [shard.gather_merge(h) for h in results]
        if rank == 0:
            single = hwc.Batch(_hjobs(hwc, full_jobs), flags=hwc.FLAG_GRAPH)
            single.launch(stream)
            torch.cuda.synchronize()
            same = True
            for i, m in enumerate(merged):
                h = single.result(i)
                same &= (m.counts.shape == h.counts.shape and bool((m.counts == h.counts).all())
                         and bool((m.mult == h.mult).all()) and m.n_total == h.n_total)
            single.close()
            line["shards_match_single_gpu"] = bool(same)
    if rank == 0 and world == 1 and not args.no_extras:
        ew = max(1, min(args.warmup, 3))
        line["config3"], _, _ = extra_workload(hwc, "config3", args.extra_steps, ew, stream, flush)
        c2, c2_jobs, c2_results = extra_workload(hwc, "config2", args.steps, ew, stream, flush, plain=False)
        line["config2"] = c2
        line["served"] = serve_leg(hwc, c2_jobs, c2_results, c2["batched"]["value"], args.serve_requests,
                                   args.serve_load)
        line["served"]["workload"] = "config2"
        if args.config != "config5":   # the genus-4 served workload: batched, then as requests
            c5, c5_jobs, c5_results = extra_workload(hwc, "config5", args.extra_steps, ew, stream, flush,
                                                     plain=False)
            line["config5"] = c5
            line["served_config5"] = serve_leg(hwc, c5_jobs, c5_results, c5["batched"]["value"],
                                               args.serve_requests, args.serve_load)
            line["served_config5"]["workload"] = "config5"
        line["table1"] = table1_leg(hwc)
    if args.serve and rank == 0 and world == 1:
        line["served_" + args.config] = serve_leg(hwc, jobs, results, value, args.serve_requests, args.serve_load)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, c, threads, sample = oracle_rate(jobs, args.cpu_seconds)
        r1, _, _, sample1 = oracle_rate(jobs, 4.0, offset_frac=0.5, threads=1)   # the paper's CPU column is 1 core
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": sample, "curves_per_s": c, "value_1core": r1, "sample_1core": sample1}
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)
    batched.close()
    plain.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
