"""Seeded synthetic workloads: the five benchmark configurations.

Job lists only (family, index range, sampling seed) and the Poisson arrival
schedule of the served configuration.  Nothing here computes any part of the
point count; the GPU library and the oracle each decode these descriptions on
their own.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ALL_DEG, MONIC_NOSUB, MONIC_NOSUB_SAMPLED = 0, 1, 2
MONIC_NOSUB_SAMPLED_WINDOW = 4   # the draws of a sampled family in a window of members

# odd prime powers below 64
ODD_PRIME_POWERS_BELOW_64 = [3, 5, 7, 9, 11, 13, 17, 19, 23, 25, 27, 29, 31, 37, 41, 43, 47, 49,
                             53, 59, 61]


@dataclass(frozen=True)
class JobSpec:
    g: int
    q: int
    kind: int
    degree: int
    first: int = 0
    count: int = -1          # -1: the whole family
    seed: int = 0
    sample_count: int = 0

    def family_members(self) -> int:
        if self.kind == ALL_DEG:
            return (self.q - 1) * self.q ** self.degree
        if self.kind in (MONIC_NOSUB, MONIC_NOSUB_SAMPLED_WINDOW):
            return self.q ** (self.degree - 1)
        return self.sample_count

    def n(self) -> int:
        return self.family_members() - self.first if self.count < 0 else self.count

    def drawn(self) -> float:
        """Members the job counts: the range, or for a window of a sampled
        family the expected number of draws landing in it."""
        if self.kind == MONIC_NOSUB_SAMPLED_WINDOW:
            return self.sample_count * self.n() / self.family_members()
        return float(self.n())

    def whole_family_draws(self) -> bool:
        """A sampled family drawn densely enough for the whole-family kernel
        (q <= 31, at least one draw per 32 members, fewer than 2^27 draws)."""
        fam = self.q ** (self.degree - 1)
        return (self.kind == MONIC_NOSUB_SAMPLED and self.q <= 31 and self.sample_count < (1 << 27)
                and 32 * self.n() >= fam)

    def nominal_evals_per_member(self) -> int:
        """Points x in F_{q^k}, k = 1..g, each member is evaluated at."""
        return sum(self.q ** k for k in range(1, self.g + 1))

    def with_range(self, first: int, count: int) -> "JobSpec":
        return JobSpec(self.g, self.q, self.kind, self.degree, first, count, self.seed, self.sample_count)


def config1():
    """g=2, q=3: every f of exact degree 5 or 6 (486 + 1458 members)."""
    return [JobSpec(2, 3, ALL_DEG, 5), JobSpec(2, 3, ALL_DEG, 6)]


def config2():
    """g=2, q=31 and q=27: full monic degree-5 and -6 families with c_{d-1}=0."""
    return [JobSpec(2, q, MONIC_NOSUB, d) for q in (31, 27) for d in (5, 6)]


def config3():
    """g=2, every odd prime power q<64 (full monic degree-5, c_4=0) plus q=293
    with 2^24 members drawn by seed 7."""
    jobs = [JobSpec(2, q, MONIC_NOSUB, 5) for q in ODD_PRIME_POWERS_BELOW_64]
    jobs.append(JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, seed=7, sample_count=1 << 24))
    return jobs


def config4():
    """g=3, q in {13, 17, 25, 27}: full monic degree-7 families with c_6=0."""
    return [JobSpec(3, q, MONIC_NOSUB, 7) for q in (13, 17, 25, 27)]


def config5():
    """g=4 served: full monic degree-9 (c_8=0) families for q in {7, 9, 11} and
    q=13 with 2^26 members drawn by seed 11."""
    jobs = [JobSpec(4, q, MONIC_NOSUB, 9) for q in (7, 9, 11)]
    jobs.append(JobSpec(4, 13, MONIC_NOSUB_SAMPLED, 9, seed=11, sample_count=1 << 26))
    return jobs


def config2_q31d5():
    """One job of config 2 (q=31, degree 5, 31^4 members): the small case used
    for detailed profiles of the count kernel."""
    return [JobSpec(2, 31, MONIC_NOSUB, 5)]


def config2_q31d6():
    """The largest job of config 2 (q=31, degree 6, 31^5 members, 29,791 groups
    of q^2 members): the small case used for profiles of the two-level kernel."""
    return [JobSpec(2, 31, MONIC_NOSUB, 6)]


def config4_q27_slice():
    """2^21 members from the middle of the g=3 q=27 degree-7 job of
    configuration 4 (2,877 groups of q^2 members): the small case used for
    detailed profiles of the two-level kernel."""
    return [JobSpec(3, 27, MONIC_NOSUB, 7, 27 ** 6 // 2, 1 << 21)]


def config3_q293_slice():
    """2^18 of the 2^24 sampled members of the q=293 job of configuration 3:
    the small case used for profiles of the per-member kernel (17-bit Zech
    table of F_{293^2} in shared memory)."""
    return [JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 1 << 18, seed=7, sample_count=1 << 24)]


def config3_q293_cls_slice():
    """The first 2^21 of the 2^24 sampled members of the q=293 job of
    configuration 3 (about 24 samples per class of (c_2, c_3)): the small case
    used for profiles of the class-sharing kernel."""
    return [JobSpec(2, 293, MONIC_NOSUB_SAMPLED, 5, 0, 1 << 21, seed=7, sample_count=1 << 24)]


def config5_q13_slice():
    """2^20 members from the middle of the full g=4 q=13 degree-9 family (6,205
    groups of q^2 members): the small case used for profiles of the two-level
    kernel with the int16 rows of F_{13^4} (the same code as the weighted run
    of configuration 5's q=13 job, without the weights)."""
    return [JobSpec(4, 13, MONIC_NOSUB, 9, 13 ** 8 // 2, 1 << 20)]


CONFIGS = {"config1": config1, "config2": config2, "config3": config3, "config4": config4,
           "config5": config5, "config2_q31d5": config2_q31d5, "config2_q31d6": config2_q31d6,
           "config4_q27_slice": config4_q27_slice, "config3_q293_slice": config3_q293_slice,
           "config5_q13_slice": config5_q13_slice, "config3_q293_cls_slice": config3_q293_cls_slice}


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 11) -> np.ndarray:
    """Arrival times (s) of n requests of a Poisson process (exponential gaps)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def _cut_by_windows(job: JobSpec) -> bool:
    """A whole densely drawn sample: cut it into windows of the enumerated
    family, each with the draws that land in it (their union is the whole
    sample), not into slices of the draws, which would each be too sparse
    for the whole-family kernel."""
    return job.whole_family_draws() and job.first == 0 and job.n() == job.sample_count


def _part(job: JobSpec, i: int, parts: int) -> JobSpec:
    """Part i of `parts` of a job: a contiguous slice of its range, or a
    window of its family (see _cut_by_windows)."""
    if _cut_by_windows(job):
        fam = job.q ** (job.degree - 1)
        a, b = (fam * i) // parts, (fam * (i + 1)) // parts
        return JobSpec(job.g, job.q, MONIC_NOSUB_SAMPLED_WINDOW, job.degree, a, b - a, job.seed, job.sample_count)
    n = job.n()
    a = job.first + (n * i) // parts
    b = job.first + (n * (i + 1)) // parts
    return job.with_range(a, b - a)


def shard_job(job: JobSpec, rank: int, world: int) -> JobSpec:
    """This rank's share of a job when every rank counts one part on its own
    GPU (possibly empty)."""
    return _part(job, rank, world)


def split_job(job: JobSpec, parts: int):
    """Cut a job into `parts` pieces of about equal work (serving requests):
    contiguous slices of its member range, or windows of a densely drawn
    sample's family; empty pieces are left out."""
    out = []
    if _cut_by_windows(job):
        for i in range(parts):
            w = _part(job, i, parts)
            if w.n() > 0:
                out.append(w)
        return out
    n = job.n()
    for i in range(parts):
        a = job.first + (n * i) // parts
        b = job.first + (n * (i + 1)) // parts
        if b > a:
            out.append(job.with_range(a, b - a))
    return out
