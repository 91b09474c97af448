"""Seeded synthetic workloads for the hard-to-round search.

This module only draws random numbers and fills job descriptors; it holds none
of the method's arithmetic, so both the CUDA library's tests and the CPU oracle
can take their inputs from it.

A job is one slice of one binade of one function (Sect. III-A of the paper:
domain split into sub-domains D_i of equal argument count inside one binade).
Field meanings:

  func    0 = exp, 1 = 2^x, 2 = log
  e_in    arguments lie in the binade [2^(e_in-1), 2^e_in)
  p       precision of the argument/result format (24 toy, 53 binary64)
  m       threshold exponent: a sub-interval is reported iff min < 2^-m
  log2_N  sub-interval length N (the paper's #D_i)
  d       Taylor degree of the block polynomial R_t
  log2_T  Taylor block length (the paper's tau*N), a multiple of N
  limbs   fixed-point word width W = 64*limbs
  start   first argument index j (X = 2^(e_in-1) + j*2^(e_in-p))
  count   number of consecutive arguments
  flags   FLAG_BP_DIRECTED selects scale 2^p instead of 2^(p+1);
          FLAG_ALL_HITS reports every argument below the threshold;
          FLAG_LEFEVRE filters with Lefevre's bound (Algorithm 3);
          FLAG_SOUND reports every argument whose polynomial value is
          within eps3 of a breakpoint (eps1: the filter's half-width)
"""
from __future__ import annotations

import dataclasses
import math
import random
from typing import List

FUNC_EXP, FUNC_EXP2, FUNC_LOG = 0, 1, 2
FUNC_NAMES = {FUNC_EXP: "exp", FUNC_EXP2: "exp2", FUNC_LOG: "log"}

FLAG_BP_DIRECTED = 1
FLAG_ALL_HITS = 2
FLAG_LEFEVRE = 4
FLAG_SOUND = 8


@dataclasses.dataclass(frozen=True)
class Job:
    func: int
    e_in: int
    p: int
    m: int
    log2_N: int
    d: int
    log2_T: int
    limbs: int
    start: int
    count: int
    flags: int = 0
    eps1: int = 0       # sound mode only: filter half-width on the 64-bit words
    eps3: int = 0       # sound mode only: exhaustive-phase half-width

    def replace(self, **kw) -> "Job":
        return dataclasses.replace(self, **kw)


# (func, e_in) choices of the mixed batches: exp on [1/2,1) or [1,2), 2^x on
# [1/2,1) or [1,2), log on [2,4) or [4,8).
MIXED_BINADES = [(FUNC_EXP, 0), (FUNC_EXP, 1), (FUNC_EXP2, 0), (FUNC_EXP2, 1),
                 (FUNC_LOG, 2), (FUNC_LOG, 3)]


def toy_job(m: int = 12, flags: int = 0) -> Job:
    """exp on all 2^23 arguments of a 24-bit format in [1/2,1); d=2 per 2^12
    arguments in 64-bit fixed point; N=2^8."""
    return Job(FUNC_EXP, 0, 24, m, 8, 2, 12, 1, 0, 1 << 23, flags)


def plain_start(seed: int = 1211, count_log2: int = 36) -> int:
    rng = random.Random(seed)
    return rng.randrange(0, (1 << 52) - (1 << count_log2), 1 << 24)


def plain_job(m: int = 40, count_log2: int = 36, seed: int = 1211, flags: int = 0) -> Job:
    """exp on a contiguous slice of 2^36 binary64 arguments in [1/2,1); d=3 per
    2^24 arguments in 192-bit fixed point; N=2^14; seeded block-aligned start."""
    return Job(FUNC_EXP, 0, 53, m, 14, 3, 24, 3, plain_start(seed, count_log2),
               1 << count_log2, flags)


def _block_log2(d: int) -> int:
    return 18 if d == 2 else 24


def batched_jobs(seed: int = 3056, njobs: int = 64, m: int = 40,
                 size_log2_range=(28.0, 34.0)) -> List[Job]:
    """Mixed batch: f and binade uniform over MIXED_BINADES, log-uniform sizes
    2^U (U uniform in the range) rounded to a multiple of N, d in {2,3}, N in
    {2^12, 2^14, 2^16}, 192-bit words, block-aligned uniform start."""
    rng = random.Random(seed)
    jobs = []
    for _ in range(njobs):
        func, e_in = rng.choice(MIXED_BINADES)
        U = rng.uniform(*size_log2_range)
        d = rng.choice((2, 3))
        log2_N = rng.choice((12, 14, 16))
        log2_T = _block_log2(d)
        N = 1 << log2_N
        count = max(N, (int(round(2.0 ** U)) // N) * N)
        span = 1 << 52
        start = rng.randrange(0, span - count - (1 << log2_T), 1 << log2_T)
        jobs.append(Job(func, e_in, 53, m, log2_N, d, log2_T, 3, start, count))
    return jobs


def large_jobs(seed: int = 1211, njobs: int = 1 << 16, total_log2: int = 40,
               log2_N: int = 16, m: int = 42) -> List[Job]:
    """2^x on one contiguous 2^40-argument slice of [1/2,1) split into uneven
    jobs: sizes N*G_j with G_j geometric (mean 2^8), rescaled so that the sizes
    sum to the slice exactly (the last job absorbs the remainder)."""
    rng = random.Random(seed)
    N = 1 << log2_N
    units = 1 << (total_log2 - log2_N)
    g = []
    for _ in range(njobs):
        # geometric with success probability 2^-8, support {1, 2, ...}
        u = 1.0 - rng.random()
        g.append(1 + int(math.log(u) / math.log(1.0 - 2.0 ** -8)))
    scale = units / float(sum(g))
    sizes = [max(1, int(x * scale)) for x in g[:-1]]
    rest = units - sum(sizes)
    while rest < 1:                      # keep every job non-empty
        i = max(range(len(sizes)), key=lambda k: sizes[k])
        sizes[i] -= 1
        rest += 1
    sizes.append(rest)
    start0 = rng.randrange(0, (1 << 52) - (1 << total_log2), 1 << 24)
    jobs, pos = [], start0
    for s in sizes:
        jobs.append(Job(FUNC_EXP2, 0, 53, m, log2_N, 3, 24, 3, pos, s * N))
        pos += s * N
    return jobs


def serving_jobs(seed: int = 2012, njobs: int = 10000,
                 size_log2_range=(20.0, 32.0)) -> List[Job]:
    """Request stream for the serving loop: f and binade as the mixed batch,
    log-uniform sizes, N in {2^12..2^16}, m uniform in [36,44]."""
    rng = random.Random(seed)
    jobs = []
    for _ in range(njobs):
        func, e_in = rng.choice(MIXED_BINADES)
        U = rng.uniform(*size_log2_range)
        d = rng.choice((2, 3))
        log2_N = rng.randint(12, 16)
        m = rng.randint(36, 44)
        log2_T = _block_log2(d)
        N = 1 << log2_N
        count = max(N, (int(round(2.0 ** U)) // N) * N)
        start = rng.randrange(0, (1 << 52) - count - (1 << log2_T), 1 << log2_T)
        jobs.append(Job(func, e_in, 53, m, log2_N, d, log2_T, 3, start, count))
    return jobs


def arrival_times(n: int, rate_per_s: float, seed: int = 2012) -> List[float]:
    """Poisson arrivals: exponential inter-arrival gaps with the given rate."""
    rng = random.Random(seed + 1)
    t, out = 0.0, []
    for _ in range(n):
        t += rng.expovariate(rate_per_s)
        out.append(t)
    return out


def random_search_words(n: int, seed: int, a_bits: int = 64, b_bits: int = 64):
    """Uniform random (B, A) search words, as Python ints, for search-only
    parity cases."""
    rng = random.Random(seed)
    return ([rng.getrandbits(b_bits) for _ in range(n)],
            [rng.getrandbits(a_bits) for _ in range(n)])
