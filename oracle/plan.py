"""Job planning: output-binade segments, Taylor blocks and sub-intervals.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

Sect. III-A splits the domain into sub-domains D_i of equal argument count
with one exponent each, and changes variable to the integer x = 2^(p-e(X_i))
(X - X_i).  Sect. IV groups tau consecutive sub-domains into one Taylor block
D_t with one polynomial R_t.  The argument X with index j in the binade
[2^(e_in-1), 2^e_in) is  X_j = (2^(p-1) + j) 2^(e_in-p).

The scaled value whose distance to the breakpoints is searched is
s f(X) with s = 2^(p+1-e_out) (floats and midpoints: the round-to-nearest
(p, eps) cases are the directed (p+1, 2 eps) cases, Sect. II-A) or
s = 2^(p-e_out) with the directed-only flag, e_out = e(f(X)) (Def. 1).  s
must be constant on a block, so the slice is first cut where e(f(X))
changes.  The plan, in order:

  segments  maximal runs of arguments with one e_out; a cut is the first
            argument j with e(f(X_j)) larger than before, found here by
            bisection on the (increasing) function itself;
  blocks    each segment is cut into blocks of T arguments from its first
            argument (the last block may be shorter);
  sub-intervals
            each block is cut into sub-intervals of N arguments from its
            first argument (the last may be shorter).

Sub-intervals are numbered 0, 1, ... over the whole job in this order.
"""
from __future__ import annotations

import dataclasses
from fractions import Fraction
from typing import List

from . import fmath

FLAG_BP_DIRECTED = 1
FLAG_ALL_HITS = 2


def argument(job, j: int) -> Fraction:
    """X_j = (2^(p-1) + j) * 2^(e_in - p)."""
    num = (1 << (job.p - 1)) + j
    sh = job.e_in - job.p
    return Fraction(num << sh) if sh >= 0 else Fraction(num, 1 << -sh)


def e_out_at(job, j: int) -> int:
    return fmath.exponent_of(job.func, argument(job, j))


@dataclasses.dataclass(frozen=True)
class Block:
    start: int        # argument index j of the block's first argument
    length: int       # number of arguments
    e_out: int        # output exponent on the block
    first_sub: int    # job-wide index of the block's first sub-interval


def segments(job) -> List[tuple]:
    """[(j0, j1, e_out)] with e(f(X_j)) = e_out for j0 <= j < j1."""
    lo_j, hi_j = job.start, job.start + job.count
    e0 = e_out_at(job, lo_j)
    e1 = e_out_at(job, hi_j - 1)
    cuts = [lo_j]
    exps = [e0]
    for e in range(e0 + 1, e1 + 1):
        # first j in [cuts[-1], hi_j) with e_out(j) >= e (bisection)
        a, b = cuts[-1], hi_j - 1
        while a < b:
            mid = (a + b) // 2
            if e_out_at(job, mid) >= e:
                b = mid
            else:
                a = mid + 1
        if e_out_at(job, a) == e:
            cuts.append(a)
            exps.append(e)
        # an exponent that is skipped entirely would need an argument where
        # f jumps by a factor 2: impossible for the slices used here
    out = []
    for i, (c, e) in enumerate(zip(cuts, exps)):
        end = cuts[i + 1] if i + 1 < len(cuts) else hi_j
        if end > c:
            out.append((c, end, e))
    return out


def blocks(job) -> List[Block]:
    T = 1 << job.log2_T
    N = 1 << job.log2_N
    out = []
    sub = 0
    for j0, j1, e in segments(job):
        b = j0
        while b < j1:
            length = min(T, j1 - b)
            out.append(Block(b, length, e, sub))
            sub += (length + N - 1) // N
            b += length
    return out


def n_subintervals(job) -> int:
    bl = blocks(job)
    N = 1 << job.log2_N
    return sum((b.length + N - 1) // N for b in bl)


def scale_log2(job, e_out: int) -> int:
    """log2 of the breakpoint scale s."""
    if job.flags & FLAG_BP_DIRECTED:
        return job.p - e_out
    return job.p + 1 - e_out
