"""Sound mode: rigorous error bounds, the exhaustive phase's candidate list,
and the exact re-check of a candidate.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

Sect. II-A tests the degree-1 approximation of each sub-domain against
eps'' = eps + eps_approx + eps_trunc instead of eps, so that no hard-to-round
argument of the function can slip through the filter; Sect. III-A's phase 3
then evaluates the polynomial at every argument of the sub-domains that fail.
Here, on the 64-bit words (units of 2^-64 of the breakpoint spacing):

  eps_approx  |R_t(y) / 2^W - s f(X_t + y u)|, any argument of the job:
              the Taylor remainder of degree d over a block of T arguments,
              s (u T)^(d+1) max|f^(d+1)| / (d+1)!, plus the rounding of the
              d+1 coefficients to 2^-W (half a unit times y^k each);
  eps_trunc   |R_t(iN + x) - (b_i + alpha_i x)| / 2^W, x < N: the terms of
              degree >= 2 of the binomial-basis expansion
              R_t(iN + x) = sum_j r_j(i) binom(x, j)  (Sect. IV-A), with
              |r_j(i)| <= max |R_t^(j)| on the block (mean value theorem for
              differences) and |c_k| <= 2^W s u^k max|f^(k)| / k! + 1/2.

The thresholds of a sound job, in units of 2^-64:

  eps3 >= 2^(64-m) + ceil(eps_approx 2^64) + 1     (every argument with
          |s f(X) cmod 1| < 2^-m has top64(R_t(y)) cmod 2^64 in [-eps3, eps3))
  eps1 >= eps3 + ceil(eps_trunc 2^64) + N + 2       (every sub-interval holding
          such an argument has a 64-bit line within [-eps1, eps1): the two
          64-bit words lose at most one unit each, the slope's unit over
          up to N - 1 steps)
  eps2 >= eps3 + ceil(eps_trunc(N/32) 2^64) + N/32 + 2  (the same for the 32
          pieces of a failing sub-interval, each with its own line: the
          paper's phase 2; min_eps_len gives it for any line length)

sound_candidates() is the definition of what the sound path reports: every
argument whose polynomial value R_t(y), evaluated by direct Horner, has
(top64(R_t(y)) + eps3) mod 2^64 < 2 eps3 -- independent of the filter.
is_hard_to_round() decides Def. 3 exactly from an enclosure of f.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb
from typing import List, Tuple

from . import fmath, plan, poly

M64 = 1 << 64


def _ceil(v: Fraction) -> int:
    return -((-v.numerator) // v.denominator)


def _deriv_max(job, k: int) -> Fraction:
    """An upper bound of |f^(k)| over the job's arguments (k >= 1 for log)."""
    x_lo = plan.argument(job, job.start)
    x_hi = plan.argument(job, job.start + job.count - 1)
    if job.func == fmath.FUNC_EXP:
        return fmath.exp_interval(x_hi, 64)[1]
    if job.func == fmath.FUNC_EXP2:
        e_hi = fmath.exp2_interval(x_hi, 64)[1]
        l_hi = fmath.ln2_interval(64)[1]
        return e_hi * l_hi ** k
    if job.func == fmath.FUNC_LOG:
        if k == 0:
            return fmath.log_interval(x_hi, 64)[1]
        return Fraction(fmath._factorial(k - 1)) / x_lo ** k
    raise ValueError("unknown function")


def _scale_max(job) -> Fraction:
    """The largest breakpoint scale s over the job (smallest output exponent)."""
    e_min = min(e for (_, _, e) in plan.segments(job))
    return fmath._pow2(plan.scale_log2(job, e_min))


def eps_approx(job) -> Fraction:
    """Bound of |R_t(y)/2^W - s f(X)| over every argument of the job."""
    d, W = job.d, 64 * job.limbs
    T = Fraction(1 << job.log2_T)
    u = fmath._pow2(job.e_in - job.p)
    s = _scale_max(job)
    rem = s * (u * T) ** (d + 1) * _deriv_max(job, d + 1) / fmath._factorial(d + 1)
    rnd = sum(Fraction(1, 2) * T ** k for k in range(d + 1)) / fmath._pow2(W)
    return rem + rnd


def eps_trunc(job, length: int = 0) -> Fraction:
    """Bound of |R_t(y0 + x) - (R_t(y0) + (R_t(y0 + 1) - R_t(y0)) x)| / 2^W
    over x < length (default N: the sub-interval lines of the filter)."""
    d, W = job.d, 64 * job.limbs
    N = length or (1 << job.log2_N)
    T = Fraction((1 << job.log2_T) + d)
    u = fmath._pow2(job.e_in - job.p)
    s = _scale_max(job)
    two_w = fmath._pow2(W)
    cbound = [two_w * s * u ** k * _deriv_max(job, k) / fmath._factorial(k) + Fraction(1, 2)
              for k in range(d + 1)]
    total = Fraction(0)
    for j in range(2, d + 1):
        rj = sum(cbound[k] * Fraction(fmath._factorial(k), fmath._factorial(k - j)) * T ** (k - j)
                 for k in range(j, d + 1))
        total += rj * comb(N - 1, j)
    return total / two_w


def min_eps(job) -> Tuple[int, int]:
    """The smallest sound (eps1, eps3) in units of 2^-64."""
    eps3 = (1 << (64 - job.m)) + _ceil(eps_approx(job) * M64) + 1
    eps1 = eps3 + _ceil(eps_trunc(job) * M64) + (1 << job.log2_N) + 2
    return eps1, eps3


def piece_length(job) -> int:
    """Arguments of a phase-2 piece: a sub-interval is cut into 32 pieces."""
    N = 1 << job.log2_N
    return (N + 31) // 32


def min_eps_len(job, eps3: int, length: int) -> int:
    """The smallest sound half-width for lines of `length` consecutive
    arguments (a stretch holding an argument within eps3 has its 64-bit line
    within this half-width): eps3 + eps_trunc(length) + length + 2."""
    return eps3 + _ceil(eps_trunc(job, length) * M64) + length + 2


def min_eps2(job, eps3: int) -> int:
    """The smallest sound phase-2 half-width, for pieces of piece_length()
    arguments."""
    return min_eps_len(job, eps3, piece_length(job))


def sound_candidates(jobs, eps3s) -> List[Tuple[int, int, int, int]]:
    """(job index, sub-interval, argument index, v) for every argument of
    every job with v = (top64(R_t(y)) + eps3) mod 2^64 < 2 eps3, sorted by
    (job, argument).  R_t by direct Horner (poly.horner)."""
    out = []
    for ji, (job, eps3) in enumerate(zip(jobs, eps3s)):
        W = 64 * job.limbs
        N = 1 << job.log2_N
        for blk in plan.blocks(job):
            c = poly.taylor_coeffs(job, blk)
            for y in range(blk.length):
                top = poly.horner(c, y, W) >> (W - 64)
                v = (top + eps3) % M64
                if v < 2 * eps3:
                    out.append((ji, blk.first_sub + y // N, blk.start + y, v))
    out.sort(key=lambda r: (r[0], r[2]))
    return out


def distance(job, j: int, bits: int = 0) -> Tuple[Fraction, Fraction]:
    """Enclosure of |s f(X_j) cmod 1| (Def. 2 on the job's scale)."""
    X = plan.argument(job, j)
    e_out = fmath.exponent_of(job.func, X)
    s = fmath._pow2(plan.scale_log2(job, e_out))
    bits = bits or job.p + job.m + 24
    while True:
        lo, hi = fmath.f_interval(job.func, X, bits)
        a, b = lo * s, hi * s
        fa = a - (a.numerator // a.denominator)
        n = a.numerator // a.denominator
        if b < n + 1:  # both ends in the same unit interval
            fb = b - n
            da = min(fa, 1 - fa)
            db = min(fb, 1 - fb)
            if (fa <= Fraction(1, 2)) == (fb <= Fraction(1, 2)):
                return (min(da, db), max(da, db))
        bits += 64
        if bits > 4096:
            raise ArithmeticError("distance undecided")


def is_hard_to_round(job, j: int) -> bool:
    """Def. 3: dist(s f(X_j)) < 2^-m, decided exactly (the enclosure is
    refined until it lies on one side of 2^-m)."""
    eps = fmath._pow2(-job.m)
    bits = job.p + job.m + 24
    while True:
        lo, hi = distance(job, j, bits)
        if hi < eps:
            return True
        if lo >= eps:
            return False
        bits += 64
        if bits > 4096:
            raise ArithmeticError("hard-to-round decision undecided")
