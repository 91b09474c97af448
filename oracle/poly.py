"""Block polynomials, their degree-1 truncations and the search words.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

All quantities are W-bit integers that stand for fractions in units of 2^-W
(the integer part of s f is dropped: only (b + a x) mod 1 matters because x
is an integer).

Taylor coefficients of the block starting at X_t, in the integer variable
y = 2^(p - e_in)(X - X_t) (Sect. III-A change of variable, Sect. IV Taylor
polynomial R_t):

    c_k = RN(2^W s u^k f^(k)(X_t)/k!) mod 2^W,     u = 2^(e_in - p),

    R_t(y) = sum_k c_k y^k  mod 2^W.

The sub-interval i of the block covers y = iN + x, 0 <= x < N_i.  Its
degree-1 approximation in the binomial basis (Sect. IV-A hierarchical
method: R_t(x + iN) = sum_j r_{t,j}(i) binom(x, j) with
r_{t,j}(i) = Delta^j[R_t](iN)) keeps the j = 0, 1 terms:

    b_i     = r_{t,0}(i) = R_t(iN)
    alpha_i = r_{t,1}(i) = R_t(iN + 1) - R_t(iN)

so that the line is b_i + alpha_i x (mod 2^W).  Here they are evaluated by
direct Horner at every sub-interval, never by stepping differences.

Search words (the one-sided test of Sect. II-A, {y + eps} < 2 eps, with
eps = 2^-m, on the paper's form b - a x of Eq. (1)):

    B = floor(((b_i + 2^(W-m)) mod 2^W) / 2^(W-64))
    A = floor(((-alpha_i) mod 2^W) / 2^(W-64))
    T_m = 2^(65-m)

and the sub-interval is a candidate iff min_{0<=x<N_i} (B - A x) mod 2^64
is below T_m.
"""
from __future__ import annotations

from typing import List, Tuple

from . import fmath
from .plan import argument, scale_log2


def taylor_coeffs(job, block) -> List[int]:
    """[c_0, ..., c_d] for the block (each reduced mod 2^W)."""
    W = 64 * job.limbs
    X_t = argument(job, block.start)
    s_log2 = scale_log2(job, block.e_out)
    mask = (1 << W) - 1
    out = []
    for k in range(job.d + 1):
        e = W + s_log2 + k * (job.e_in - job.p)
        out.append(fmath.rn_scaled_coeff(job.func, X_t, k, e) & mask)
    return out


def horner(coeffs: List[int], y: int, W: int) -> int:
    """sum_k c_k y^k mod 2^W by Horner's rule."""
    acc = 0
    for c in reversed(coeffs):
        acc = acc * y + c
    return acc % (1 << W)


def line(coeffs: List[int], i: int, N: int, W: int) -> Tuple[int, int]:
    """(b_i, alpha_i) of sub-interval i."""
    r0 = horner(coeffs, i * N, W)
    r1 = horner(coeffs, i * N + 1, W)
    return r0, (r1 - r0) % (1 << W)


def search_words(b: int, alpha: int, m: int, W: int) -> Tuple[int, int]:
    """(B, A) of the one-sided test for eps = 2^-m."""
    mod = 1 << W
    B = ((b + (1 << (W - m))) % mod) >> (W - 64)
    A = ((-alpha) % mod) >> (W - 64)
    return B, A


def threshold(m: int) -> int:
    return 1 << (65 - m)
