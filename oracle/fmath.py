"""Rigorous enclosures of exp, 2^x and log and of their Taylor coefficients.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle): nothing on the product
path imports this module.

Every function returns an interval [lo, hi] of exact rationals (Fraction)
that provably contains the real value, with hi - lo <= 2^-bits.  The
enclosures come from exact partial sums of power series plus an explicit
bound on the tail, so a reader can check each one against the series it
sums:

  exp(x)     = sum_n x^n / n!                      (0 <= x <= 4)
  exp(x)     = exp(x / 2^j)^(2^j)                   (x > 4, x / 2^j <= 1)
  atanh(z)   = sum_n z^(2n+1) / (2n+1)              (0 <= z < 1)
  ln 2       = 2 atanh(1/3)
  2^x        = exp(x ln 2)                          (x < 4)
  2^x        = 2^n 2^(x - n),  n = floor(x)         (x >= 4, 2^n exact)
  log(X)     = e ln 2 - 2 atanh((1 - Y)/(1 + Y)),   X = Y 2^e, 1/2 <= Y < 1

The Taylor coefficients f^(k)(X)/k! needed by the block polynomials of
Sect. IV (Taylor approximation R_t of degree delta at the left end of each
block) are

  exp:  exp(X) / k!
  2^x:  2^X (ln 2)^k / k!
  log:  log(X) for k = 0,  (-1)^(k-1) / (k X^k) for k >= 1  (exact).

Exact points (2^X at integer X, the log coefficients of order >= 1) are
returned as degenerate intervals lo == hi.
"""
from __future__ import annotations

import functools
from fractions import Fraction
from typing import Tuple

Interval = Tuple[Fraction, Fraction]

FUNC_EXP, FUNC_EXP2, FUNC_LOG = 0, 1, 2


def _pow2(e: int) -> Fraction:
    return Fraction(1 << e) if e >= 0 else Fraction(1, 1 << -e)


def exp_interval(x: Fraction, bits: int) -> Interval:
    """exp(x) for rational x >= 0.

    Partial sum S_n = sum_{i<=n} x^i/i!; for n + 2 > x the tail is bounded by
    the geometric majorant x^(n+1)/(n+1)! * 1/(1 - x/(n+2)).  Above x = 4
    (the binades [4, 8) and up) the argument is halved j times and the
    enclosure squared back, see _exp_by_squaring."""
    x = Fraction(x)
    if x < 0:
        raise ValueError("exp_interval needs x >= 0")
    if x == 0:
        return Fraction(1), Fraction(1)
    if x > 4:
        return _exp_by_squaring(x, bits)
    # x = a / b.  The partial sum is kept over the common denominator
    # Q = b^n n! (the denominator of the n-th term x^n / n! = a^n / Q), so
    # S_n = U / Q with U <- U b n + a^n: the same exact rational as adding
    # the terms one by one, without reducing a fraction at every step.
    a, b = x.numerator, x.denominator
    P = Q = U = 1   # a^n, b^n n!, S_n Q; n = 0: S_0 = 1
    n = 0
    while True:
        n += 1
        P *= a
        Q *= b * n
        U = U * b * n + P
        if (n + 2) * b > a:  # n + 2 > x
            # tail = x^(n+1)/(n+1)! / (1 - x/(n+2))
            #      = a^(n+1) (n+2) / (Q (n+1) ((n+2) b - a))
            tn = P * a * (n + 2)
            td = Q * (n + 1) * ((n + 2) * b - a)
            if _at_most_pow2(tn, td, -bits):
                s = Fraction(U, Q)
                return s, s + Fraction(tn, td)


def _at_most_pow2(num: int, den: int, e: int) -> bool:
    """num / den <= 2^e for integers num >= 0, den > 0."""
    if e >= 0:
        return num <= den << e
    return num << -e <= den


def atanh_interval(z: Fraction, bits: int) -> Interval:
    """atanh(z) for rational 0 <= z < 1.

    Tail after the term z^(2n+1)/(2n+1) is at most
    z^(2n+3)/((2n+3)(1 - z^2))."""
    z = Fraction(z)
    if not (0 <= z < 1):
        raise ValueError("atanh_interval needs 0 <= z < 1")
    if z == 0:
        return Fraction(0), Fraction(0)
    # z = c / e.  Term n is z^(2n+1) / (2n+1) = c^(2n+1) / (e^(2n+1) (2n+1));
    # the partial sum is kept over the common denominator
    # Q = e^(2n+1) * 1 * 3 * ... * (2n+1) as S_n = U / Q (the same exact
    # rational as adding the terms one by one).
    c, e = z.numerator, z.denominator
    c2, e2 = c * c, e * e
    C, E, R = c, e, 1   # c^(2n+1), e^(2n+1), 1 * 3 * ... * (2n+1)
    U = c               # n = 0: S_0 = z = c / e
    n = 0
    while True:
        # tail after term n: z^(2n+3) / ((2n+3) (1 - z^2))
        #                  = C c^2 / (E (2n+3) (e^2 - c^2))
        tn = C * c2
        td = E * (2 * n + 3) * (e2 - c2)
        if _at_most_pow2(tn, td, -bits):
            s = Fraction(U, E * R)
            return s, s + Fraction(tn, td)
        n += 1
        k = 2 * n + 1
        # U / (E R) + C c^2 / (E e^2 k) over the new denominator E e^2 R k
        U = U * e2 * k + C * c2 * R
        C *= c2
        E *= e2
        R *= k


@functools.lru_cache(maxsize=None)
def ln2_interval(bits: int) -> Interval:
    """ln 2 = 2 atanh(1/3) (memoised: the 2^x coefficients of every block of
    a job ask for the same few precisions)."""
    lo, hi = atanh_interval(Fraction(1, 3), bits + 1)
    return 2 * lo, 2 * hi


def _round_down(x: Fraction, bits: int) -> Fraction:
    """Largest multiple of 2^-bits not above x."""
    return Fraction((x.numerator << bits) // x.denominator, 1 << bits)


def _round_up(x: Fraction, bits: int) -> Fraction:
    return Fraction(-((-x.numerator << bits) // x.denominator), 1 << bits)


def _exp_by_squaring(x: Fraction, bits: int) -> Interval:
    """exp(x) = exp(x / 2^j)^(2^j) for x > 4 with x / 2^j <= 1.

    The series encloses exp(x / 2^j); each squaring maps an enclosure of
    positive numbers to one of their squares (t -> t^2 increases on t > 0),
    and the ends are rounded outward to the grid 2^-g after every step so
    that the fractions stay short.  The relative width at most doubles per
    squaring plus two grid steps, which g = bits + 1.45 x + 2 j + 8 covers;
    the width is checked at the end and g raised if it is not met."""
    j = 0
    while x / (1 << j) > 1:
        j += 1
    y = x / (1 << j)
    eps = _pow2(-bits)
    g = bits + int(x * Fraction(145, 100)) + 2 * j + 8
    while True:
        lo, hi = exp_interval(y, g)
        lo, hi = _round_down(lo, g), _round_up(hi, g)
        for _ in range(j):
            lo, hi = _round_down(lo * lo, g), _round_up(hi * hi, g)
        if hi - lo <= eps:
            return lo, hi
        g += 64


def exp2_interval(x: Fraction, bits: int) -> Interval:
    """2^x for rational x >= 0: exact at integers, else exp(x ln 2) (x >= 4:
    2^n times 2^(x - n), n = floor(x)).

    The argument x ln 2 is enclosed, rounded outward to a dyadic grid, and
    exp is increasing, so exp(lower argument) <= 2^x <= exp(upper argument)."""
    x = Fraction(x)
    if x < 0:
        raise ValueError("exp2_interval needs x >= 0")
    if x.denominator == 1:
        v = Fraction(1 << int(x))
        return v, v
    if x >= 4:  # 2^x = 2^n 2^(x - n), the power of two exact
        n = x.numerator // x.denominator
        lo, hi = exp2_interval(x - n, bits + n)
        return lo * (1 << n), hi * (1 << n)
    g = bits + 8 + int(x) + 2
    l_lo, l_hi = ln2_interval(g + 2)
    a_lo = _round_down(x * l_lo, g)
    a_hi = _round_up(x * l_hi, g)
    lo, _ = exp_interval(a_lo, g)
    _, hi = exp_interval(a_hi, g)
    return lo, hi


def log_interval(x: Fraction, bits: int) -> Interval:
    """log(x) for rational x >= 1/2 (only x > 1 is used by the jobs).

    x = Y 2^e with 1/2 <= Y < 1, log x = e ln 2 + log Y, and
    log Y = -2 atanh(z) with z = (1 - Y)/(1 + Y) in (0, 1/3]."""
    x = Fraction(x)
    if x <= 0:
        raise ValueError("log_interval needs x > 0")
    e = 0
    y = x
    while y >= 1:
        y /= 2
        e += 1
    while y < Fraction(1, 2):
        y *= 2
        e -= 1
    z = (1 - y) / (1 + y)
    g = bits + 4 + max(1, abs(e)).bit_length()
    a_lo, a_hi = atanh_interval(z, g)
    l_lo, l_hi = ln2_interval(g)
    if e >= 0:
        return e * l_lo - 2 * a_hi, e * l_hi - 2 * a_lo
    return e * l_hi - 2 * a_hi, e * l_lo - 2 * a_lo


def f_interval(func: int, x: Fraction, bits: int) -> Interval:
    if func == FUNC_EXP:
        return exp_interval(x, bits)
    if func == FUNC_EXP2:
        return exp2_interval(x, bits)
    if func == FUNC_LOG:
        return log_interval(x, bits)
    raise ValueError("unknown function")


def _factorial(k: int) -> int:
    r = 1
    for i in range(2, k + 1):
        r *= i
    return r


def taylor_coeff_interval(func: int, x: Fraction, k: int, bits: int) -> Interval:
    """Enclosure of f^(k)(x)/k!, width <= 2^-bits (values here are below 2^4)."""
    x = Fraction(x)
    if k == 0:
        return f_interval(func, x, bits)
    if func == FUNC_EXP:
        lo, hi = exp_interval(x, bits + 2)
        kf = _factorial(k)
        return lo / kf, hi / kf
    if func == FUNC_EXP2:
        g = bits + 4 + 2 * k + int(x)
        e_lo, e_hi = exp2_interval(x, g)
        l_lo, l_hi = ln2_interval(g)
        kf = _factorial(k)
        return e_lo * l_lo ** k / kf, e_hi * l_hi ** k / kf
    if func == FUNC_LOG:
        v = Fraction((-1) ** (k - 1), k) / x ** k
        return v, v
    raise ValueError("unknown function")


def round_nearest(v: Fraction) -> int:
    """floor(v + 1/2): nearest integer, halves rounded up."""
    t = v + Fraction(1, 2)
    return t.numerator // t.denominator


def rn_scaled_coeff(func: int, x: Fraction, k: int, scale_log2: int) -> int:
    """RN(2^scale_log2 * f^(k)(x)/k!) as an exact integer (Ziv's strategy:
    raise the enclosure precision until both ends round alike)."""
    bits = max(scale_log2, 0) + 64
    while True:
        lo, hi = taylor_coeff_interval(func, x, k, bits)
        s = _pow2(scale_log2)
        r_lo = round_nearest(lo * s)
        r_hi = round_nearest(hi * s)
        if r_lo == r_hi:
            return r_lo
        bits += 64
        if bits > 8192:
            raise ArithmeticError("rounding undecided at 8192 bits")


def exponent_of(func: int, x: Fraction) -> int:
    """e(f(x)): the integer e with 2^(e-1) <= f(x) < 2^e (Def. 1)."""
    bits = 64
    while True:
        lo, hi = f_interval(func, x, bits)
        if lo <= 0:
            raise ValueError("f(x) must be positive")
        e_lo = _exponent_exact(lo)
        e_hi = _exponent_exact(hi)
        if e_lo == e_hi:
            return e_lo
        bits += 64
        if bits > 8192:
            raise ArithmeticError("exponent undecided at 8192 bits")


def _exponent_exact(v: Fraction) -> int:
    """The e with 2^(e-1) <= v < 2^e for a positive rational v."""
    e = v.numerator.bit_length() - v.denominator.bit_length()
    # now 2^(e-1) < v < 2^(e+1); fix up exactly
    while v >= _pow2(e):
        e += 1
    while v < _pow2(e - 1):
        e -= 1
    return e
