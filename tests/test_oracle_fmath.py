"""Pins of the oracle's f enclosures: exact points, identities, libm and
(when importable) mpmath at higher precision."""
import math
import random
from fractions import Fraction

import pytest

from oracle import fmath

F = Fraction


def contains(iv, v):
    return iv[0] <= v <= iv[1]


def test_exact_points():
    assert fmath.exp_interval(F(0), 100) == (1, 1)
    for k in range(0, 8):
        assert fmath.exp2_interval(F(k), 100) == (2 ** k, 2 ** k)
    # log(1) = 0 and log(2^k) = k ln 2 lie in the enclosures
    assert contains(fmath.log_interval(F(1), 200), 0)
    l2 = fmath.ln2_interval(300)
    for k in range(1, 9):
        lo, hi = fmath.log_interval(F(2 ** k), 200)
        assert lo <= k * l2[1] and k * l2[0] <= hi


def test_widths():
    for bits in (64, 200, 400):
        for iv in (fmath.exp_interval(F(3, 5), bits), fmath.ln2_interval(bits),
                   fmath.exp2_interval(F(7, 11), bits), fmath.log_interval(F(29, 7), bits)):
            assert 0 <= iv[1] - iv[0] <= F(1, 2 ** bits)


def test_against_libm():
    rng = random.Random(3)
    for _ in range(200):
        x = F(rng.randrange(1, 1 << 30), 1 << 29)     # (0, 2)
        assert abs(float(fmath.exp_interval(x, 80)[0]) - math.exp(x)) <= 4e-16 * math.exp(x)
        assert abs(float(fmath.exp2_interval(x, 80)[0]) - 2.0 ** float(x)) <= 4e-16 * 2.0 ** float(x)
        y = F(rng.randrange(1 << 30, 1 << 33), 1 << 29)   # [2, 16)
        assert abs(float(fmath.log_interval(y, 80)[0]) - math.log(y)) <= 4e-16 * math.log(y)


def test_against_mpmath_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    rng = random.Random(5)
    for _ in range(12):
        x = F(rng.randrange(1, 1 << 53), 1 << 53) + rng.choice([0, 1])
        e = mpmath.exp(mpmath.mpf(x.numerator) / x.denominator)
        lo, hi = fmath.exp_interval(x, 320)
        assert mpmath.mpf(lo.numerator) / lo.denominator <= e <= mpmath.mpf(hi.numerator) / hi.denominator
        e2 = mpmath.power(2, mpmath.mpf(x.numerator) / x.denominator)
        lo, hi = fmath.exp2_interval(x, 320)
        assert mpmath.mpf(lo.numerator) / lo.denominator <= e2 <= mpmath.mpf(hi.numerator) / hi.denominator
        y = x * 4 + 2
        lg = mpmath.log(mpmath.mpf(y.numerator) / y.denominator)
        lo, hi = fmath.log_interval(y, 320)
        assert mpmath.mpf(lo.numerator) / lo.denominator <= lg <= mpmath.mpf(hi.numerator) / hi.denominator


def test_identities():
    # exp(log x) = x  and  exp(a) exp(b) = exp(a + b)  and  2^x 2^(1-x) = 2
    for x in (F(5, 2), F(7, 1), F(123456789, 2 ** 25)):
        lo, hi = fmath.log_interval(x, 120)
        assert fmath.exp_interval(lo, 120)[0] <= x <= fmath.exp_interval(hi, 120)[1]
    a, b = F(3, 7), F(5, 11)
    ea, eb, eab = fmath.exp_interval(a, 150), fmath.exp_interval(b, 150), fmath.exp_interval(a + b, 150)
    assert ea[0] * eb[0] <= eab[1] and eab[0] <= ea[1] * eb[1]
    x = F(3, 10)
    p, q = fmath.exp2_interval(x, 150), fmath.exp2_interval(1 - x, 150)
    assert p[0] * q[0] <= 2 <= p[1] * q[1]


@pytest.mark.parametrize("func,x0", [(fmath.FUNC_EXP, F(5, 8)), (fmath.FUNC_EXP2, F(3, 4)),
                                     (fmath.FUNC_LOG, F(11, 4))])
def test_taylor_coefficients_reproduce_f(func, x0):
    """sum_k f^(k)(x0)/k! h^k matches f(x0 + h) to the Lagrange remainder:
    a wrong derivative formula (sign, factor, order) fails this."""
    deg = 7
    for h in (F(1, 2 ** 8), F(3, 2 ** 9), F(-1, 2 ** 8)):
        s_lo = sum(fmath.taylor_coeff_interval(func, x0, k, 200)[0] * h ** k for k in range(deg + 1))
        lo, hi = fmath.f_interval(func, x0 + h, 200)
        # |f^(8)/8!| <= 8 on these points; remainder bound with margin
        rem = 8 * abs(h) ** (deg + 1) + F(1, 2 ** 150)
        assert lo - rem <= s_lo <= hi + rem


def test_round_nearest_and_scaled():
    assert fmath.round_nearest(F(1, 2)) == 1
    assert fmath.round_nearest(F(-1, 2)) == 0
    assert fmath.round_nearest(F(3, 2)) == 2
    assert fmath.round_nearest(F(-7, 4)) == -2
    # exact: log coefficient k=1 at x=2 is 1/2, scaled by 2^10 gives 512
    assert fmath.rn_scaled_coeff(fmath.FUNC_LOG, F(2), 1, 10) == 512
    assert fmath.rn_scaled_coeff(fmath.FUNC_LOG, F(2), 2, 10) == -128
    # 2^x at x = 1, order 0, scale 2^5: exactly 64
    assert fmath.rn_scaled_coeff(fmath.FUNC_EXP2, F(1), 0, 5) == 64
    # a transcendental value: RN(2^60 e) against libm to 1e-15 relative
    v = fmath.rn_scaled_coeff(fmath.FUNC_EXP, F(1), 0, 60)
    assert abs(v / 2.0 ** 60 - math.e) < 1e-15


def test_exponent_of():
    assert fmath.exponent_of(fmath.FUNC_EXP, F(1, 2)) == 1     # e^0.5 in [1, 2)
    assert fmath.exponent_of(fmath.FUNC_EXP, F(7, 10)) == 2    # e^0.7 in [2, 4)
    assert fmath.exponent_of(fmath.FUNC_EXP2, F(1)) == 2       # 2 = (1/2) 2^2
    assert fmath.exponent_of(fmath.FUNC_LOG, F(3)) == 1        # log 3 in [1, 2)
    assert fmath.exponent_of(fmath.FUNC_LOG, F(5, 2)) == 0     # log 2.5 in [1/2, 1)


def test_large_arguments_against_libm():
    """exp and 2^x on [4, 512) (the halving-squaring and integer-split
    reductions) against libm, relative 1e-15."""
    rng = random.Random(11)
    for e_in in (3, 5, 8, 9):
        for _ in range(20):
            x = F(rng.randrange(1 << 40, 1 << 41), 1 << (41 - e_in))   # [2^(e_in-1), 2^e_in)
            if x > 700:
                continue
            lo, hi = fmath.exp_interval(x, 64)
            assert abs(float(lo) / math.exp(x) - 1) < 1e-15 and lo <= hi
            lo2, hi2 = fmath.exp2_interval(x, 64)
            assert abs(float(lo2) / 2.0 ** float(x) - 1) < 1e-15 and lo2 <= hi2


def test_squaring_path_matches_series():
    """exp(a + b) from the squaring path against exp(a) exp(b) from the
    plain series (a, b <= 4), and the absolute width at several precisions."""
    for a, b in ((F(3, 1), F(7, 4)), (F(37, 10), F(39, 10)), (F(1, 3), F(4))):
        ea, eb = fmath.exp_interval(a, 200), fmath.exp_interval(b, 200)
        lo, hi = fmath.exp_interval(a + b, 200)
        assert ea[0] * eb[0] <= hi and lo <= ea[1] * eb[1]
    for bits in (40, 128, 300):
        for x in (F(4) + F(1, 2 ** 45), F(200 * 2 ** 45 + 12345, 2 ** 45)):
            lo, hi = fmath.exp_interval(x, bits)
            assert 0 <= hi - lo <= F(1, 2 ** bits)
            lo, hi = fmath.exp2_interval(x, bits)
            assert 0 < hi - lo <= F(1, 2 ** bits)


def test_exp_brackets_powers_of_two():
    """For dyadic x_lo < K ln 2 < x_hi (ln 2 from the atanh series, not exp),
    exp(x_lo) < 2^K < exp(x_hi): ties the large-argument exp to ln 2."""
    l_lo, l_hi = fmath.ln2_interval(200)
    for K in (6, 100, 185, 369, 738):
        x_lo = F((K * l_lo.numerator << 120) // l_lo.denominator, 1 << 120)
        x_hi = x_lo + F(2, 1 << 120)
        assert x_lo < K * l_lo and K * l_hi < x_hi
        assert fmath.exp_interval(x_lo, 160)[1] < 2 ** K < fmath.exp_interval(x_hi, 160)[0]
        # and e(f) flips exactly there
        assert fmath.exponent_of(fmath.FUNC_EXP, x_lo) == K
        assert fmath.exponent_of(fmath.FUNC_EXP, x_hi) == K + 1


def test_exponent_of_against_libm_over_all_binades():
    """e(f(X)) (Def. 1) against frexp of libm's f(X) at random X of every
    supported binade: exp and 2^x on [2^-17, 2^-16) .. [256, 512), log on
    [2, 4) .. [2^15, 2^16); points within 1e-9 of a power of two skipped."""
    rng = random.Random(1211)
    for func, e_ins in ((fmath.FUNC_EXP, range(-16, 10)), (fmath.FUNC_EXP2, range(-16, 10)),
                        (fmath.FUNC_LOG, range(2, 17))):
        fn = {fmath.FUNC_EXP: math.exp, fmath.FUNC_EXP2: lambda v: 2.0 ** v, fmath.FUNC_LOG: math.log}[func]
        for e_in in e_ins:
            for _ in range(4):
                x = F(rng.randrange(1 << 52, 1 << 53), 1 << (53 - e_in))   # [2^(e_in-1), 2^e_in)
                v = fn(float(x))
                m, e = math.frexp(v)
                if abs(m - 0.5) < 1e-9 or abs(m - 1.0) < 1e-9:
                    continue
                assert fmath.exponent_of(func, x) == e, (func, e_in, float(x))
