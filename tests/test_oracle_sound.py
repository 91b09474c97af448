"""Pins of the oracle's sound mode (Sect. II-A's eps'' = eps + eps_approx +
eps_trunc and the exhaustive phase 3 of Sect. III-A): each error bound holds
against the exact function and the exact integer lines, and the exhaustive
candidate list contains every hard-to-round argument (Def. 3), decided
exactly argument by argument on small formats."""
import random
from fractions import Fraction

import pytest

import workloads as wl
from oracle import fmath, plan, poly, sound

SMALL = [
    wl.Job(wl.FUNC_EXP, 0, 24, 10, 8, 2, 12, 1, 3 << 20, 1 << 13),
    wl.Job(wl.FUNC_EXP2, 1, 22, 7, 7, 3, 11, 1, 12345, 1 << 11, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_LOG, 2, 20, 8, 6, 2, 10, 1, 100, 1 << 12),
    wl.Job(wl.FUNC_EXP, 0, 20, 7, 6, 2, 10, 2, 0, 1 << 19),      # crosses e_out at ln 2, W = 128
]

# The binade [128, 256) (range-reduced coefficients): exp across the cut at
# 260 ln 2 (a one-argument first segment), 2^x across X = 200.
BIG_BINADE = [
    wl.Job(wl.FUNC_EXP, 8, 24, 7, 2, 2, 4, 1, 1837266934047447 >> 29, 1 << 11),
    wl.Job(wl.FUNC_EXP2, 8, 24, 10, 3, 2, 5, 1, (72 << 16) - 700, 1 << 11),
]


def frac_cmod(v: Fraction) -> Fraction:
    """v cmod 1 in [-1/2, 1/2)."""
    f = v - (v.numerator // v.denominator)
    return f - 1 if f >= Fraction(1, 2) else f


@pytest.mark.parametrize("job", SMALL + BIG_BINADE[:1], ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}")
def test_eps_approx_holds_on_sampled_arguments(job):
    """|R_t(y)/2^W - s f(X)| cmod 1 <= eps_approx, X exact from enclosures."""
    ea = sound.eps_approx(job)
    W = 64 * job.limbs
    rng = random.Random(job.count)
    blocks = plan.blocks(job)
    for blk in rng.sample(blocks, min(6, len(blocks))):
        c = poly.taylor_coeffs(job, blk)
        s = fmath._pow2(plan.scale_log2(job, blk.e_out))
        for y in [0, blk.length - 1] + [rng.randrange(blk.length) for _ in range(20)]:
            X = plan.argument(job, blk.start + y)
            lo, hi = fmath.f_interval(job.func, X, 96)
            r = Fraction(poly.horner(c, y, W), 1 << W)
            for v in (lo * s, hi * s):
                assert abs(frac_cmod(r - v)) <= ea + Fraction(1, 1 << 90)


@pytest.mark.parametrize("job", SMALL + [wl.plain_job(count_log2=30)] + BIG_BINADE,
                         ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}N{j.log2_N}")
def test_eps_trunc_holds_on_sampled_subintervals(job):
    """max_x |R_t(iN + x) - (b_i + alpha_i x)| cmod 2^W <= eps_trunc 2^W over
    whole sub-intervals (exact integers)."""
    et = sound.eps_trunc(job)
    W, N = 64 * job.limbs, 1 << job.log2_N
    mod = 1 << W
    rng = random.Random(7 + job.count)
    blocks = plan.blocks(job)
    worst = Fraction(0)
    for blk in rng.sample(blocks, min(3, len(blocks))):
        c = poly.taylor_coeffs(job, blk)
        nsub = (blk.length + N - 1) // N
        for i in sorted({0, nsub - 1, rng.randrange(nsub)}):
            b, a = poly.line(c, i, N, W)
            xs = range(min(N, blk.length - i * N))
            if N > 4096:
                xs = [0, 1, 2, N // 2, N - 2, N - 1] + [rng.randrange(N) for _ in range(200)]
            for x in xs:
                diff = (poly.horner(c, i * N + x, W) - b - a * x) % mod
                if diff >= mod // 2:
                    diff -= mod
                worst = max(worst, Fraction(abs(diff), mod))
    assert worst <= et
    assert worst > et / 64   # the bound is not vacuous either


@pytest.mark.parametrize("job", SMALL[:3] + BIG_BINADE[:1], ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}")
def test_sound_candidates_contain_every_hard_to_round_argument(job):
    """Every argument of the job decided hard-to-round from the exact f is
    in the exhaustive list taken at the smallest sound eps3; the list holds
    nothing farther than eps3."""
    e1, e3 = sound.min_eps(job)
    cands = sound.sound_candidates([job], [e3])
    listed = {r[2] for r in cands}
    hr = [j for j in range(job.start, job.start + job.count) if sound.is_hard_to_round(job, j)]
    assert len(hr) > 10
    assert set(hr) <= listed
    assert all(r[3] < 2 * e3 for r in cands)
    # eps3 exceeds 2^-m only by the approximation bound: the list is about
    # eps3 / 2^(64-m) times the hard-to-round set
    assert len(listed) <= len(hr) * 1.5 * e3 / (1 << (64 - job.m)) + 8


def test_min_eps_orders():
    for job in SMALL + [wl.plain_job()]:
        e1, e3 = sound.min_eps(job)
        assert e3 > 1 << (64 - job.m)
        assert e1 > e3 + (1 << job.log2_N)


def test_planted_exact_point_is_hard_to_round():
    """2^x on [1,2) at X = 1: s 2^X is an integer, distance 0."""
    job = wl.Job(wl.FUNC_EXP2, 1, 24, 20, 8, 2, 12, 1, 0, 1 << 12)
    assert sound.is_hard_to_round(job, 0)
    e1, e3 = sound.min_eps(job)
    assert sound.sound_candidates([job], [e3])[0][:3] == (0, 0, 0)


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("job", SMALL[:3] + [wl.plain_job(count_log2=30)] + BIG_BINADE[:1],
                         ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}N{j.log2_N}")
def test_piece_truncation_bound_holds(job, level):
    """eps_trunc for the phase-2 pieces (N/32 arguments) and for their 32
    sub-pieces (level 2: ceil(N/32/32) arguments), a line from the two values
    at the start, against the exact integer polynomial."""
    n2 = sound.piece_length(job)
    if level == 2:
        n2 = (n2 + 31) // 32
    et = sound.eps_trunc(job, n2)
    W = 64 * job.limbs
    mod = 1 << W
    rng = random.Random(31 + job.count)
    worst = Fraction(0)
    blocks = plan.blocks(job)
    for blk in rng.sample(blocks, min(2, len(blocks))):
        c = poly.taylor_coeffs(job, blk)
        for _ in range(6):
            y0 = rng.randrange(0, max(1, blk.length - n2))
            r0 = poly.horner(c, y0, W)
            a = (poly.horner(c, y0 + 1, W) - r0) % mod
            for x in range(n2):
                diff = (poly.horner(c, y0 + x, W) - r0 - a * x) % mod
                if diff >= mod // 2:
                    diff -= mod
                worst = max(worst, Fraction(abs(diff), mod))
    assert worst <= et
    e1, e3 = sound.min_eps(job)
    assert e3 < sound.min_eps_len(job, e3, n2) <= sound.min_eps2(job, e3) < e1
