"""Whole-chain pins of the oracle on small formats.

Exhaustive sandwich: for EVERY argument of a reduced-precision format the
oracle's degree-1 line (b_i + alpha_i x) / 2^W must sit within the
truncation and Taylor-remainder bounds of s f(X) computed by libm (numpy's
exp / exp2 / log in float64, an implementation independent of the oracle's
series).  Planted mistakes in the oracle (a dropped coefficient, a wrong
scale, a wrong derivative sign) push the error far past the bound; the
mutation tests at the end check exactly that."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import candidates, fmath, plan, poly


def _libm(func):
    return {wl.FUNC_EXP: np.exp, wl.FUNC_EXP2: np.exp2, wl.FUNC_LOG: np.log}[func]


def _deriv_max(func, x_lo, x_hi, order):
    """max |f^(order)| on [x_lo, x_hi] (each f^(order) is monotone there)."""
    if func == wl.FUNC_EXP:
        return math.exp(x_hi)
    if func == wl.FUNC_EXP2:
        return 2.0 ** x_hi * math.log(2) ** order
    return math.factorial(order - 1) / x_lo ** order


def sandwich_max_error(job):
    """(max over blocks of error/bound, largest bound): error is the largest
    |(s f(X) - line(x)) cmod 1| over the block's arguments, bound the sum of
    the degree-1 truncation s u^2 max|f''| N^2/2 and the Taylor remainder
    s (T u)^(d+1) max|f^(d+1)|/(d+1)!, doubled, plus float64 rounding."""
    assert job.limbs == 1
    W = 64
    N = 1 << job.log2_N
    u = 2.0 ** (job.e_in - job.p)
    f = _libm(job.func)
    worst_ratio, max_bound = 0.0, 0.0
    for blk in plan.blocks(job):
        c, B, A, n = candidates.block_lines(job, blk)
        j = np.arange(blk.start, blk.start + blk.length, dtype=np.int64)
        X = (2.0 ** (job.p - 1) + j.astype(np.float64)) * u
        fx = f(X)
        # Def. 1 straight from libm: f = m 2^e with 1/2 <= m < 1
        _, e_out = np.frexp(fx)
        s_exp = (job.p - e_out) if job.flags & wl.FLAG_BP_DIRECTED else (job.p + 1 - e_out)
        y = np.ldexp(fx, s_exp)
        frac_true = y - np.floor(y)
        i = (j - blk.start) // N
        x = (j - blk.start) % N
        lines = [poly.line(c, int(k), N, W) for k in range(len(B))]
        b = np.array([t[0] for t in lines], dtype=np.uint64)
        al = np.array([t[1] for t in lines], dtype=np.uint64)
        lin = b[i] + al[i] * x.astype(np.uint64)          # mod 2^64
        frac_lin = lin.astype(np.float64) / 2.0 ** 64
        diff = frac_true - frac_lin
        diff -= np.round(diff)
        err = float(np.max(np.abs(diff)))
        sc = 2.0 ** float(np.max(s_exp))
        x_lo, x_hi = float(X[0]), float(X[-1])
        trunc = sc * u * u * _deriv_max(job.func, x_lo, x_hi, 2) / 2 * N * N
        taylor = (sc * (blk.length * u) ** (job.d + 1)
                  * _deriv_max(job.func, x_lo, x_hi, job.d + 1) / math.factorial(job.d + 1))
        float_err = 2.0 ** (job.p + 1) * 2.0 ** -51 + 2.0 ** -52
        bound = 2 * (trunc + taylor) + float_err
        worst_ratio = max(worst_ratio, err / bound)
        max_bound = max(max_bound, bound)
    return worst_ratio, max_bound


SANDWICH_JOBS = [
    wl.toy_job(),                                                         # exp, p=24
    wl.Job(wl.FUNC_EXP, 1, 20, 12, 6, 3, 12, 1, 0, 1 << 19),             # exp on [1,2)
    wl.Job(wl.FUNC_EXP2, 0, 20, 12, 6, 2, 10, 1, 0, 1 << 19),            # 2^x on [1/2,1)
    wl.Job(wl.FUNC_LOG, 2, 20, 12, 6, 2, 10, 1, 0, 1 << 19),             # log on [2,4)
    wl.Job(wl.FUNC_LOG, 3, 20, 12, 6, 3, 11, 1, 1000, 300000, 1),        # log on [4,8), directed
]


@pytest.mark.parametrize("job", SANDWICH_JOBS, ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}d{j.d}")
def test_exhaustive_sandwich(job):
    ratio, bound = sandwich_max_error(job)
    assert ratio <= 1.0, (ratio, bound)
    assert bound < 0.05          # tight enough that a wrong term cannot hide


def test_toy_segments_cut_at_ln2():
    job = wl.toy_job()
    segs = plan.segments(job)
    assert len(segs) == 2 and segs[0][2] == 1 and segs[1][2] == 2
    cut = segs[1][0]
    X_cut = plan.argument(job, cut)
    X_prev = plan.argument(job, cut - 1)
    assert float(X_prev) < math.log(2) <= float(X_cut)
    l2 = fmath.ln2_interval(200)
    assert X_prev < l2[0] and l2[1] < X_cut


def test_planted_exact_hit():
    """2^x on [1, 2) at X = 1: s f(1) = 2^(p+1-2) * 2 = 2^p is an integer, so
    b = 0 and the first argument is a hit with value exactly 2^(64-m)."""
    job = wl.Job(wl.FUNC_EXP2, 1, 24, 16, 8, 2, 12, 1, 0, 1 << 12)
    blk = plan.blocks(job)[0]
    c = poly.taylor_coeffs(job, blk)
    assert c[0] == 0
    got = candidates.job_candidates(job)
    assert got[0] == (0, 0, 0, 1 << (64 - 16))
    job3 = wl.Job(wl.FUNC_EXP2, 1, 53, 40, 14, 3, 24, 3, 0, 1 << 14)
    assert candidates.job_candidates(job3)[0] == (0, 0, 0, 1 << 24)


def test_toy_hit_statistics():
    """Every argument's value is below 2^(65-m) with probability 2^(1-m):
    2^23 * 2^-11 = 4096 expected hits."""
    job = wl.toy_job(flags=wl.FLAG_ALL_HITS)
    hits = candidates.candidates([job])
    assert 0.9 * 4096 < len(hits) < 1.1 * 4096
    subs = {h[1] for h in hits}
    plain = candidates.candidates([wl.toy_job()])
    assert {r[1] for r in plain} == subs
    # each candidate is the smallest of its sub-interval's hits
    best = {}
    for h in hits:
        if h[1] not in best or h[3] < best[h[1]][3]:
            best[h[1]] = h
    assert sorted(best.values(), key=lambda r: (r[0], r[2], r[3])) == plain


# ---- planted mistakes (in the oracle, on the CPU): the pins must catch them

def _mutated_error(monkeypatch, job, target, replacement):
    monkeypatch.setattr(target[0], target[1], replacement)
    return sandwich_max_error(job)


def test_mutation_dropped_quadratic_term(monkeypatch):
    orig = poly.taylor_coeffs
    ratio, _ = _mutated_error(monkeypatch, wl.toy_job(), (poly, "taylor_coeffs"),
                              lambda job, blk: orig(job, blk)[:2] + [0] * (job.d - 1))
    assert ratio > 10


def test_mutation_wrong_scale(monkeypatch):
    orig = poly.scale_log2
    job = wl.Job(wl.FUNC_EXP2, 0, 20, 12, 6, 2, 10, 1, 0, 1 << 16)
    ratio, _ = _mutated_error(monkeypatch, job, (poly, "scale_log2"),
                              lambda j, e: orig(j, e) + 1)
    assert ratio > 10


def test_mutation_log_derivative_sign(monkeypatch):
    orig = fmath.taylor_coeff_interval

    def bad(func, x, k, bits):
        lo, hi = orig(func, x, k, bits)
        return (-hi, -lo) if (func == fmath.FUNC_LOG and k == 2) else (lo, hi)
    job = wl.Job(wl.FUNC_LOG, 2, 20, 12, 6, 2, 10, 1, 0, 1 << 16)
    ratio, _ = _mutated_error(monkeypatch, job, (fmath, "taylor_coeff_interval"), bad)
    assert ratio > 10


def test_mutation_transposed_line_operands(monkeypatch):
    orig = poly.line
    monkeypatch.setattr(poly, "line", lambda c, i, N, W: tuple(reversed(orig(c, i, N, W))))
    ratio, _ = sandwich_max_error(wl.toy_job())
    assert ratio > 10


def test_mutation_block_origin(monkeypatch):
    """Taylor expansion taken at the wrong point (one argument late)."""
    orig = poly.argument
    monkeypatch.setattr(poly, "argument", lambda job, j: orig(job, j + 1))
    ratio, _ = sandwich_max_error(wl.Job(wl.FUNC_EXP2, 0, 20, 12, 6, 2, 10, 1, 0, 1 << 14))
    assert ratio > 2
