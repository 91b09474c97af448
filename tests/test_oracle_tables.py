"""Pins of the oracle's difference-table routines (Sect. IV): the paper's
Figs. 5 and 6, the binomial-basis identity, and agreement with direct
Horner at every point."""
import random

from conftest import read_golden
from oracle import poly, search


def test_fig5_newton_interpolation_of_x3():
    want = [[int(v) for v in r] for r in read_golden("fig5_newton_x3.txt")]
    assert search.forward_differences([x ** 3 for x in range(4)]) == want


def test_fig6_tabulated_differences_of_i3():
    rows = [[int(v) for v in r] for r in read_golden("fig6_tabdiff_i3.txt")]
    col0 = [r[0] for r in rows]                      # Delta^l[r](0)
    cols = search.tabulated_shift(col0, len(rows[0]))
    for i, col in enumerate(cols):
        assert col == [rows[l][i] for l in range(len(rows))]


def test_binomial_basis_reconstruction():
    """R(x) = sum_j Delta^j[R](0) binom(x, j) (Sect. IV-A)."""
    from math import comb
    rng = random.Random(1)
    for _ in range(20):
        deg = rng.randrange(1, 6)
        c = [rng.randrange(-1000, 1000) for _ in range(deg + 1)]
        R = lambda x: sum(ck * x ** k for k, ck in enumerate(c))
        coef = [r[0] for r in search.forward_differences([R(x) for x in range(deg + 1)])]
        for x in range(40):
            assert R(x) == sum(coef[j] * comb(x, j) for j in range(deg + 1))


def test_straightforward_equals_tabulated():
    rng = random.Random(2)
    mod = 1 << 192
    for _ in range(10):
        col = [rng.getrandbits(192) for _ in range(rng.randrange(2, 6))]
        steps = search.tabulated_shift(col, 70, mod)
        for n in (0, 1, 5, 37, 69):
            assert search.straightforward_shift(col, n, mod) == steps[n]


def test_tables_equal_horner_at_every_point():
    """The step-N difference tables of g0(i) = R(iN) and
    g1(i) = R(iN+1) - R(iN), stepped by additions mod 2^W, reproduce the
    oracle's direct-Horner (b_i, alpha_i) at every sub-interval."""
    rng = random.Random(3)
    for W, d, N, n in ((64, 2, 256, 16), (192, 3, 1 << 14, 1024), (128, 2, 4096, 64)):
        mod = 1 << W
        c = [rng.getrandbits(W) for _ in range(d + 1)]
        g0 = [poly.horner(c, i * N, W) for i in range(d + 1)]
        g1 = [(poly.horner(c, i * N + 1, W) - poly.horner(c, i * N, W)) % mod for i in range(d)]
        t0 = [r[0] % mod for r in search.forward_differences(g0)]
        t1 = [r[0] % mod for r in search.forward_differences(g1)]
        s0 = search.tabulated_shift(t0, n, mod)
        s1 = search.tabulated_shift(t1, n, mod)
        for i in range(n):
            assert (s0[i][0], s1[i][0]) == poly.line(c, i, N, W)
