"""Search definitions: brute-force minimum, three-distance geometry, the
continued-fraction lower bounds, and difference tables.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

The quantity the hot path decides is Eq. (1) of Sect. II-A,
    min { (b - a x) mod 1 : 0 <= x < N },
here on integers scaled by a modulus M (M = 2^64 for the search words):
    min { (B - A x) mod M : 0 <= x < N }.
`brute_min` is that definition written out.  The other routines are the
paper's machinery, kept here so the tests can pin it and compare the CUDA
filter with it value by value:

  gaps_in_order     lengths of the intervals cut by {a x mod 1 : x < n}
                    (Thm. 1, Fig. 3);
  cf_configurations the two-length configurations (i, t) with
                    theta_{i-1,t}, theta_i, q_{i-1,t}, q_i, k_{i+1} (Sect.
                    II-B recurrences, Table 1, Eq. 2, Property 1);
  regular_lb        the regular lower bound of Algorithm 2;
  regular_lb_unrolled
                    the same computation unrolled twice (Algorithm 4),
                    with the degenerate endings (a remainder reaching 0
                    for rational a) made explicit;
  lefevre_lb, lefevre_swap_lb, lefevre_test
                    Lefevre's lower bound (Algorithm 1) and its branch-
                    merged form with swaps (Algorithm 3), and the Boolean
                    test of Algorithm 1;
  nmdm              the loop-divergence indicator of Sect. II-B;
  forward_differences, tabulated_shift, straightforward_shift
                    Sect. IV difference tables (Figs. 5 and 6).
"""
from __future__ import annotations

from math import comb
from typing import List, Tuple


def brute_min(B: int, A: int, n: int, M: int = 1 << 64) -> Tuple[int, int]:
    """(min, smallest argmin) of (B - A x) mod M over 0 <= x < n."""
    best, arg = None, 0
    for x in range(n):
        v = (B - A * x) % M
        if best is None or v < best:
            best, arg = v, x
    return best, arg


def gaps_in_order(a: int, M: int, n: int) -> List[int]:
    """Interval lengths, left to right, cut on [0, M) by {a x mod M : x < n}."""
    pts = sorted({(a * x) % M for x in range(n)})
    pts.append(M)
    return [pts[i + 1] - pts[i] for i in range(len(pts) - 1)]


def cf_configurations(a: int, M: int):
    """Rows (i, t, q_{i-1,t}, q_i, theta_{i-1,t}, theta_i, k_{i+1}) of the
    two-length configurations of a/M (lengths scaled by M), in the order of
    Property 1, until theta_i = 0.  For the final row (theta_i = 0) k_{i+1}
    is undefined and reported as None."""
    rows = []
    th_prev, th = M, a           # theta_{-1} = 1, theta_0 = a  (scaled)
    q_prev, q = 0, 1             # q_{-1}, q_0
    i = 0
    while True:
        if th == 0:
            rows.append((i, 0, q_prev, q, th_prev, th, None))
            return rows
        k = th_prev // th
        for t in range(k):
            rows.append((i, t, q_prev + t * q, q, th_prev - t * th, th, k))
        th_prev, th = th, th_prev - k * th
        q_prev, q = q, q_prev + k * q
        i += 1


def regular_lb(B: int, A: int, N: int, M: int = 1 << 64) -> Tuple[int, int, int]:
    """Algorithm 2 on integers: returns (lower bound d, points u+v, loop
    iterations).  p <- A, q <- M, d <- B, u <- 1, v <- 0; each iteration
    reduces the longer length by the division-based Euclidean step and
    updates d; stops when u + v >= N.  A length reaching 0 ends the
    expansion (rational a): d is then final (the points form a lattice)."""
    p, q, d, u, v = A, M, B % M, 1, 0
    it = 0
    while True:
        if p == 0:
            return d % q, u + v, it
        if q == 0:
            return d, u + v, it
        it += 1
        if p < q:
            k = q // p
            q = q - k * p
            u = u + k * v
            d = d % p
        else:
            k = p // q
            p = p - k * q
            v = v + k * u
            if d >= p:
                d = (d - p) % q
        if u + v >= N:
            return d, u + v, it


def regular_lb_unrolled(B: int, A: int, N: int, M: int = 1 << 64) -> Tuple[int, int, int]:
    """Algorithm 4 on integers (the two branches of Algorithm 2 alternate,
    so two iterations are written one after the other).  Returns
    (d, u+v, half-steps).  Endings: p = 0 returns d mod q; q = 0 returns d."""
    p, q, d, u, v = A, M, B % M, 1, 0
    hs = 0
    while True:
        if p == 0:
            return d % q, u + v, hs
        k = q // p
        q = q - k * p
        u = u + k * v
        d = d % p
        hs += 1
        if u + v >= N or q == 0:
            return d, u + v, hs
        k = p // q
        p = p - k * q
        v = v + k * u
        if d >= p:
            d = (d - p) % q
        hs += 1
        if u + v >= N:
            return d, u + v, hs


def lefevre_lb(B: int, A: int, N: int, M: int = 1 << 64, specific: bool = False) -> Tuple[int, int, int]:
    """Algorithm 1 (Lefevre's lower bound computation) run to its Success
    exit, i.e. the test with eps'' = 0; returns (d, u+v, loop iterations).
    p <- a, q <- 1 - a, d <- b, u <- v <- 1 (scaled by M).  Each iteration
    either (d < p: the point added last lies right of b) takes a whole
    quotient k = floor(q/p) off q and the first unit of the next one off p,
    or (d >= p) moves d to the point just added at its left (d -= p) and
    takes k = floor(p/q) off p and one unit off q.  The test of Algorithm 1
    fails exactly when this d is below eps'' (d never grows).
    Degenerate endings (rational a, not covered by the printed algorithm):
    a division leaving a zero remainder means every interval now has the
    other length, so d reduced modulo that length is the distance over the
    whole lattice of points and the loop ends there.  A = 0: every point
    is 0, d = b.

    specific=True: Lefevre's "specific instructions" (Sect. III-B mentions
    them without printing them), read here as taking a run of consecutive
    iterations whose quotient is 0 in one iteration with divisions: in the
    second branch (d >= p, p < q: each d -= p, q -= p, u += v) r =
    min(floor(d/p), ceil(q/p) - 1, iterations left before u + v >= N); in
    the first (d < p, q < p: each p -= q, v += u) r = ceil((p - max(d, q))
    / q), the run ending earlier if u + v reaches N.  The states, hence d
    and u + v at the exit, are those of the plain loop; only the iteration
    count shrinks."""
    A %= M
    B %= M
    if A == 0:
        return B, 1, 0
    p, q, d, u, v = A, M - A, B, 1, 1
    it = 0
    while True:
        it += 1
        if specific and d < p and q < p:
            # a run of first-branch iterations with quotient 0: each p -= q,
            # v += u while p stays above both d and q
            r = (p - max(d, q) + q - 1) // q
            jx = 1 if u + v >= N else (N - v + u - 1) // u
            if jx <= r:
                return d, u + v + (jx - 1) * u, it
            p -= r * q
            v += r * u
        elif d < p:
            k = q // p
            q -= k * p
            u += k * v
            if u + v >= N:
                return d, u + v, it
            if q == 0:
                return d % p, u + v, it
            p -= q
            v += u
        elif specific and p < q:
            r = min(d // p, (q - 1) // p)
            jx = 1 if u + v >= N else (N - u - v + v - 1) // v + 1
            r = min(r, jx)
            d -= r * p
            if u + r * v >= N:
                return d, u + r * v, it
            q -= r * p
            u += r * v
        else:
            d -= p
            k = p // q
            p -= k * q
            v += k * u
            if u + v >= N:
                return d, u + v, it
            if p == 0:
                return d % q, u + v, it
            q -= p
            u += v


def lefevre_swap_lb(B: int, A: int, N: int, M: int = 1 << 64) -> Tuple[int, int, int]:
    """Algorithm 3: Algorithm 1 with its two branches merged by swapping
    (p, q) and (u, v) whenever b changes side (are_swapped), so that only
    the update of d stays conditional.  Reading of the printed listing
    (which subtracts and compares p in the swapped state, and then differs
    from Algorithm 1 on the first step of a = b): the length taken off d,
    and compared with d to decide the next swap, is Algorithm 1's p, which
    the swap has moved into q -- l = q when swapped, p otherwise.  Same
    (d, u+v, iterations) as lefevre_lb, same degenerate endings."""
    A %= M
    B %= M
    if A == 0:
        return B, 1, 0
    p, q, d, u, v = A, M - A, B, 1, 1
    sw = False
    if d >= p:
        p, q, u, v, sw = q, p, v, u, True
    it = 0
    while True:
        it += 1
        if sw:
            d -= q
        k = q // p
        q -= k * p
        u += k * v
        if u + v >= N:
            return d, u + v, it
        if q == 0:
            return d % p, u + v, it
        p -= q
        v += u
        if sw != (d >= (q if sw else p)):
            p, q, u, v, sw = q, p, v, u, not sw


def lefevre_test(B: int, A: int, N: int, eps: int, M: int = 1 << 64) -> bool:
    """Algorithm 1 as a Boolean test, returning at the first d < eps''
    (Failure, False) or at u + v >= N (Success, True); degenerate endings
    as in lefevre_lb."""
    A %= M
    B %= M
    if B < eps:
        return False
    if A == 0:
        return True
    p, q, d, u, v = A, M - A, B, 1, 1
    while True:
        if d < p:
            k = q // p
            q -= k * p
            u += k * v
            if u + v >= N:
                return True
            if q == 0:
                return d % p >= eps
            p -= q
            v += u
        else:
            d -= p
            if d < eps:
                return False
            k = p // q
            p -= k * q
            v += k * u
            if u + v >= N:
                return True
            if p == 0:
                return d % q >= eps
            q -= p
            u += v


def nmdm(iterations: List[int]) -> float:
    """Normalized mean deviation to the maximum of a warp's loop iteration
    counts (Sect. II-B): 1 - mean / max, the share of the warp's iterations
    a thread spends idle."""
    mx = max(iterations)
    return 0.0 if mx == 0 else 1.0 - (sum(iterations) / len(iterations)) / mx


def forward_differences(values: List[int]) -> List[List[int]]:
    """Rows Delta^0 .. Delta^n of the values (Def. of Delta, Fig. 5)."""
    rows = [list(values)]
    while len(rows[-1]) > 1:
        r = rows[-1]
        rows.append([r[i + 1] - r[i] for i in range(len(r) - 1)])
    return rows


def tabulated_shift(column: List[int], steps: int, mod: int = 0) -> List[List[int]]:
    """Columns [Delta^0(i), ..., Delta^g(i)] for i = 0 .. steps-1 from the
    column at i = 0, by Delta^(l-1)(i+1) = Delta^(l-1)(i) + Delta^l(i)
    (Sect. IV-B, Fig. 6); optionally reduced mod `mod`."""
    col = list(column)
    out = []
    for _ in range(steps):
        out.append(list(col))
        col = [col[l] + (col[l + 1] if l + 1 < len(col) else 0) for l in range(len(col))]
        if mod:
            col = [c % mod for c in col]
    return out


def straightforward_shift(column: List[int], n: int, mod: int = 0) -> List[int]:
    """The column at i = n directly: Delta^l(n) = sum_{k>=l} binom(n, k-l)
    Delta^k(0) (the upper-triangular Toeplitz binomial matrix of Sect. IV-B)."""
    g = len(column) - 1
    out = [sum(comb(n, k - l) * column[k] for k in range(l, g + 1)) for l in range(g + 1)]
    if mod:
        out = [c % mod for c in out]
    return out
