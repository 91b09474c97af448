"""GPU parity of the search stage through the C ABI: the Algorithm 4 lower
bound value by value, and candidate lists record by record against brute
force, on random and degenerate lines."""
import random

import pytest

from gpu_util import to_u32_list, to_u64_list, u32_tensor, u64_tensor
from oracle import candidates as oc
from oracle import search
import workloads as wl

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def ctx():
    c = tmd.Context(0)
    yield c
    c.close()


def edge_lines():
    """Degenerate lines: a = 0, powers of two (the expansion ends), tiny a
    (huge first quotient: exact slow division), a near 1, b = 0, N = 1."""
    out = []
    for A in [0, 1, 2, 3, 1 << 20, 1 << 44, 1 << 63, M64, M64 - 1, (1 << 63) + 1, 12345,
              0x9E3779B97F4A7C15, 1 << 62, 3 << 61, 0x5555555555555555]:
        for B in [0, 1, M64, 1 << 63, 0x243F6A8885A308D3]:
            for n in [1, 2, 31, 32, 33, 1000, 1 << 14, 1 << 16]:
                out.append((B, A, n))
    return out


def random_lines(n, seed):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        kind = rng.random()
        if kind < 0.7:
            A = rng.getrandbits(64)
        elif kind < 0.85:
            A = rng.getrandbits(rng.randrange(1, 64))       # small a: large quotients
        else:
            A = M64 - rng.getrandbits(rng.randrange(1, 64))  # a near 1
        out.append((rng.getrandbits(64), A, rng.choice([1, 7, 64, 256, 1000, 1 << 12, 1 << 14, 1 << 16])))
    return out


def run_lower_bounds(ctx, lines):
    B = u64_tensor([l[0] for l in lines])
    A = u64_tensor([l[1] for l in lines])
    n = u32_tensor([l[2] for l in lines])
    lb = torch.empty_like(B)
    hs = torch.empty_like(n)
    tmd.tmd_lower_bounds(ctx, B, A, n, lb, hs)
    torch.cuda.synchronize()
    return to_u64_list(lb), to_u32_list(hs)


def test_lower_bound_equals_algorithm4_edges(ctx):
    lines = edge_lines()
    lb, hs = run_lower_bounds(ctx, lines)
    for (B, A, n), g, h in zip(lines, lb, hs):
        want, _, whs = search.regular_lb_unrolled(B, A, n)
        assert (g, h) == (want, whs), (hex(B), hex(A), n)


def test_lower_bound_equals_algorithm4_random(ctx):
    lines = random_lines(20000, 5)
    lb, hs = run_lower_bounds(ctx, lines)
    for (B, A, n), g, h in zip(lines, lb, hs):
        want, _, whs = search.regular_lb_unrolled(B, A, n)
        assert (g, h) == (want, whs), (hex(B), hex(A), n)


def clustered_lines(n_warps, seed):
    """Warps of 32 lines whose slopes lie close together, as neighbouring
    sub-intervals of one job do (their continued fractions share all but
    the last partial quotients): spreads from 0 to the whole circle, slopes
    near 0 (huge first quotient) and with trailing zero bits (the expansion
    ends early), shuffled lanes, equal and mixed lengths, and a zero slope
    among close ones."""
    rng = random.Random(seed)
    out = []
    for w in range(n_warps):
        kind = w % 8
        A0 = rng.getrandbits(64)
        if kind == 5:
            A0 = rng.getrandbits(rng.randrange(1, 50))
        spread = rng.choice([0, 1, 1 << rng.randrange(0, 48), rng.getrandbits(rng.randrange(1, 64))])
        As = [(A0 + l * spread) & M64 for l in range(32)]
        if kind == 4:
            z = rng.randrange(0, 60)
            As = [a & ~((1 << z) - 1) & M64 for a in As]
        if kind == 6:
            rng.shuffle(As)
        if kind == 7:
            As[rng.randrange(32)] = 0
        mode = rng.randrange(4)
        if mode == 0:
            ns = [1 << 14] * 32
        elif mode == 1:
            ns = [rng.choice([1, 2, 3, 100, 4096, 1 << 14, 1 << 16]) for _ in range(32)]
        elif mode == 2:
            ns = [1 << 16] * 31 + [rng.randrange(1, 1 << 16)]
        else:
            ns = [rng.choice([1 << 12, 1 << 16])] * 32
        out += [(rng.getrandbits(64), a, nn) for a, nn in zip(As, ns)]
    return out


def test_lower_bound_equals_algorithm4_clustered(ctx):
    lines = clustered_lines(1500, 17)
    lb, hs = run_lower_bounds(ctx, lines)
    for (B, A, n), g, h in zip(lines, lb, hs):
        want, _, whs = search.regular_lb_unrolled(B, A, n)
        assert (g, h) == (want, whs), (hex(B), hex(A), n)


@pytest.mark.parametrize("job", [
    wl.plain_job(m=40, count_log2=30),
    wl.Job(wl.FUNC_LOG, 3, 53, 40, 16, 2, 18, 3, 1 << 44, 1 << 30),
    wl.Job(wl.FUNC_EXP2, 1, 53, 40, 12, 3, 24, 3, 3 << 48, 1 << 28),
], ids=["exp-N14", "log-N16", "exp2-N12"])
def test_lower_bound_on_generated_lines(ctx, job):
    """Lines of real jobs, generated on the device: bound and half-step
    count compared line by line with Algorithm 4 on a sample of warps."""
    need = tmd.tmd_generate(ctx, [job], None)
    d_lin = torch.empty(need // 8, dtype=torch.int64, device="cuda:0")
    tmd.tmd_generate(ctx, [job], d_lin)
    half = d_lin.numel() // 2
    B, A = d_lin[:half].contiguous(), d_lin[half:].contiguous()
    n = torch.full((half,), 1 << job.log2_N, dtype=torch.int32, device="cuda:0")
    lb = torch.empty_like(B)
    hs = torch.empty_like(n)
    tmd.tmd_lower_bounds(ctx, B, A, n, lb, hs)
    Bh, Ah = to_u64_list(B), to_u64_list(A)
    lbh, hsh = to_u64_list(lb), to_u32_list(hs)
    rng = random.Random(job.count)
    for w in rng.sample(range(half // 32), 300):
        for s in range(32 * w, 32 * w + 32):
            want, _, whs = search.regular_lb_unrolled(Bh[s], Ah[s], 1 << job.log2_N)
            assert (lbh[s], hsh[s]) == (want, whs), s


def brute_records(lines, m, all_hits=False):
    import numpy as np
    T = 1 << (65 - m)
    B = np.array([l[0] for l in lines], dtype=np.uint64)
    A = np.array([l[1] for l in lines], dtype=np.uint64)
    n = np.array([l[2] for l in lines], dtype=np.uint32)
    if all_hits:
        recs = [(0, i, x, v) for (i, x, v) in oc.brute_hits_many(B, A, n, T)]
    else:
        mins, args = oc.brute_min_many(B, A, n)
        recs = [(0, i, int(args[i]), int(mins[i])) for i in range(len(lines)) if int(mins[i]) < T]
    return sorted(recs, key=lambda r: (r[0], r[2], r[3]))


def sort_by_line(recs):
    return sorted(recs, key=lambda r: (r[1], r[2], r[3]))


@pytest.mark.parametrize("m", [2, 6, 10, 20])
def test_search_lines_match_brute_force(ctx, m):
    lines = random_lines(3000, 100 + m) + edge_lines()
    B = u64_tensor([l[0] for l in lines])
    A = u64_tensor([l[1] for l in lines])
    n = u32_tensor([l[2] for l in lines])
    d_cand, d_count = tmd.alloc_candidates(len(lines) + 16)
    tmd.tmd_search_lines(ctx, B, A, n, m, 0, d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    want = brute_records(lines, m)
    assert count == len(want)
    assert sort_by_line(got) == sort_by_line(want)
    st = tmd.tmd_stats_read(ctx)
    assert st["lines"] == len(lines)
    # the filter flags exactly the lines whose Algorithm 4 bound is below T_m
    T = 1 << (65 - m)
    flagged = sum(1 for (Bv, Av, nv) in lines if search.regular_lb_unrolled(Bv, Av, nv)[0] < T)
    assert st["filter_fail"] == flagged


def exact_min_hard_lines(seed):
    """Lines for the exact minimum: slopes with every count of trailing zero
    bits (periodic point sets, tied minima: the smallest argmin is the
    reported one), tiny slopes (huge quotients in the recursion), slopes
    next to 2^64, and the extreme offsets, at the longest length."""
    rng = random.Random(seed)
    out = []
    for t in range(64):
        for _ in range(3):
            A = ((rng.getrandbits(64 - t) | 1) << t) & M64
            out.append((rng.getrandbits(64), A, rng.choice([1 << 16, 1 << 14, 777, 2])))
    for A in list(range(1, 40)) + [M64 - k for k in range(40)] + [1 << 32, (1 << 32) + 1, 3 << 62]:
        out.append((rng.choice([0, 1, M64, rng.getrandbits(64)]), A, 1 << 16))
    return out


def test_exact_minimum_on_hard_lines(ctx):
    """m = 2 flags nearly every line, so every line goes through the exact
    minimum; records must equal brute force (value and smallest argmin)."""
    lines = exact_min_hard_lines(11)
    B = u64_tensor([l[0] for l in lines])
    A = u64_tensor([l[1] for l in lines])
    n = u32_tensor([l[2] for l in lines])
    d_cand, d_count = tmd.alloc_candidates(len(lines) + 16)
    tmd.tmd_search_lines(ctx, B, A, n, 2, 0, d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    want = brute_records(lines, 2)
    assert count == len(want) > 0.8 * len(lines)
    assert sort_by_line(got) == sort_by_line(want)


def test_search_lines_all_hits(ctx):
    rng = random.Random(9)
    lines = [(rng.getrandbits(64), rng.getrandbits(64), rng.choice([100, 4096, 65536])) for _ in range(400)]
    lines += [(5, 1 << 60, 64), (0, 0, 100), (7, 1 << 63, 1000)]     # ties and repeated values
    B = u64_tensor([l[0] for l in lines])
    A = u64_tensor([l[1] for l in lines])
    n = u32_tensor([l[2] for l in lines])
    d_cand, d_count = tmd.alloc_candidates(1 << 16)
    tmd.tmd_search_lines(ctx, B, A, n, 12, tmd.TMD_ALL_HITS, d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    want = brute_records(lines, 12, all_hits=True)
    assert count == len(want)
    assert sort_by_line(got) == sort_by_line(want)


def test_overflow_keeps_exact_count(ctx):
    rng = random.Random(3)
    lines = [(rng.getrandbits(64), rng.getrandbits(64), 4096) for _ in range(2000)]
    B = u64_tensor([l[0] for l in lines])
    A = u64_tensor([l[1] for l in lines])
    n = u32_tensor([l[2] for l in lines])
    want = brute_records(lines, 6)
    d_cand, d_count = tmd.alloc_candidates(10)
    tmd.tmd_search_lines(ctx, B, A, n, 6, 0, d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    assert count == len(want) > 10
    assert len(got) == 10 and set(got) <= set(want)


def test_empty_input(ctx):
    B = torch.empty(0, dtype=torch.int64, device="cuda:0")
    d_cand, d_count = tmd.alloc_candidates(4)
    tmd.tmd_search_lines(ctx, B, B, torch.empty(0, dtype=torch.int32, device="cuda:0"), 20, 0,
                         d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    assert got == [] and count == 0


def test_bad_lengths_reported(ctx):
    B = u64_tensor([1, 2, 3])
    n = u32_tensor([5, 0, 70000])
    d_cand, d_count = tmd.alloc_candidates(4)
    tmd.tmd_search_lines(ctx, B, B, n, 20, 0, d_cand, d_count)
    with pytest.raises(tmd.TmdError):
        tmd.tmd_candidates(ctx, d_cand, d_count)


def narrow_lines(w, ns):
    """Every (A, B) of w-bit words at each length in ns, placed at the top of
    the 64-bit words: (B 2^s - A 2^s x) mod 2^64 = 2^s ((B - A x) mod 2^w)
    with s = 64 - w, so the 64-bit kernels run w-bit arithmetic exactly."""
    s = 64 - w
    return [(b << s, a << s, n) for a in range(1 << w) for b in range(1 << w) for n in ns]


def test_exhaustive_narrow_words(ctx):
    """All 8-bit (A, B) at seven lengths (every rational slope, tie and
    degenerate ending of that width): the Algorithm 4 bound and half-step
    count equal the oracle's line by line and never exceed the brute-force
    minimum, and the search's records (minimum below 2^63) are brute
    force's, smallest argmin included."""
    import numpy as np
    lines = narrow_lines(8, [1, 2, 3, 16, 100, 256, 1000])
    lb, hs = run_lower_bounds(ctx, lines)
    mins, _ = oc.brute_min_many(np.array([l[0] for l in lines], dtype=np.uint64),
                                np.array([l[1] for l in lines], dtype=np.uint64),
                                np.array([l[2] for l in lines], dtype=np.uint32))
    for (B, A, n), g, h, mn in zip(lines, lb, hs, mins):
        want, _, whs = search.regular_lb_unrolled(B, A, n)
        assert (g, h) == (want, whs), (hex(B), hex(A), n)
        assert g <= int(mn)
    d_cand, d_count = tmd.alloc_candidates(len(lines) + 16)
    tmd.tmd_search_lines(ctx, u64_tensor([l[0] for l in lines]), u64_tensor([l[1] for l in lines]),
                         u32_tensor([l[2] for l in lines]), 2, 0, d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    want = brute_records(lines, 2)
    assert count == len(want) > 100000
    assert sort_by_line(got) == sort_by_line(want)


def test_exhaustive_narrow_words_all_hits(ctx):
    """All 6-bit (A, B) at three lengths, every argument below 2^61
    reported (all-hits mode) against brute force."""
    lines = narrow_lines(6, [1, 7, 64])
    d_cand, d_count = tmd.alloc_candidates(1 << 19)
    tmd.tmd_search_lines(ctx, u64_tensor([l[0] for l in lines]), u64_tensor([l[1] for l in lines]),
                         u32_tensor([l[2] for l in lines]), 4, tmd.TMD_ALL_HITS, d_cand, d_count)
    got, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    want = brute_records(lines, 4, all_hits=True)
    assert count == len(want) > 10000
    assert sort_by_line(got) == sort_by_line(want)
