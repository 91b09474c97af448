"""GPU parity on the binade [128, 256) of exp, the second workload of
Sect. V (Table 7): exp is far from linear there, so the degree-1 lines'
truncation error dwarfs eps and the sound mode's first filter fails on
nearly every line.  Through the C ABI:

  * the literal-threshold search (range-reduced block coefficients on the
    device) reports exactly the oracle's brute-force list, fused and
    batched, across an output-binade cut, for exp and 2^x, up to the last
    binade [256, 512) below binary64's overflow of exp;
  * the sound mode reports exactly the oracle's Horner list, with the
    regular and with Lefevre's filter, in the fused, unfused and batched
    forms;
  * the counters show the heavy-failure regime (every line of a mid-binade
    slice fails the first filter), and the argument counts of phase 3's
    input and of its one-by-one evaluation cover every piece and sub-piece
    that holds a reported argument.
"""
import pytest

import workloads as wl
from oracle import candidates as oc
from oracle import plan, sound

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu

# first argument index with e(exp(X)) = 261 on [128, 256): X >= 260 ln 2
CUT_260 = 1837266934047447
# 2^x at X = 200 on [128, 256), p = 53
X_200 = 72 << 45


@pytest.fixture(scope="module")
def ctx():
    c = tmd.Context(0)
    yield c
    c.close()


LITERAL = [
    wl.Job(wl.FUNC_EXP, 8, 53, 20, 14, 3, 20, 3, CUT_260 - (1 << 23), 1 << 24),
    wl.Job(wl.FUNC_EXP2, 8, 53, 20, 12, 3, 18, 3, X_200 - (1 << 21) - 77, (1 << 22) + 555),
    wl.Job(wl.FUNC_EXP, 9, 53, 20, 14, 3, 20, 3, (1 << 52) - (1 << 24), 1 << 24),
    wl.Job(wl.FUNC_EXP, 3, 53, 20, 16, 3, 24, 3, 12345 << 24, 1 << 25, wl.FLAG_BP_DIRECTED),
]


@pytest.mark.parametrize("job", LITERAL, ids=lambda j: f"f{j.func}e{j.e_in}")
def test_literal_search_equals_oracle(ctx, job):
    want = oc.job_candidates(job, 0)
    assert len(want) > 0
    got, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 18)
    assert n == len(want) and got == want


def test_literal_batched_equals_oracle(ctx):
    d_cand, d_count = tmd.alloc_candidates(1 << 18)
    b = tmd.Batch(ctx, LITERAL, d_cand, d_count)
    b.launch()
    got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
    b.close()
    want = sorted([r for i, j in enumerate(LITERAL) for r in oc.job_candidates(j, i)],
                  key=lambda r: (r[0], r[2], r[3]))
    assert n == len(want) and got == want


# mid-binade slices (X near 208.25): generic slopes, every line fails the
# first filter.  Next to a cut (f(X) near a power of two) the slope is
# nearly an integer, the N points of a line cover a short arc only and most
# lines truly miss the window; there Lefevre's bound sees it and Algorithm 4
# (first partial quotient above N) does not -- parity only.
MID = 2823693648527360
SOUND = [
    wl.Job(wl.FUNC_EXP, 8, 53, 14, 14, 3, 20, 3, MID, 1 << 20),
    wl.Job(wl.FUNC_EXP2, 8, 53, 14, 14, 3, 20, 3, MID + 12345, (1 << 19) + 333),
]
SOUND_CUT = [
    wl.Job(wl.FUNC_EXP, 8, 53, 14, 14, 3, 20, 3, CUT_260 - (1 << 19), 1 << 20),
    wl.Job(wl.FUNC_EXP2, 8, 53, 14, 14, 3, 20, 3, X_200 - (1 << 18), (1 << 19) + 333),
]


def unit_args(job, records, level):
    """Arguments in the distinct phase-2 pieces (level 1: 32 per
    sub-interval) or phase-3 sub-pieces (level 2: 32 per piece of more than
    64 arguments) that hold a listed argument."""
    N = 1 << job.log2_N
    n2 = (N + 31) // 32
    n3 = (n2 + 31) // 32 if level == 2 and n2 > 64 else n2
    blocks = plan.blocks(job)
    units = set()
    total = 0
    for r in records:
        blk = next(b for b in blocks if b.first_sub <= r[1] < b.first_sub + (b.length + N - 1) // N)
        s0 = blk.start + (r[1] - blk.first_sub) * N
        s_len = min(N, blk.start + blk.length - s0)
        x = r[2] - s0
        px0 = x // n2 * n2
        pend = min(px0 + n2, s_len)
        u0 = px0 + (x - px0) // n3 * n3
        if (r[1], u0) not in units:
            units.add((r[1], u0))
            total += min(u0 + n3, pend) - u0
    return total


def check_phase_counts(st, job, records):
    assert unit_args(job, records, 1) <= st["refined_args"] <= job.count
    assert unit_args(job, records, 2) <= st["exhaustive_args"] <= st["refined_args"]


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "unfused"])
@pytest.mark.parametrize("lefevre", [False, True], ids=["regular", "lefevre"])
@pytest.mark.parametrize("job", SOUND, ids=lambda j: f"f{j.func}e{j.e_in}")
def test_sound_heavy_failure_equals_oracle(ctx, job, lefevre, fused):
    sj = tmd.sound_job(job.replace(flags=job.flags | (wl.FLAG_LEFEVRE if lefevre else 0)))
    # the regime: the first filter's threshold exceeds 1/(2N) of the unit
    assert sj.eps1 * 2 * (1 << job.log2_N) > 1 << 64
    want = sound.sound_candidates([sj], [sj.eps3])
    assert len(want) > 20
    got, n = tmd.run([sj], ctx=ctx, fused=fused, cap=1 << 18)
    assert n == len(want) and got == want
    st = tmd.tmd_stats_read(ctx)
    assert st["filter_fail"] >= 0.99 * st["lines"]
    check_phase_counts(st, job, want)


@pytest.mark.parametrize("job", SOUND_CUT, ids=lambda j: f"f{j.func}e{j.e_in}")
def test_sound_across_a_cut_equals_oracle(ctx, job):
    """Slices across an output-binade cut: same list with either filter;
    Lefevre's filter fails no more lines than Algorithm 4's."""
    want = None
    fails = []
    for flags in (0, wl.FLAG_LEFEVRE):
        sj = tmd.sound_job(job.replace(flags=job.flags | flags))
        if want is None:
            want = sound.sound_candidates([sj], [sj.eps3])
            assert len(want) > 20
        got, n = tmd.run([sj], ctx=ctx, fused=True, cap=1 << 18)
        assert n == len(want) and got == want
        fails.append(tmd.tmd_stats_read(ctx)["filter_fail"])
    assert fails[1] <= fails[0]


def test_sound_batched_with_literal_jobs(ctx):
    """Sound jobs of [128, 256) beside literal ones in one persistent launch."""
    jobs = [tmd.sound_job(SOUND_CUT[0]), LITERAL[0], tmd.sound_job(SOUND[1])]
    d_cand, d_count = tmd.alloc_candidates(1 << 18)
    b = tmd.Batch(ctx, jobs, d_cand, d_count)
    b.launch()
    got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
    st = b.stats()
    b.close()
    want_sound = sound.sound_candidates([jobs[0], jobs[2]], [jobs[0].eps3, jobs[2].eps3])
    remap = {0: 0, 1: 2}
    want = sorted([(remap[r[0]],) + r[1:] for r in want_sound] + oc.job_candidates(jobs[1], 1),
                  key=lambda r: (r[0], r[2], r[3]))
    assert n == len(want) and got == want
    for lv, key in ((1, "refined_args"), (2, "exhaustive_args")):
        assert st[key] >= (unit_args(SOUND_CUT[0], [r for r in want_sound if r[0] == 0], lv) +
                           unit_args(SOUND[1], [r for r in want_sound if r[0] == 1], lv))


def test_allocation_free_entry_equals_oracle():
    """The allocation-free entry (host-computed tables, anchored on the
    job's first block within one output binade) on [128, 256): a literal
    slice across the cut at 260 ln 2 and a sound slice across X = 200."""
    import numpy as np
    jobs = [LITERAL[0], tmd.sound_job(SOUND_CUT[1])]
    want = sorted(oc.job_candidates(jobs[0], 0) +
                  [(1,) + r[1:] for r in sound.sound_candidates([jobs[1]], [jobs[1].eps3])],
                  key=lambda r: (r[0], r[2], r[3]))
    d_cand, d_count = tmd.alloc_candidates(1 << 14)
    tmd.tmd_search_static(jobs, d_cand, d_count)
    torch.cuda.synchronize()
    n = int(d_count.cpu().item())
    raw = d_cand[: n * tmd.CANDIDATE_BYTES].cpu().numpy()
    rec = np.frombuffer(raw.tobytes(), dtype=np.dtype([("job", "<u4"), ("subint", "<u4"),
                                                      ("arg", "<u8"), ("value", "<u8")]))
    got = sorted(((int(r["job"]), int(r["subint"]), int(r["arg"]), int(r["value"])) for r in rec),
                 key=lambda r: (r[0], r[2], r[3]))
    assert n == len(want) and got == want


def test_full_size_sound_slice_sampled(ctx):
    """The benchmark's [128, 256) workload at full size in its launch form
    (2^36 arguments, sound (53, 2^-32), N = 2^16, one batched replay):
    every reported value is the oracle's (top64(R_t(y)) + eps3) mod 2^64 at
    that argument, and on whole Taylor blocks (2^20 arguments each: those of
    the first and last records and a seeded one) the records are exactly the
    oracle's list."""
    import random
    from oracle import poly
    start = random.Random(128256).randrange(0, (1 << 52) - (1 << 36), 1 << 20)
    job = tmd.sound_job(wl.Job(wl.FUNC_EXP, 8, 53, 32, 16, 3, 20, 3, start, 1 << 36))
    d_cand, d_count = tmd.alloc_candidates(1 << 16)
    b = tmd.Batch(ctx, [job], d_cand, d_count)
    b.launch()
    got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
    b.close()
    assert n == len(got) and 10 <= n <= 200
    T = 1 << job.log2_T
    W = 64 * job.limbs
    for r in got:
        b0 = r[2] - (r[2] - start) % T
        # e_out from the oracle's own exponent of f at the block start
        blk = plan.Block(b0, T, plan.e_out_at(job, b0), 0)
        c = poly.taylor_coeffs(job, blk)
        top = poly.horner(c, r[2] - blk.start, W) >> (W - 64)
        assert (top + job.eps3) % (1 << 64) == r[3] < 2 * job.eps3
    picks = {(got[0][2] - start) // T, (got[-1][2] - start) // T, random.Random(7).randrange(1 << 16)}
    for bi in sorted(picks):
        sub = job.replace(start=start + bi * T, count=T)
        want = sound.sound_candidates([sub], [job.eps3])
        got_b = [(0, r[2]) for r in got if start + bi * T <= r[2] < start + (bi + 1) * T]
        assert got_b == [(0, w[2]) for w in want]
