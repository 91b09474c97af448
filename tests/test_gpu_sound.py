"""GPU parity of the sound mode (Sect. II-A's eps'' filter, then Sect.
III-A's exhaustive phase) through the C ABI: the reported arguments and
values equal the oracle's Horner definition exactly, in the fused, unfused,
batched and allocation-free forms, every argument decided hard-to-round from the
exact function is among them, and Table 2's count of (53, 2^-32)
hard-to-round cases of exp on [1, 1+2^-13[ is compared with the exact
decision of every listed argument."""
from fractions import Fraction

import pytest

import workloads as wl
from oracle import sound

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = tmd.Context(0)
    yield c
    c.close()


# exact decisions in the 2^-31 list of Table 2's domain: arguments whose
# exp comes within 1.01 x 2^-32 of a binary64 number (241 below 2^-32)
TABLE2_WITHIN_1_01 = 243

SMALL = [
    wl.Job(wl.FUNC_EXP, 0, 24, 10, 8, 2, 12, 1, 3 << 20, 1 << 13),
    wl.Job(wl.FUNC_EXP2, 1, 22, 7, 7, 3, 11, 1, 12345, 1 << 11, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_LOG, 2, 20, 8, 6, 2, 10, 1, 100, 1 << 12),
    wl.Job(wl.FUNC_EXP, 0, 20, 7, 6, 2, 10, 2, 0, 1 << 19),                  # cut at ln 2, W = 128
    wl.Job(wl.FUNC_EXP, 0, 53, 14, 14, 3, 24, 3, wl.plain_start(), 1 << 20),   # binary64, W = 192
    wl.Job(wl.FUNC_LOG, 2, 53, 13, 16, 2, 18, 3, 0x3243F6A8885A3, (1 << 19) + 333),  # N = 2^16, ragged end
]


def oracle_list(jobs):
    return sound.sound_candidates(jobs, [j.eps3 for j in jobs])


@pytest.mark.parametrize("job", SMALL, ids=lambda j: f"f{j.func}p{j.p}N{j.log2_N}")
def test_sound_fused_equals_oracle(ctx, job):
    sj = tmd.sound_job(job)
    want = oracle_list([sj])
    assert len(want) > 0
    got, n = tmd.run([sj], ctx=ctx, fused=True, cap=1 << 18)
    assert n == len(want) and got == want


def test_sound_batched_mixed_equals_oracle(ctx):
    """Sound and ordinary jobs in one persistent launch."""
    jobs = [tmd.sound_job(SMALL[0]), SMALL[2], tmd.sound_job(SMALL[4]), tmd.sound_job(SMALL[1])]
    d_cand, d_count = tmd.alloc_candidates(1 << 18)
    b = tmd.Batch(ctx, jobs, d_cand, d_count)
    b.launch()
    got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
    b.close()
    from oracle import candidates as oc
    want_sound = oracle_list([jobs[0], jobs[2], jobs[3]])
    remap = {0: 0, 1: 2, 2: 3}
    want = sorted([(remap[r[0]],) + r[1:] for r in want_sound] + oc.job_candidates(jobs[1], 1),
                  key=lambda r: (r[0], r[2], r[3]))
    assert n == len(want) and got == want


def test_sound_allocation_free_entry_equals_oracle():
    """The allocation-free entry (plan in the library's fixed device array,
    tables and coefficients by the host) gives the same sound list."""
    jobs = [tmd.sound_job(SMALL[0]), tmd.sound_job(SMALL[2])]
    want = oracle_list(jobs)
    import numpy as np
    d_cand, d_count = tmd.alloc_candidates(1 << 12)
    tmd.tmd_search_static(jobs, d_cand, d_count)
    torch.cuda.synchronize()
    n = int(d_count.cpu().item())
    raw = d_cand[: n * tmd.CANDIDATE_BYTES].cpu().numpy()
    rec = np.frombuffer(raw.tobytes(), dtype=np.dtype([("job", "<u4"), ("subint", "<u4"),
                                                      ("arg", "<u8"), ("value", "<u8")]))
    got = sorted(((int(r["job"]), int(r["subint"]), int(r["arg"]), int(r["value"])) for r in rec),
                 key=lambda r: (r[0], r[2], r[3]))
    assert n == len(want) and got == want


def test_sound_list_holds_every_hard_to_round_argument(ctx):
    job = tmd.sound_job(SMALL[0])
    got, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 16)
    listed = {r[2] for r in got}
    plain = SMALL[0]
    hr = [j for j in range(plain.start, plain.start + plain.count) if sound.is_hard_to_round(plain, j)]
    assert len(hr) > 10 and set(hr) <= listed


def test_sound_unfused_pair_equals_oracle(ctx):
    """tmd_generate writes the lines, tmd_search searches them: sound jobs of
    different (limbs, degree) next to an ordinary job, so that warps of the
    line search straddle jobs, give the oracle's lists."""
    jobs = [tmd.sound_job(SMALL[0]), SMALL[2], tmd.sound_job(SMALL[3]), tmd.sound_job(SMALL[1]),
            tmd.sound_job(SMALL[4])]
    got, n = tmd.run(jobs, ctx=ctx, fused=False, cap=1 << 18)
    from oracle import candidates as oc
    sound_idx = [0, 2, 3, 4]
    want_sound = oracle_list([jobs[i] for i in sound_idx])
    want = sorted([(sound_idx[r[0]],) + r[1:] for r in want_sound] + oc.job_candidates(jobs[1], 1),
                  key=lambda r: (r[0], r[2], r[3]))
    assert n == len(want) and got == want


def test_table2_hard_to_round_cases_of_exp(ctx):
    """Table 2: the (53, 2^-32) hard-to-round cases of exp in [1, 1+2^-13[
    -- 2^39 binary64 arguments, breakpoints the binary64 numbers (Def. 3,
    directed rounding, Sect. V) -- are printed as 243.  The sound path lists
    every argument within eps3 of a breakpoint on the block polynomials and
    each listed argument is decided exactly from enclosures of exp: there
    are exactly 241.  The next arguments lie just above 2^-32 (0.16 % and
    1.0 % above it), so a count taken with a threshold about 1 % above
    2^-32 (an approximation error left in the paper's last check) gives the
    printed 243.  With the threshold 2^-31 every argument below
    1.01 x 2^-32 is listed, and the count in that window is pinned too."""
    job = tmd.sound_job(wl.Job(wl.FUNC_EXP, 1, 53, 32, 15, 3, 24, 3, 0, 1 << 39, wl.FLAG_BP_DIRECTED))
    got, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 16)
    assert n == len(got) < 1 << 16
    plain = job.replace(flags=wl.FLAG_BP_DIRECTED, eps1=0, eps3=0)
    hr = [r[2] for r in got if sound.is_hard_to_round(plain, r[2])]
    print("listed", n, "hard-to-round", len(hr))
    assert len(hr) == 241
    wide = tmd.sound_job(plain.replace(m=31))
    got31, n31 = tmd.run([wide], ctx=ctx, fused=True, cap=1 << 16)
    assert set(hr) <= {r[2] for r in got31}
    dist = sorted(float(sound.distance(plain, r[2])[1] * (1 << 32)) for r in got31)
    above = [x for x in dist if x >= 1.0][:4]
    near = [x for x in dist if x < 1.01]
    print("within 1.01 x 2^-32:", len(near), "next distances / 2^-32:", above)
    assert len([x for x in dist if x < 1.0]) == 241
    assert len(near) == TABLE2_WITHIN_1_01
