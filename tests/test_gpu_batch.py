"""GPU parity of the batched form: one persistent, graph-captured launch over
uneven mixed jobs gives the oracle's candidate list, replay after replay, and
the same records as the per-job plain launches."""
import pytest

import workloads as wl
from oracle import candidates as oc

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = tmd.Context(0)
    yield c
    c.close()


MIXED = [
    wl.Job(wl.FUNC_EXP2, 1, 24, 16, 8, 2, 12, 1, 0, 1 << 16),
    wl.Job(wl.FUNC_LOG, 2, 30, 14, 8, 3, 14, 2, 12345, 1 << 20),
    wl.Job(wl.FUNC_EXP, 0, 53, 20, 14, 3, 24, 3, wl.plain_start(), 1 << 26),
    wl.Job(wl.FUNC_EXP, 1, 53, 18, 12, 4, 20, 3, 7 << 40, (1 << 24) + 777),
    wl.Job(wl.FUNC_LOG, 3, 28, 14, 6, 2, 10, 1, 1 << 25, 1 << 21, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_EXP2, 0, 53, 22, 16, 1, 18, 2, 5 << 30, 1 << 24),
    wl.toy_job(),
]


def batch_records(b, d_cand, d_count):
    recs, n = tmd.tmd_candidates(b.ctx, d_cand, d_count)
    return recs, n


def test_batch_matches_oracle_over_replays(ctx):
    want = oc.candidates(MIXED)
    d_cand, d_count = tmd.alloc_candidates(1 << 16)
    b = tmd.Batch(ctx, MIXED, d_cand, d_count)
    for _ in range(3):
        b.launch()
        got, n = batch_records(b, d_cand, d_count)
        assert n == len(want)
        assert got == want
    st = b.stats()
    assert st["lines"] == sum(__import__("oracle").plan.n_subintervals(j) for j in MIXED)
    b.close()


def test_batch_equals_plain_per_job(ctx):
    jobs = wl.batched_jobs(njobs=6, m=24, size_log2_range=(24.0, 27.0))
    d_cand, d_count = tmd.alloc_candidates(1 << 18)
    b = tmd.Batch(ctx, jobs, d_cand, d_count)
    b.launch()
    got, n = batch_records(b, d_cand, d_count)
    b.close()
    plain = []
    for j, job in enumerate(jobs):
        recs, _ = tmd.run([job], ctx=ctx, fused=True, cap=1 << 18)
        plain.extend((j,) + r[1:] for r in recs)
    plain.sort(key=lambda r: (r[0], r[2], r[3]))
    assert got == plain and n == len(plain)
    # and one job of the batch against the oracle in full
    k = min(range(len(jobs)), key=lambda i: jobs[i].count)
    want = oc.job_candidates(jobs[k], k)
    assert [r for r in got if r[0] == k] == sorted(want, key=lambda r: (r[0], r[2], r[3]))


def test_large_batch_sample_exact(ctx):
    """The first 256 jobs of the large 2^x batch (uneven sizes, N = 2^16,
    192-bit words) at the m = 22 twin in one persistent launch; sampled jobs
    record by record against the oracle, all counts consistent."""
    jobs = [j.replace(m=22) for j in wl.large_jobs()[:256]]
    d_cand, d_count = tmd.alloc_candidates(1 << 16)
    b = tmd.Batch(ctx, jobs, d_cand, d_count)
    b.launch()
    got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
    b.close()
    assert n == len(got) > 500
    import random
    rng = random.Random(4)
    for k in sorted(rng.sample(range(len(jobs)), 12)) + [0, 255]:
        want = oc.job_candidates(jobs[k], k)
        assert [r for r in got if r[0] == k] == sorted(want, key=lambda r: (r[0], r[2], r[3])), k


@pytest.mark.parametrize("tiling", [(8, 1), (6, 2), (4, 3), (2, 1), (1, 2), (3, 0), (8, 3, 2, 1), (8, 2, 4, 2),
                                    (6, 3, 2, 2), (1, 1, 4, 1), (5, 0, 1, 2), (8, 0, 4, 0)])
def test_every_tiling_gives_the_oracle_list(ctx, tiling):
    """The tiling only changes how the work is cut (packet length, resident
    CTAs, lanes per line in the filter, difference steps per iteration),
    never the records."""
    want = oc.candidates(MIXED)
    d_cand, d_count = tmd.alloc_candidates(1 << 16)
    b = tmd.Batch(ctx, MIXED, d_cand, d_count, tiling=tiling)
    b.launch()
    got, n = batch_records(b, d_cand, d_count)
    nu, per_sm, lanes, unroll = b.tiling()
    st = b.stats()
    b.close()
    assert got == want and n == len(want)
    assert nu == tiling[0]
    assert per_sm >= 1 and (tiling[1] == 0 or per_sm <= tiling[1])
    t = tuple(tiling) + (0, 0)
    assert lanes == (t[2] or 1) and unroll == (t[3] or 1)
    assert st["lines"] == sum(__import__("oracle").plan.n_subintervals(j) for j in MIXED)


def test_autotune_picks_a_valid_tiling_and_batches_use_it(ctx):
    jobs = wl.batched_jobs(njobs=6, m=24, size_log2_range=(24.0, 27.0))
    best = tmd.tmd_autotune(ctx, jobs)
    assert best["nu"] in (1, 2, 4, 6, 8) and best["ctas_per_sm"] >= 1 and best["ms"] > 0
    assert best["lanes"] in (1, 2, 4) and best["unroll"] in (1, 2)
    d_cand, d_count = tmd.alloc_candidates(1 << 18)
    b = tmd.Batch(ctx, jobs, d_cand, d_count)      # takes the tuned tiling
    nu, per_sm, lanes, unroll = b.tiling()
    assert 1 <= nu <= best["nu"] and 1 <= per_sm <= best["ctas_per_sm"]
    assert (lanes, unroll) == (best["lanes"], best["unroll"])
    b.launch()
    got, n = batch_records(b, d_cand, d_count)
    b.close()
    ref = tmd.Batch(ctx, jobs, d_cand, d_count, tiling=(8, 0))
    ref.launch()
    want, m = batch_records(ref, d_cand, d_count)
    ref.close()
    assert got == want and n == m
