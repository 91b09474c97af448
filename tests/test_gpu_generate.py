"""GPU parity of the generation stage and of the whole path (through the C
ABI) against the oracle: search words of every sub-interval, and candidate
lists record by record, fused and unfused."""
import random

import numpy as np
import pytest

import workloads as wl
from oracle import candidates as oc
from oracle import plan

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = tmd.Context(0)
    yield c
    c.close()


def generated_words(ctx, jobs):
    need = tmd.tmd_generate(ctx, jobs, None)
    d_lin = torch.empty(need // 8, dtype=torch.int64, device="cuda:0")
    tmd.tmd_generate(ctx, jobs, d_lin)
    torch.cuda.synchronize()
    w = d_lin.cpu().numpy().view(np.uint64)
    half = len(w) // 2
    return w[:half], w[half:]


GEN_JOBS = [
    wl.toy_job(),
    wl.Job(wl.FUNC_EXP2, 1, 24, 16, 8, 2, 12, 1, 0, 1 << 16),
    wl.Job(wl.FUNC_LOG, 2, 30, 20, 8, 3, 14, 2, 12345, 1 << 22),          # W=128, ragged start
    wl.Job(wl.FUNC_EXP, 0, 53, 40, 14, 3, 24, 3, wl.plain_start(), 1 << 28),
    wl.Job(wl.FUNC_EXP, 1, 53, 30, 12, 4, 20, 3, 7 << 40, (1 << 26) + 777),  # d=4, ragged end
    wl.Job(wl.FUNC_EXP2, 0, 53, 42, 16, 1, 18, 2, 5 << 30, 1 << 24),         # d=1
    wl.Job(wl.FUNC_EXP, 2, 40, 30, 10, 2, 16, 2, 0, 1 << 39),                # three cuts
]


@pytest.mark.parametrize("job", GEN_JOBS, ids=lambda j: f"f{j.func}e{j.e_in}p{j.p}d{j.d}L{j.limbs}")
def test_generated_words_match_oracle_horner(ctx, job):
    B, A = generated_words(ctx, [job])
    blocks = plan.blocks(job)
    assert len(B) == plan.n_subintervals(job)
    rng = random.Random(job.count)
    picks = sorted(set([0, len(blocks) - 1] + [rng.randrange(len(blocks)) for _ in range(12)]))
    for b in picks:
        blk = blocks[b]
        _, ob, oa, _ = oc.block_lines(job, blk)
        s = blk.first_sub
        assert list(B[s:s + len(ob)]) == list(ob), (b,)
        assert list(A[s:s + len(oa)]) == list(oa), (b,)


def test_batch_words_in_job_order(ctx):
    jobs = [GEN_JOBS[1], GEN_JOBS[2], GEN_JOBS[5]]
    B, A = generated_words(ctx, jobs)
    off = 0
    for job in jobs:
        blk = plan.blocks(job)[-1]
        _, ob, oa, _ = oc.block_lines(job, blk)
        s = off + blk.first_sub
        assert list(B[s:s + len(ob)]) == list(ob)
        assert list(A[s:s + len(oa)]) == list(oa)
        off += plan.n_subintervals(job)
    assert off == len(B)


def test_table_forms_agree_and_match_oracle(ctx):
    """Plans of up to 16 k blocks build their tables with four threads per
    block, larger plans with one thread per block: the same jobs give the
    same words in both.  The small plan mixes the three functions with a
    block count that leaves warps partly filled (lanes of other functions
    and past the plan's end share warps with working ones) and is checked
    against the oracle too."""
    small = [GEN_JOBS[1], GEN_JOBS[2],
             wl.Job(wl.FUNC_EXP, 0, 53, 40, 14, 3, 24, 3, wl.plain_start(), 5 << 24), GEN_JOBS[4]]
    big = wl.Job(wl.FUNC_EXP2, 0, 53, 40, 8, 2, 12, 1, 3 << 36, 1 << 27)    # 32768 blocks
    n_small = sum(len(plan.blocks(j)) for j in small)
    assert n_small <= 16384 and n_small % 8 != 0
    assert n_small + len(plan.blocks(big)) > 16384
    B1, A1 = generated_words(ctx, small)
    B2, A2 = generated_words(ctx, small + [big])
    n = len(B1)
    assert (B2[:n] == B1).all() and (A2[:n] == A1).all()
    off = 0
    for job in small + [big]:
        blocks = plan.blocks(job)
        for b in sorted({0, len(blocks) - 1}):
            _, ob, oa, _ = oc.block_lines(job, blocks[b])
            s = off + blocks[b].first_sub
            assert list(B2[s:s + len(ob)]) == list(ob), (job, b)
            assert list(A2[s:s + len(oa)]) == list(oa), (job, b)
        off += plan.n_subintervals(job)
    assert off == len(B2)


@pytest.mark.parametrize("fused", [True, False])
def test_toy_candidates_exact(ctx, fused):
    job = wl.toy_job()
    got, n = tmd.run([job], ctx=ctx, fused=fused, cap=1 << 14)
    want = oc.candidates([job])
    assert n == len(want) == len(got)
    assert got == want


def test_toy_all_hits_exact(ctx):
    job = wl.toy_job(flags=wl.FLAG_ALL_HITS)
    got, n = tmd.run([job], ctx=ctx, cap=1 << 14)
    want = oc.candidates([job])
    assert got == want and n == len(want)


def test_small_jobs_mixed_batch_exact(ctx):
    jobs = [
        wl.Job(wl.FUNC_EXP2, 1, 24, 16, 8, 2, 12, 1, 0, 1 << 16),             # planted x = 0 hit
        wl.Job(wl.FUNC_LOG, 2, 30, 14, 8, 3, 14, 2, 12345, 1 << 20),
        wl.Job(wl.FUNC_EXP, 0, 53, 20, 14, 3, 24, 3, wl.plain_start(), 1 << 26),
        wl.Job(wl.FUNC_EXP, 1, 53, 18, 12, 4, 20, 3, 7 << 40, (1 << 24) + 777),
        wl.Job(wl.FUNC_LOG, 3, 28, 14, 6, 2, 10, 1, 1 << 25, 1 << 21, wl.FLAG_BP_DIRECTED),
    ]
    want = oc.candidates(jobs)
    for fused in (True, False):
        got, n = tmd.run(jobs, ctx=ctx, fused=fused, cap=1 << 16)
        assert n == len(want)
        assert got == want
    assert want[0][:3] == (0, 0, 0)            # the exact point 2^1 = 2


def test_plain_dense_twin_sampled_blocks(ctx):
    """The binary64 plain workload (2^36 arguments, d=3, 192-bit words,
    N=2^14) at m=20, in the fused launch the benchmark times; sampled blocks
    are compared record by record with the oracle."""
    job = wl.plain_job(m=20)
    got, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 20)
    assert n == len(got)
    blocks = plan.blocks(job)
    rng = random.Random(20)
    picks = sorted(set([0, len(blocks) - 1] + rng.sample(range(len(blocks)), 24)))
    by_block = {}
    for r in got:
        b = (r[2] - job.start) >> job.log2_T
        by_block.setdefault(b, []).append(r)
    for b in picks:
        want = oc.job_candidates(job, blocks=[blocks[b]])
        assert sorted(by_block.get(b, [])) == sorted(want), b
    # density check: about 2^22 (1 - exp(-2^14 2^-19)) ~ 1.3e5 sub-intervals
    assert 1.1e5 < n < 1.5e5
