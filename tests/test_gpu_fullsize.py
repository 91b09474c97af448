"""Bit-exact parity at the benchmark workloads' full sizes.

The batched form the benchmark times (persistent work-queue kernel replayed
as a CUDA graph, tiling picked by tmd_autotune) runs each workload whole,
and its sorted records are compared, record by record, with the CPU
oracle's (Eq. (1) by definition: correctly rounded Taylor coefficients,
direct Horner lines, brute force over every argument; tests/oracle_pool.py
spreads the oracle's blocks over the host cores).  Integer results, so the
tolerance is zero.

  * exp on the 2^36-argument binary64 slice of [1/2, 1) (d = 3, W = 192,
    N = 2^14): in full at m = 40 and at its dense twin m = 20;
  * the 64-job mixed batch (exp, 2^x, log on six binades, d in {2, 3},
    N in {2^12, 2^14, 2^16}, 2.2e11 arguments) at its m = 20 twin, every
    job in full, in one launch;
  * the large batch (2^x, 2^40 arguments in 2^16 uneven jobs, N = 2^16) at
    its m = 22 twin in one launch, with a seeded 1/64 of the jobs (1024
    jobs, about 2^34 arguments) compared in full and every job's count
    checked against the launch's total.
"""
import random

import pytest

import workloads as wl
from oracle_pool import oracle_lists

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = tmd.Context(0)
    yield c
    c.close()


def batched_records(ctx, jobs, cap):
    """One autotuned persistent graph launch over `jobs`, read back."""
    tmd.tmd_autotune(ctx, jobs)
    d_cand, d_count = tmd.alloc_candidates(cap)
    b = tmd.Batch(ctx, jobs, d_cand, d_count)
    b.launch()
    got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
    st = b.stats()
    b.close()
    return got, n, st


def test_plain_slice_in_full_at_m40_and_its_dense_twin(ctx):
    jobs = {m: wl.plain_job(m=m) for m in (40, 20)}
    want = oracle_lists([jobs[40]], [40, 20])
    for m in (40, 20):
        got, n, st = batched_records(ctx, [jobs[m]], 1 << 18)
        assert st["lines"] == 1 << 22
        assert n == len(got) == len(want[m]), m
        assert got == want[m], m
    # m = 40: about 2^22 (1 - exp(-2^14 2^-39)) = 0.13 expected records;
    # m = 20: about 2^22 (1 - exp(-2^14 2^-19)) = 1.3e5
    assert len(want[40]) <= 5
    assert 1.1e5 < len(want[20]) < 1.5e5


def test_mixed_batch_of_64_jobs_in_full_at_m20(ctx):
    jobs = wl.batched_jobs(m=20)
    assert len(jobs) == 64
    want = oracle_lists(jobs, [20])[20]
    got, n, st = batched_records(ctx, jobs, 1 << 20)
    assert n == len(got) == len(want)
    assert got == want
    assert len(want) > 1e5
    assert {r[0] for r in want} == set(range(64))   # every job has records


def test_large_batch_one_launch_seeded_64th_of_jobs_in_full_at_m22(ctx):
    jobs = [j.replace(m=22) for j in wl.large_jobs()]
    got, n, st = batched_records(ctx, jobs, 1 << 20)
    assert n == len(got) and st["lines"] == 1 << 24
    idx = sorted(random.Random(64).sample(range(len(jobs)), len(jobs) // 64))
    want = oracle_lists([jobs[k] for k in idx], [22], job_indexes=idx)[22]
    picked = set(idx)
    assert [r for r in got if r[0] in picked] == want
    # about 3 % of the 2^24 lines have an argument within 2^-22
    assert 3e5 < n < 7e5
