"""GPU parity of the served form: jobs arriving (Poisson gaps) while others
run are admitted as slots free up, overlap on the device, and each result is
exactly the one the same job gives alone (integer results: tolerance 0)."""
import random
import time

import pytest

import workloads as wl

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu


def serve_all(srv, jobs, gaps):
    got = {}
    for tag, (job, gap) in enumerate(zip(jobs, gaps)):
        time.sleep(gap)
        srv.submit(job, tag)
        for r, recs in srv.poll():
            got[r["id"]] = (r, recs)
    deadline = time.time() + 120
    while len(got) < len(jobs) and time.time() < deadline:
        for r, recs in srv.poll(wait_ms=100):
            got[r["id"]] = (r, recs)
    return got


def test_served_results_equal_solo_runs():
    jobs = wl.serving_jobs(njobs=40, size_log2_range=(18.0, 25.0))
    jobs = [j.replace(m=rng_m) for j, rng_m in zip(jobs, random.Random(7).choices([20, 24, 30], k=40))]
    rng = random.Random(5)
    gaps = [rng.expovariate(2000.0) for _ in jobs]
    with tmd.Context(0) as ctx:
        with tmd.Server(ctx, max_inflight=4, chunk_tasks=16, cand_cap=1 << 16) as srv:
            got = serve_all(srv, jobs, gaps)
            assert srv.pending() == 0
        assert len(got) == len(jobs)
        total = 0
        for tag, job in enumerate(jobs):
            r, recs = got[tag]
            solo, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 16)
            assert r["status"] == 0
            assert r["count"] == n and recs == solo, tag
            assert r["t_submit"] <= r["t_start"] <= r["t_done"]
            total += n
        assert total > 50


def test_served_overflow_keeps_exact_count():
    job = wl.Job(wl.FUNC_EXP, 0, 53, 18, 14, 3, 24, 3, wl.plain_start(), 1 << 28)
    with tmd.Context(0) as ctx:
        solo, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 16)
        assert n > 20
        with tmd.Server(ctx, cand_cap=8) as srv:
            srv.submit(job, 99)
            res = srv.poll(wait_ms=30000)
        assert len(res) == 1
        r, recs = res[0]
        assert r["status"] == tmd.TMD_EOVERFLOW and r["count"] == n
        assert len(recs) == 8 and set(recs) <= set(solo)
