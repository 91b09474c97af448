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


def test_group_overflow_reruns_jobs_alone_with_exact_counts():
    """Jobs admitted together whose records overflow the group's buffer are
    re-run one by one: few-candidate jobs come back complete, the others
    with TMD_EOVERFLOW and their exact count."""
    many = wl.Job(wl.FUNC_EXP, 0, 53, 18, 14, 3, 24, 3, wl.plain_start(), 1 << 28)
    few = [wl.Job(wl.FUNC_EXP2, 1, 24, 14, 8, 2, 12, 1, 0, 1 << 14),
           wl.Job(wl.FUNC_LOG, 2, 53, 40, 14, 2, 18, 3, 5 << 40, 1 << 20)]
    jobs = [few[0], many, few[1]]
    with tmd.Context(0) as ctx:
        solo = [tmd.run([j], ctx=ctx, fused=True, cap=1 << 16) for j in jobs]
        assert solo[0][1] < 8 and solo[2][1] < 8 and solo[1][1] > 8
        with tmd.Server(ctx, cand_cap=8, max_batch=8, max_inflight=1) as srv:
            for tag, j in enumerate(jobs):
                srv.submit(j, tag)
            got = {}
            deadline = time.time() + 60
            while len(got) < 3 and time.time() < deadline:
                for r, recs in srv.poll(wait_ms=100):
                    got[r["id"]] = (r, recs)
    for tag in (0, 2):
        r, recs = got[tag]
        assert r["status"] == 0 and recs == solo[tag][0] and r["count"] == solo[tag][1]
    r, recs = got[1]
    assert r["status"] == tmd.TMD_EOVERFLOW and r["count"] == solo[1][1]
    assert len(recs) == 8 and set(recs) <= set(solo[1][0])


def test_served_filter_variants_and_sound_jobs_equal_the_oracle():
    """Jobs of the general kernel variant (Lefevre's filter, sound mode)
    served in a mix with ordinary ones, admitted together: each result
    equals the oracle's list for that job alone (the candidate list, or for
    a sound job the exhaustive list at its eps3)."""
    from oracle import candidates as oc
    from oracle import sound
    base = [wl.Job(wl.FUNC_EXP, 0, 24, 10, 8, 2, 12, 1, 3 << 20, 1 << 13),
            wl.Job(wl.FUNC_LOG, 2, 20, 8, 6, 2, 10, 1, 100, 1 << 12),
            wl.Job(wl.FUNC_EXP, 0, 53, 18, 14, 3, 24, 3, wl.plain_start(), 1 << 26)]
    jobs = [tmd.sound_job(base[0]), base[1].replace(flags=wl.FLAG_LEFEVRE), base[2],
            tmd.sound_job(base[1]), base[2].replace(flags=wl.FLAG_LEFEVRE)]
    with tmd.Context(0) as ctx:
        with tmd.Server(ctx, max_inflight=2, chunk_tasks=8, cand_cap=1 << 16, max_batch=8) as srv:
            got = serve_all(srv, jobs, [0.0] * len(jobs))
        assert len(got) == len(jobs)
    for tag, job in enumerate(jobs):
        r, recs = got[tag]
        if job.flags & wl.FLAG_SOUND:
            want = [(0,) + w[1:] for w in sound.sound_candidates([job], [job.eps3])]
        else:
            want = oc.job_candidates(job, 0)
        assert r["status"] == 0 and r["count"] == len(want)
        assert recs == sorted(want, key=lambda w: (w[0], w[2], w[3])), tag


def test_scheduled_arrivals_equal_solo_runs_and_counters():
    """A Poisson arrival stream replayed by the server's clock
    (tmd_server_submit_many): every job is admitted no earlier than its
    arrival, groups overlap on the device, each result equals the job's solo
    run, and the server's counters cover every line of every job once."""
    from oracle import plan
    jobs = wl.serving_jobs(njobs=60, size_log2_range=(18.0, 26.0))
    jobs = [j.replace(m=m) for j, m in zip(jobs, random.Random(9).choices([20, 24, 30], k=60))]
    delays = wl.arrival_times(len(jobs), 20000.0, seed=3)
    with tmd.Context(0) as ctx:
        with tmd.Server(ctx, max_inflight=3, max_batch=16, cand_cap=1 << 16) as srv:
            t0 = srv.clock()
            srv.submit_many(jobs, list(range(len(jobs))), delays)
            got = {}
            deadline = time.time() + 120
            while len(got) < len(jobs) and time.time() < deadline:
                for r, recs in srv.poll(wait_ms=100):
                    got[r["id"]] = (r, recs)
            st = srv.stats()
            assert srv.pending() == 0
        assert len(got) == len(jobs)
        for tag, job in enumerate(jobs):
            r, recs = got[tag]
            solo, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 16)
            assert r["status"] == 0 and r["count"] == n and recs == solo, tag
            assert r["t_submit"] >= t0 + delays[tag] - 1e-3
            assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    assert st["lines"] == sum(plan.n_subintervals(j) for j in jobs)
    assert st["count"] == sum(got[t][0]["count"] for t in got)
    assert st["groups"] >= 4
