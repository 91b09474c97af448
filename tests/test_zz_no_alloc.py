"""The allocation-free search entry point, through the C ABI.

tmd_search_static serves callers that may not allocate device memory while
they search (their allocator owns the pool, their host forbids it, or their
loop allows no allocation after start-up): it keeps the plan in the
library's fixed device array.  Its records must equal those of the ordinary
entry point (tmd_search, fused) exactly -- integer results, so the tolerance
is zero -- on two calls in a row, the second with a smaller job list, which
also checks that what the first call left in the array does not leak into
the second.  This file is
collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
tmd = pytest.importorskip("paper_1211_3056_gb300")
pytestmark = pytest.mark.gpu

JOBS = [
    wl.toy_job(),
    wl.Job(wl.FUNC_EXP, 0, 53, 22, 14, 3, 24, 3, wl.plain_start(), 1 << 32),
    wl.Job(wl.FUNC_LOG, 2, 30, 14, 8, 3, 14, 2, 12345, 1 << 20),
]


def read_back(d_cand, d_count):
    """Records straight from the caller's buffers (no context involved)."""
    n = int(d_count.cpu().item())
    cap = d_cand.numel() // tmd.CANDIDATE_BYTES
    k = min(n, cap)
    raw = d_cand[: k * tmd.CANDIDATE_BYTES].cpu().numpy()
    rec = np.frombuffer(raw.tobytes(), dtype=np.dtype([("job", "<u4"), ("subint", "<u4"),
                                                      ("arg", "<u8"), ("value", "<u8")]))
    out = sorted((int(r["job"]), int(r["subint"]), int(r["arg"]), int(r["value"])) for r in rec)
    return sorted(out, key=lambda r: (r[0], r[2], r[3])), n


def test_static_equals_ordinary_entry_point_twice():
    """Two calls in a row: the first with all of JOBS (the larger plan), the
    second with a smaller, different list, whose plan overwrites only part of
    what the first call left in the array."""
    torch.cuda.set_device(0)
    calls = [JOBS, [JOBS[2], JOBS[0]]]
    with tmd.Context(0) as ctx:
        wants = [tmd.run(jobs, ctx=ctx, fused=True, cap=1 << 16) for jobs in calls]
    assert wants[0][1] > 1000 and wants[1][1] > 100
    for call, (jobs, (want, n_want)) in enumerate(zip(calls, wants)):
        d_cand, d_count = tmd.alloc_candidates(1 << 16)
        d_cand.fill_(0xAB)
        d_count.fill_(12345)                  # the entry point must clear it
        tmd.tmd_search_static(jobs, d_cand, d_count)
        torch.cuda.synchronize()
        got, n = read_back(d_cand, d_count)
        assert n == n_want, call
        assert got == want, call


def test_static_rejects_oversized_plan():
    big = wl.Job(wl.FUNC_EXP, 0, 53, 40, 14, 3, 24, 3, 0, 1 << 40)     # 65536 blocks
    d_cand, d_count = tmd.alloc_candidates(16)
    with pytest.raises(tmd.TmdError) as e:
        tmd.tmd_search_static([big], d_cand, d_count)
    assert e.value.status == tmd._lib.TMD_ENOMEM
