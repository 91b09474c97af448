"""GPU parity on edge cases of the plan: the largest packet offsets (2^16
sub-intervals per block, where the straightforward-shift binomials peak),
a one-argument job, a job shorter than one sub-interval, a slice that ends
exactly at the binade's end, and a cut that falls inside a sub-interval."""
import random

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


def test_max_subintervals_per_block(ctx):
    # N = 2^6, T = 2^22: 65536 sub-intervals per block; dense threshold
    job = wl.Job(wl.FUNC_EXP, 0, 40, 12, 6, 3, 22, 2, 1 << 30, 3 << 22)
    got, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 20)
    assert n == len(got)
    blocks = plan.blocks(job)
    for blk in blocks:
        want = oc.job_candidates(job, blocks=[blk])
        mine = [r for r in got if blk.start <= r[2] < blk.start + blk.length]
        assert sorted(mine) == sorted(want)


@pytest.mark.parametrize("job", [
    wl.Job(wl.FUNC_EXP, 0, 53, 30, 14, 3, 24, 3, 123456789, 1),                   # one argument
    wl.Job(wl.FUNC_LOG, 2, 53, 20, 14, 2, 18, 3, 5 << 40, 1000),                  # shorter than N
    wl.Job(wl.FUNC_EXP2, 0, 53, 24, 12, 3, 24, 3, (1 << 52) - (1 << 26), 1 << 26),  # ends at 2^52
    wl.Job(wl.FUNC_EXP, 0, 30, 20, 10, 2, 16, 1, 0, 1 << 29),                     # cut mid sub-interval
], ids=["one_arg", "short", "binade_end", "cut"])
def test_plan_edges_exact(ctx, job):
    want = oc.candidates([job])
    for fused in (True, False):
        got, n = tmd.run([job], ctx=ctx, fused=fused, cap=1 << 16)
        assert n == len(want) and got == want


def test_cut_splits_a_subinterval():
    job = wl.Job(wl.FUNC_EXP, 0, 30, 20, 10, 2, 16, 1, 0, 1 << 29)
    segs = plan.segments(job)
    assert len(segs) == 2 and segs[1][0] % (1 << 10) != 0


def test_pipe_rates_are_plausible():
    """The probe behind the roofline's measured denominator: every rate is a
    lane count per SM per clock between a quarter and twice the issue width."""
    r = tmd.tmd_pipe_rates(0)
    for k in ("add_u32", "lop3", "mad_u32", "ffma"):
        assert 32 <= r[k] <= 260, (k, r[k])
    assert r["add_u32"] >= r["lop3"]
    assert 200 < r["sm_mhz"] < 4000


@pytest.mark.parametrize("job", [
    wl.Job(wl.FUNC_EXP2, -16, 53, 20, 14, 3, 20, 3, 1 << 40, 1 << 26),
    wl.Job(wl.FUNC_EXP, -16, 60, 24, 14, 3, 20, 3, 5 << 50, 1 << 26),
], ids=["exp2_shift69", "exp_shift76"])
def test_argument_shift_of_64_and_more(ctx, job):
    """X = M 2^-q with q = p - e_in >= 64 (the smallest binades): block
    starts whose low bits are zero are not integer arguments; the device
    tables and the search give the oracle's list."""
    want = oc.job_candidates(job, 0)
    assert len(want) > 0
    got, n = tmd.run([job], ctx=ctx, fused=True, cap=1 << 16)
    assert n == len(want) and got == want
