"""The parallel driver of the oracle used by the full-size GPU parity tests
gives exactly the oracle's own candidate lists (oracle.candidates, one job
after the other in this process), at each threshold it is asked for."""
import workloads as wl
from oracle import candidates as oc

from oracle_pool import oracle_lists

JOBS = [
    wl.toy_job(),                                                        # cut at ln 2
    wl.Job(wl.FUNC_EXP2, 1, 24, 16, 8, 2, 12, 1, 0, 1 << 16),             # exact point 2^1
    wl.Job(wl.FUNC_LOG, 3, 28, 14, 6, 2, 10, 1, 1 << 25, 1 << 21, wl.FLAG_BP_DIRECTED),
    wl.Job(wl.FUNC_EXP, 0, 53, 20, 14, 3, 24, 3, wl.plain_start(), (1 << 25) + 3 * (1 << 13) + 5),
]


def test_pool_equals_the_oracle_at_two_thresholds():
    got = oracle_lists(JOBS, [12, 16], processes=3, blocks_per_task=2)
    for m in (12, 16):
        want = oc.candidates([j.replace(m=m) for j in JOBS])
        assert got[m] == want, m
        assert len(want) > 100


def test_pool_job_indexes_and_serial_path():
    got = oracle_lists(JOBS[1:3], [14], job_indexes=[7, 3], processes=1)[14]
    want = sorted([(7,) + r[1:] for r in oc.job_candidates(JOBS[1].replace(m=14))] +
                  [(3,) + r[1:] for r in oc.job_candidates(JOBS[2].replace(m=14))],
                  key=lambda r: (r[0], r[2], r[3]))
    assert got == want
