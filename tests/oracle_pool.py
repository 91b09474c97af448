"""The CPU oracle's candidate lists of large workloads, block by block on
every host core.

TEST INFRASTRUCTURE ONLY: it runs the oracle (oracle/) and nothing else.  For
each Taylor block of a job the oracle computes the correctly rounded
coefficients (Sect. IV), evaluates every sub-interval's line by direct Horner,
forms the search words of each requested threshold 2^-m and takes the
minimum over every argument by brute force (Eq. (1)).  The lines of a block
are computed once and searched at every requested m, so a workload and its
dense twin cost one Horner pass.

The blocks are spread over a pool of worker processes started with the
"spawn" method (a process forked from one that has used CUDA can hang);
each worker runs the brute force on one thread.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from typing import Dict, List, Sequence, Tuple

Record = Tuple[int, int, int, int]


def _search_blocks(task):
    """Records of some blocks of one job at each threshold of `ms`:
    {m: [(job_index, subint, arg_index, value), ...]}."""
    job_index, job, blocks, ms = task
    import numpy as np

    from oracle import candidates as oc
    from oracle import poly

    W = 64 * job.limbs
    N = 1 << job.log2_N
    out = {m: [] for m in ms}
    for blk in blocks:
        c = poly.taylor_coeffs(job, blk)
        nsub = (blk.length + N - 1) // N
        lines = [poly.line(c, i, N, W) for i in range(nsub)]
        ns = np.array([min(N, blk.length - i * N) for i in range(nsub)], dtype=np.uint32)
        for m in ms:
            words = [poly.search_words(b, a, m, W) for b, a in lines]
            B = np.array([w[0] for w in words], dtype=np.uint64)
            A = np.array([w[1] for w in words], dtype=np.uint64)
            mins, args = oc.brute_min_many(B, A, ns, threads=1)
            Tm = np.uint64(poly.threshold(m))
            for i in np.nonzero(mins < Tm)[0]:
                i = int(i)
                out[m].append((job_index, blk.first_sub + i, blk.start + i * N + int(args[i]),
                               int(mins[i])))
    return out


def _tasks(jobs: Sequence, ms: Sequence[int], job_indexes: Sequence[int], blocks_per_task: int):
    from oracle import plan
    tasks = []
    for k, job in zip(job_indexes, jobs):
        bl = plan.blocks(job)
        # blocks of one task: about the same number of lines in each
        nsub = max(1, (1 << job.log2_T) >> job.log2_N)
        step = max(1, blocks_per_task * 1024 // nsub) if nsub < 1024 else blocks_per_task
        for i in range(0, len(bl), step):
            tasks.append((k, job, bl[i:i + step], tuple(ms)))
    return tasks


def oracle_lists(jobs: Sequence, ms: Sequence[int], job_indexes: Sequence[int] = None,
                 processes: int = 0, blocks_per_task: int = 4) -> Dict[int, List[Record]]:
    """{m: candidate list} of `jobs` searched at each threshold in `ms` (the
    jobs' own m is ignored), every block of every job, sorted by (job,
    argument index, value) as tmd_candidates sorts.  job_indexes gives the
    job field of the records (default 0, 1, ...)."""
    from oracle import candidates as oc
    if oc._brute_lib() is None:
        oc.build_brute()
    if job_indexes is None:
        job_indexes = list(range(len(jobs)))
    tasks = _tasks(jobs, ms, job_indexes, blocks_per_task)
    procs = processes or os.cpu_count() or 1
    out = {m: [] for m in ms}
    if procs <= 1 or len(tasks) <= 1:
        results = map(_search_blocks, tasks)
        for r in results:
            for m in ms:
                out[m].extend(r[m])
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            for r in pool.imap_unordered(_search_blocks, tasks, chunksize=1):
                for m in ms:
                    out[m].extend(r[m])
    for m in ms:
        out[m].sort(key=lambda r: (r[0], r[2], r[3]))
    return out
