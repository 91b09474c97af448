"""The oracle's candidate list: what the hot path must reproduce bit-exactly.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

For every job, every block and every sub-interval (plan.py), the oracle
  1. computes the block's Taylor coefficients from exact enclosures of f
     (fmath.py, Ziv's strategy for the rounding),
  2. evaluates b_i and alpha_i by direct Horner (poly.py),
  3. forms the search words B, A and the threshold T_m,
  4. takes min_{0<=x<N_i} (B - A x) mod 2^64 and its smallest argmin by
     brute force over every x (the C loop of brute.c, or numpy),
  5. reports (job, sub-interval, argument index of the argmin, min) when
     min < T_m; with FLAG_ALL_HITS it reports every x with a value < T_m.
The list is sorted by (job, argument index, value).
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterator, List, Sequence, Tuple

import numpy as np

from . import plan, poly

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _brute_lib():
    """The compiled brute.c (built by build_brute()); None when absent."""
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "_brute.so")
        if not os.path.exists(path):
            return None
        lib = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_brute_min.argtypes = [ctypes.c_size_t, u64p, u64p, u32p, u64p, u32p, ctypes.c_int]
        lib.oracle_brute_min.restype = None
        lib.oracle_brute_hits.argtypes = [ctypes.c_size_t, u64p, u64p, u32p, ctypes.c_uint64,
                                          u32p, u32p, u64p, ctypes.c_size_t]
        lib.oracle_brute_hits.restype = ctypes.c_size_t
        lib.oracle_threads_available.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def build_brute() -> str:
    """Compile brute.c into oracle/_brute.so with the system C compiler."""
    src = os.path.join(_HERE, "brute.c")
    out = os.path.join(_HERE, "_brute.so")
    cmd = f"gcc -O2 -fPIC -shared -fopenmp -o {out} {src}"
    rc = os.system(cmd)
    if rc != 0:
        raise RuntimeError("building the oracle's brute-force helper failed: " + cmd)
    global _LIB
    _LIB = None
    return out


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def brute_min_many(B: np.ndarray, A: np.ndarray, n: np.ndarray, threads: int = 0):
    """Vector of (min, argmin) for many lines; C loop when built, else numpy."""
    B = np.ascontiguousarray(B, dtype=np.uint64)
    A = np.ascontiguousarray(A, dtype=np.uint64)
    n = np.ascontiguousarray(n, dtype=np.uint32)
    mins = np.empty(len(B), dtype=np.uint64)
    args = np.empty(len(B), dtype=np.uint32)
    lib = _brute_lib()
    if lib is not None:
        lib.oracle_brute_min(len(B), _ptr(B, ctypes.c_uint64), _ptr(A, ctypes.c_uint64),
                             _ptr(n, ctypes.c_uint32), _ptr(mins, ctypes.c_uint64),
                             _ptr(args, ctypes.c_uint32), int(threads))
        return mins, args
    # numpy: uint64 array arithmetic wraps mod 2^64
    for i in range(len(B)):
        x = np.arange(int(n[i]), dtype=np.uint64)
        v = B[i] - A[i] * x
        k = int(np.argmin(v))
        mins[i] = v[k]
        args[i] = k
    return mins, args


def brute_hits_many(B, A, n, T: int):
    """All (line, x, value) with (B - A x) mod 2^64 < T."""
    B = np.ascontiguousarray(B, dtype=np.uint64)
    A = np.ascontiguousarray(A, dtype=np.uint64)
    n = np.ascontiguousarray(n, dtype=np.uint32)
    lib = _brute_lib()
    if lib is not None:
        cap = 1 << 16
        while True:
            lo = np.empty(cap, dtype=np.uint32)
            xo = np.empty(cap, dtype=np.uint32)
            vo = np.empty(cap, dtype=np.uint64)
            got = lib.oracle_brute_hits(len(B), _ptr(B, ctypes.c_uint64), _ptr(A, ctypes.c_uint64),
                                        _ptr(n, ctypes.c_uint32), ctypes.c_uint64(T),
                                        _ptr(lo, ctypes.c_uint32), _ptr(xo, ctypes.c_uint32),
                                        _ptr(vo, ctypes.c_uint64), cap)
            if got <= cap:
                return [(int(lo[i]), int(xo[i]), int(vo[i])) for i in range(got)]
            cap = int(got)
    out = []
    for i in range(len(B)):
        x = np.arange(int(n[i]), dtype=np.uint64)
        v = B[i] - A[i] * x
        for k in np.nonzero(v < np.uint64(T))[0]:
            out.append((i, int(k), int(v[k])))
    return out


def block_lines(job, block) -> Tuple[List[int], np.ndarray, np.ndarray, np.ndarray]:
    """(coefficients, B[], A[], N_i[]) for every sub-interval of one block."""
    W = 64 * job.limbs
    N = 1 << job.log2_N
    c = poly.taylor_coeffs(job, block)
    nsub = (block.length + N - 1) // N
    Bs = np.empty(nsub, dtype=np.uint64)
    As = np.empty(nsub, dtype=np.uint64)
    ns = np.empty(nsub, dtype=np.uint32)
    for i in range(nsub):
        b, alpha = poly.line(c, i, N, W)
        B, A = poly.search_words(b, alpha, job.m, W)
        Bs[i] = B
        As[i] = A
        ns[i] = min(N, block.length - i * N)
    return c, Bs, As, ns


def job_lines(job) -> Iterator[Tuple[object, List[int], np.ndarray, np.ndarray, np.ndarray]]:
    for blk in plan.blocks(job):
        c, B, A, n = block_lines(job, blk)
        yield blk, c, B, A, n


def job_candidates(job, job_index: int = 0, blocks: Sequence = None, threads: int = 0):
    """Candidate records (job, subint, arg_index, value) of one job; with
    `blocks` given, only those blocks (a sample of the plan) are searched."""
    N = 1 << job.log2_N
    Tm = poly.threshold(job.m)
    out = []
    bl = plan.blocks(job) if blocks is None else blocks
    for blk in bl:
        _, B, A, n = block_lines(job, blk)
        if job.flags & plan.FLAG_ALL_HITS:
            for i, x, v in brute_hits_many(B, A, n, Tm):
                out.append((job_index, blk.first_sub + i, blk.start + i * N + x, v))
        else:
            mins, args = brute_min_many(B, A, n, threads)
            for i in np.nonzero(mins < np.uint64(Tm))[0]:
                i = int(i)
                out.append((job_index, blk.first_sub + i, blk.start + i * N + int(args[i]),
                            int(mins[i])))
    return out


def candidates(jobs, threads: int = 0):
    """Sorted candidate list of a batch of jobs."""
    out = []
    for j, job in enumerate(jobs):
        out.extend(job_candidates(job, j, threads=threads))
    out.sort(key=lambda r: (r[0], r[2], r[3]))
    return out
