"""GB300 hard-to-round argument search (arXiv 1211.3056 hot path).

Thin Python binding of the C ABI in include/tmd.h: every function below only
marshals arguments to libtmd.so, where all the work runs (host C++ planning
and correctly rounded tables, CUDA kernels for generation and search).
PyTorch supplies device memory and streams.  Importing this package raises
ImportError when libtmd.so has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence, Tuple

from . import _lib
from ._lib import (TMD_ALL_HITS, TMD_BP_DIRECTED, TMD_LEFEVRE, TMD_SOUND, TMD_EXP, TMD_EXP2, TMD_LOG, TMD_OK,  # noqa: F401
                   TMD_EOVERFLOW, TmdError, check, job_array, lib, make_job)

lib()  # fail loudly at import when the extension is missing

CANDIDATE_BYTES = ctypes.sizeof(_lib.tmd_candidate)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Context:
    """Owns one tmd_ctx (device scratch, pinned staging, resident plan)."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        check(lib().tmd_create(ctypes.byref(h), int(device)), "tmd_create")
        self.handle = h
        self.device = int(device)
        self._h_out = None  # host record buffer of tmd_candidates, reused

    def host_records(self, n: int):
        """A host array of at least n candidate records, kept between calls
        (a fresh one per call costs a zeroed allocation of its whole size)."""
        n = max(1, int(n))
        if self._h_out is None or len(self._h_out) < n:
            self._h_out = (_lib.tmd_candidate * n)()
        return self._h_out

    def close(self):
        if self.handle:
            lib().tmd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmd_version() -> str:
    return lib().tmd_version().decode()


def tmd_create(device: int = 0) -> Context:
    return Context(device)


def tmd_destroy(ctx: Context) -> None:
    ctx.close()


def tmd_evict(ctx: Context) -> None:
    check(lib().tmd_evict(ctx.handle), "tmd_evict")


def tmd_plan(job) -> dict:
    info = _lib.tmd_plan_info()
    check(lib().tmd_plan(ctypes.byref(make_job(job)), ctypes.byref(info)), "tmd_plan")
    return {"n_blocks": info.n_blocks, "n_subints": info.n_subints, "n_segments": info.n_segments,
            "e_out_first": info.e_out_first, "cuts": [info.cut[i] for i in range(info.n_segments - 1)]}


def _words_to_ints(arr, count: int, limbs: int) -> List[int]:
    out = []
    for w in range(count):
        v = 0
        for l in range(limbs):
            v |= int(arr[w * limbs + l]) << (64 * l)
        out.append(v)
    return out


def tmd_block_tables(job, block: int) -> Tuple[List[int], List[int], dict]:
    """(coefficients c_0..c_d, the 2d+1 table words, block info) as ints."""
    L, d = job.limbs, job.d
    coeffs = (ctypes.c_uint64 * ((d + 1) * L))()
    table = (ctypes.c_uint64 * ((2 * d + 1) * L))()
    info = _lib.tmd_block_info()
    check(lib().tmd_block_tables(ctypes.byref(make_job(job)), int(block), coeffs, table,
                                 ctypes.byref(info)), "tmd_block_tables")
    return (_words_to_ints(coeffs, d + 1, L), _words_to_ints(table, 2 * d + 1, L),
            {"start": info.start, "length": info.length, "first_sub": info.first_sub,
             "e_out": info.e_out, "scale_log2": info.scale_log2})


def tmd_generate(ctx: Context, jobs: Sequence, d_lin=None, stream=None) -> int:
    """Plan + tables + generation kernel; returns the bytes d_lin needs."""
    arr = job_array(jobs)
    need = ctypes.c_size_t(0)
    nbytes = 0 if d_lin is None else d_lin.numel() * d_lin.element_size()
    check(lib().tmd_generate(ctx.handle, arr, len(jobs), _ptr(d_lin), nbytes, ctypes.byref(need),
                             _stream_ptr(stream)), "tmd_generate")
    return need.value


def tmd_search(ctx: Context, jobs: Sequence, d_lin, d_cand, d_count, stream=None) -> None:
    arr = job_array(jobs)
    cap = 0 if d_cand is None else (d_cand.numel() * d_cand.element_size()) // CANDIDATE_BYTES
    check(lib().tmd_search(ctx.handle, arr, len(jobs), _ptr(d_lin), _ptr(d_cand), cap, _ptr(d_count),
                           _stream_ptr(stream)), "tmd_search")


def tmd_candidates(ctx: Context, d_cand, d_count, h_cap: Optional[int] = None, stream=None):
    """(sorted records as (job, subint, arg_index, value) tuples, exact count)."""
    cap = 0 if d_cand is None else (d_cand.numel() * d_cand.element_size()) // CANDIDATE_BYTES
    if h_cap is None:
        h_cap = cap
    out = ctx.host_records(h_cap)
    n = ctypes.c_uint64(0)
    st = lib().tmd_candidates(ctx.handle, _ptr(d_cand), _ptr(d_count), cap, out, h_cap,
                              ctypes.byref(n), _stream_ptr(stream))
    check(st, "tmd_candidates", ok=(TMD_OK, TMD_EOVERFLOW))
    k = min(n.value, cap, h_cap)
    recs = [(out[i].job, out[i].subint, out[i].arg_index, out[i].value) for i in range(k)]
    return recs, n.value


def tmd_search_lines(ctx: Context, d_B, d_A, d_len, m: int, flags: int, d_cand, d_count,
                     stream=None) -> None:
    n = d_B.numel()
    cap = 0 if d_cand is None else (d_cand.numel() * d_cand.element_size()) // CANDIDATE_BYTES
    check(lib().tmd_search_lines(ctx.handle, _ptr(d_B), _ptr(d_A), _ptr(d_len), n, int(m), int(flags),
                                 _ptr(d_cand), cap, _ptr(d_count), _stream_ptr(stream)),
          "tmd_search_lines")


def tmd_lower_bounds(ctx: Context, d_B, d_A, d_len, d_lb, d_hs=None, stream=None) -> None:
    check(lib().tmd_lower_bounds(ctx.handle, _ptr(d_B), _ptr(d_A), _ptr(d_len), d_B.numel(),
                                 _ptr(d_lb), _ptr(d_hs), _stream_ptr(stream)), "tmd_lower_bounds")


def tmd_sound_eps(job) -> tuple:
    """(eps1, eps3): the sound thresholds of a job on the 64-bit words (host)."""
    j = make_job(job)
    e1, e3 = ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(lib().tmd_sound_eps(ctypes.byref(j), ctypes.byref(e1), ctypes.byref(e3)), "tmd_sound_eps")
    return e1.value, e3.value


def tmd_sound_piece_eps(job) -> int:
    """The phase-2 half-width the library uses for a sound job (host)."""
    j = make_job(job)
    e2 = ctypes.c_uint64(0)
    check(lib().tmd_sound_piece_eps(ctypes.byref(j), ctypes.byref(e2)), "tmd_sound_piece_eps")
    return e2.value


def tmd_sound_line_eps(job, length: int) -> int:
    """The sound half-width for lines of `length` arguments of a sound job
    (host): what the library tests the sub-pieces of phase 3 against."""
    j = make_job(job)
    e = ctypes.c_uint64(0)
    check(lib().tmd_sound_line_eps(ctypes.byref(j), ctypes.c_uint64(int(length)), ctypes.byref(e)),
          "tmd_sound_line_eps")
    return e.value


def sound_job(job):
    """The job in sound mode with the library's sound thresholds."""
    e1, e3 = tmd_sound_eps(job)
    return job.replace(flags=job.flags | TMD_SOUND, eps1=e1, eps3=e3)


def tmd_lefevre_bounds(ctx: Context, d_B, d_A, d_len, d_lb, d_iters=None, stream=None,
                       specific: bool = True) -> None:
    check(lib().tmd_lefevre_bounds(ctx.handle, _ptr(d_B), _ptr(d_A), _ptr(d_len), d_B.numel(),
                                   1 if specific else 0, _ptr(d_lb), _ptr(d_iters), _stream_ptr(stream)),
          "tmd_lefevre_bounds")


def tmd_stats_read(ctx: Context, stream=None) -> dict:
    s = _lib.tmd_stats()
    check(lib().tmd_stats_read(ctx.handle, ctypes.byref(s), _stream_ptr(stream)), "tmd_stats_read")
    return {"lines": s.lines, "filter_fail": s.filter_fail, "candidates": s.candidates,
            "half_steps": s.half_steps, "upload_bytes": s.upload_bytes, "count": s.count,
            "exhaustive_args": s.exhaustive_args, "refined_args": s.refined_args}


class Batch:
    """A tmd_batch: resident plan of many jobs plus its captured graph."""

    def __init__(self, ctx: Context, jobs: Sequence, d_cand, d_count, stream=None, tiling=None):
        """tiling: None = the context's autotuned tiling for this batch
        signature (else the default); or (nu, ctas_per_sm[, lanes[, unroll]])."""
        self.ctx = ctx
        self.jobs = list(jobs)
        self.d_cand, self.d_count = d_cand, d_count   # kept alive with the batch
        cap = 0 if d_cand is None else (d_cand.numel() * d_cand.element_size()) // CANDIDATE_BYTES
        h = ctypes.c_void_p()
        up = ctypes.c_uint64(0)
        if tiling is None:
            check(lib().tmd_batch_create(ctx.handle, job_array(self.jobs), len(self.jobs), _ptr(d_cand),
                                         cap, _ptr(d_count), _stream_ptr(stream), ctypes.byref(h),
                                         ctypes.byref(up)), "tmd_batch_create")
        else:
            tl = list(tiling) + [0] * (4 - len(tiling))
            t = _lib.tmd_tiling(int(tl[0]), int(tl[1]), int(tl[2]), int(tl[3]))
            check(lib().tmd_batch_create_tiled(ctx.handle, job_array(self.jobs), len(self.jobs), _ptr(d_cand),
                                               cap, _ptr(d_count), _stream_ptr(stream), ctypes.byref(t),
                                               ctypes.byref(h), ctypes.byref(up)), "tmd_batch_create_tiled")
        self.handle = h
        self.upload_bytes = up.value

    def tiling(self) -> tuple:
        """(nu, ctas_per_sm, lanes, unroll) the batch was built with."""
        t = _lib.tmd_tiling()
        check(lib().tmd_batch_tiling(self.handle, ctypes.byref(t)), "tmd_batch_tiling")
        return (t.nu, t.ctas_per_sm, t.lanes, t.unroll)

    def launch(self, stream=None):
        check(lib().tmd_batch_launch(self.handle, _stream_ptr(stream)), "tmd_batch_launch")

    def stats(self, stream=None) -> dict:
        s = _lib.tmd_stats()
        check(lib().tmd_batch_stats(self.handle, ctypes.byref(s), _stream_ptr(stream)), "tmd_batch_stats")
        return {"lines": s.lines, "filter_fail": s.filter_fail, "candidates": s.candidates,
                "half_steps": s.half_steps, "upload_bytes": s.upload_bytes, "count": s.count,
                "exhaustive_args": s.exhaustive_args, "refined_args": s.refined_args}

    def close(self):
        if getattr(self, "handle", None):
            lib().tmd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmd_batch_create(ctx: Context, jobs: Sequence, d_cand, d_count, stream=None, tiling=None) -> Batch:
    return Batch(ctx, jobs, d_cand, d_count, stream, tiling)


def tmd_autotune(ctx: Context, jobs: Sequence, stream=None) -> dict:
    """Time the batch under every candidate tiling; the fastest is kept in the
    context for batches of the same signature.  Returns {"nu", "ctas_per_sm",
    "lanes", "unroll", "ms"}."""
    t = _lib.tmd_tiling()
    ms = ctypes.c_float(0.0)
    check(lib().tmd_autotune(ctx.handle, job_array(list(jobs)), len(jobs), _stream_ptr(stream),
                             ctypes.byref(t), ctypes.byref(ms)), "tmd_autotune")
    return {"nu": t.nu, "ctas_per_sm": t.ctas_per_sm, "lanes": t.lanes, "unroll": t.unroll, "ms": ms.value}


def tmd_batch_launch(batch: Batch, stream=None) -> None:
    batch.launch(stream)


def tmd_batch_stats(batch: Batch, stream=None) -> dict:
    return batch.stats(stream)


def tmd_batch_destroy(batch: Batch) -> None:
    batch.close()


class Server:
    """A tmd_server: continuous batching of submitted jobs on ctx's device."""

    def __init__(self, ctx: Context, device_budget: int = 0, max_inflight: int = 0,
                 chunk_tasks: int = 0, cand_cap: int = 0, max_batch: int = 0):
        cfg = _lib.tmd_server_config(device_budget, max_inflight, chunk_tasks, cand_cap, max_batch, 0)
        h = ctypes.c_void_p()
        check(lib().tmd_server_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "tmd_server_create")
        self.handle = h
        self.ctx = ctx

    def submit(self, job, tag: int) -> None:
        check(lib().tmd_server_submit(self.handle, ctypes.byref(make_job(job)), int(tag)), "tmd_server_submit")

    def submit_many(self, jobs: Sequence, tags: Sequence[int], delays_s: Sequence[float]) -> None:
        """Queue jobs that arrive later: job i becomes eligible delays_s[i]
        seconds after this call (server clock)."""
        n = len(jobs)
        ids = (ctypes.c_uint64 * max(1, n))(*[int(t) for t in tags])
        dl = (ctypes.c_double * max(1, n))(*[float(d) for d in delays_s])
        check(lib().tmd_server_submit_many(self.handle, job_array(list(jobs)), ids, dl, n),
              "tmd_server_submit_many")

    def stats(self) -> dict:
        """Counters summed over the groups served so far."""
        s = _lib.tmd_stats()
        g = ctypes.c_uint64(0)
        check(lib().tmd_server_stats(self.handle, ctypes.byref(s), ctypes.byref(g)), "tmd_server_stats")
        return {"lines": s.lines, "filter_fail": s.filter_fail, "half_steps": s.half_steps, "count": s.count,
                "exhaustive_args": s.exhaustive_args, "refined_args": s.refined_args, "groups": g.value}

    def poll(self, cap: int = 256, rec_cap: int = 1 << 16, wait_ms: int = 0):
        """[(result dict, [(job, subint, arg_index, value), ...]), ...]"""
        # result and record arrays kept between polls (fresh zeroed arrays of
        # rec_cap records would cost more than a poll)
        if getattr(self, "_poll_bufs", None) is None or len(self._poll_bufs[0]) < cap \
                or len(self._poll_bufs[1]) < max(1, rec_cap):
            self._poll_bufs = ((_lib.tmd_job_result * cap)(), (_lib.tmd_candidate * max(1, rec_cap))())
        res, recs = self._poll_bufs
        n = ctypes.c_uint32(0)
        nr = ctypes.c_uint64(0)
        check(lib().tmd_server_poll(self.handle, res, cap, ctypes.byref(n), recs, rec_cap, ctypes.byref(nr),
                                    int(wait_ms)), "tmd_server_poll")
        out, pos = [], 0
        for i in range(n.value):
            r = res[i]
            k = r.n_records
            rr = [(recs[j].job, recs[j].subint, recs[j].arg_index, recs[j].value) for j in range(pos, pos + k)]
            pos += k
            out.append(({"id": r.id, "status": r.status, "count": r.count, "n_records": k,
                         "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done}, rr))
        return out

    def pending(self) -> int:
        n = ctypes.c_uint64(0)
        check(lib().tmd_server_pending(self.handle, ctypes.byref(n)), "tmd_server_pending")
        return n.value

    def clock(self) -> float:
        return lib().tmd_server_clock(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().tmd_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmd_server_create(ctx: Context, **cfg) -> Server:
    return Server(ctx, **cfg)


def tmd_search_static(jobs: Sequence, d_cand, d_count, stream=None) -> None:
    """Fused search of `jobs` on the current device without any device
    allocation: the plan goes into the library's fixed device array
    (include/tmd.h, TMD_STATIC_SCRATCH_BYTES).  For callers that may not
    allocate device memory while they search; calls that overlap on the GPU
    share that array and race.  Raises TmdError(TMD_ENOMEM) when the plan does
    not fit."""
    arr = job_array(jobs)
    cap = 0 if d_cand is None else (d_cand.numel() * d_cand.element_size()) // CANDIDATE_BYTES
    check(lib().tmd_search_static(arr, len(jobs), _ptr(d_cand), cap, _ptr(d_count),
                                  _stream_ptr(stream)), "tmd_search_static")


# ------------------------------------------------------------- conveniences
def alloc_candidates(cap: int, device: int = 0):
    """Device buffers for cap records and the count (torch tensors)."""
    import torch
    d_cand = torch.empty(cap * CANDIDATE_BYTES, dtype=torch.uint8, device=f"cuda:{device}")
    d_count = torch.zeros(1, dtype=torch.int64, device=f"cuda:{device}")
    return d_cand, d_count


def run(jobs: Sequence, ctx: Optional[Context] = None, fused: bool = True, cap: int = 1 << 20,
        device: int = 0, stream=None):
    """Generate + search + read back; returns (sorted records, exact count)."""
    import torch
    own = ctx is None
    if own:
        ctx = Context(device)
    try:
        d_cand, d_count = alloc_candidates(cap, device)
        d_lin = None
        if not fused:
            need = tmd_generate(ctx, jobs, None, stream)
            d_lin = torch.empty(max(need, 16) // 8, dtype=torch.int64, device=f"cuda:{device}")
            tmd_generate(ctx, jobs, d_lin, stream)
        tmd_search(ctx, jobs, d_lin, d_cand, d_count, stream)
        return tmd_candidates(ctx, d_cand, d_count, stream=stream)
    finally:
        if own:
            ctx.close()


def tmd_pipe_rates(device: int = 0) -> dict:
    """Measured lane-operations per SM per clock of 32-bit add, 3-input logic,
    32-bit multiply-add and FP32 FMA chains, and the SM clock (MHz)
    (libtmd_probe.so, include/tmd_probe.h)."""
    out = (ctypes.c_double * 5)()
    check(_lib.probe_lib().tmd_pipe_rates(int(device), out, 5), "tmd_pipe_rates")
    return {"add_u32": out[0], "lop3": out[1], "mad_u32": out[2], "ffma": out[3], "sm_mhz": out[4]}
