"""ctypes view of include/tmd.h: structures, status codes and the loaded
library.  Loading fails loudly when libtmd.so has not been built."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmd.so")
PROBE_PATH = os.path.join(HERE, "libtmd_probe.so")

TMD_OK, TMD_EINVAL, TMD_ENOMEM, TMD_EOVERFLOW, TMD_ETIMEOUT, TMD_ECUDA, TMD_EUNSUPPORTED = range(7)
TMD_EXP, TMD_EXP2, TMD_LOG = 0, 1, 2
TMD_BP_DIRECTED = 1
TMD_ALL_HITS = 2
TMD_LEFEVRE = 4
TMD_SOUND = 8


class TmdError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} (status {status})")


class tmd_job(ctypes.Structure):
    _fields_ = [("func", ctypes.c_int32), ("e_in", ctypes.c_int32), ("p", ctypes.c_int32),
                ("m", ctypes.c_int32), ("log2_N", ctypes.c_uint32), ("d", ctypes.c_int32),
                ("log2_T", ctypes.c_uint32), ("limbs", ctypes.c_uint32), ("start", ctypes.c_uint64),
                ("count", ctypes.c_uint64), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("eps1", ctypes.c_uint64), ("eps3", ctypes.c_uint64)]


class tmd_candidate(ctypes.Structure):
    _fields_ = [("job", ctypes.c_uint32), ("subint", ctypes.c_uint32),
                ("arg_index", ctypes.c_uint64), ("value", ctypes.c_uint64)]


class tmd_plan_info(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_uint64), ("n_subints", ctypes.c_uint64),
                ("n_segments", ctypes.c_uint32), ("e_out_first", ctypes.c_int32),
                ("cut", ctypes.c_uint64 * 4)]


class tmd_block_info(ctypes.Structure):
    _fields_ = [("start", ctypes.c_uint64), ("length", ctypes.c_uint64),
                ("first_sub", ctypes.c_uint64), ("e_out", ctypes.c_int32),
                ("scale_log2", ctypes.c_int32)]


class tmd_server_config(ctypes.Structure):
    _fields_ = [("device_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("chunk_tasks", ctypes.c_uint32), ("cand_cap", ctypes.c_uint64),
                ("max_batch", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class tmd_job_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("count", ctypes.c_uint64), ("n_records", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class tmd_stats(ctypes.Structure):
    _fields_ = [("lines", ctypes.c_uint64), ("filter_fail", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("half_steps", ctypes.c_uint64),
                ("upload_bytes", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("exhaustive_args", ctypes.c_uint64), ("refined_args", ctypes.c_uint64)]


class tmd_tiling(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32), ("lanes", ctypes.c_uint32),
                ("unroll", ctypes.c_uint32)]


_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_i32 = ctypes.c_int32
_sz = ctypes.c_size_t

# name -> (restype, argtypes); the declarations of include/tmd.h
SIGNATURES = {
    "tmd_version": (ctypes.c_char_p, []),
    "tmd_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tmd_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
    "tmd_destroy": (ctypes.c_int, [_vp]),
    "tmd_evict": (ctypes.c_int, [_vp]),
    "tmd_plan": (ctypes.c_int, [ctypes.POINTER(tmd_job), ctypes.POINTER(tmd_plan_info)]),
    "tmd_block_tables": (ctypes.c_int, [ctypes.POINTER(tmd_job), _u64, _vp, _vp,
                                        ctypes.POINTER(tmd_block_info)]),
    "tmd_generate": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), _u32, _vp, _sz,
                                    ctypes.POINTER(_sz), _vp]),
    "tmd_search": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), _u32, _vp, _vp, _u64, _vp, _vp]),
    "tmd_candidates": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp, _u64, ctypes.POINTER(_u64), _vp]),
    "tmd_search_lines": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _i32, _u32, _vp, _u64, _vp, _vp]),
    "tmd_lower_bounds": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp]),
    "tmd_lefevre_bounds": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp]),
    "tmd_sound_eps": (ctypes.c_int, [ctypes.POINTER(tmd_job), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "tmd_sound_piece_eps": (ctypes.c_int, [ctypes.POINTER(tmd_job), ctypes.POINTER(_u64)]),
    "tmd_sound_line_eps": (ctypes.c_int, [ctypes.POINTER(tmd_job), _u64, ctypes.POINTER(_u64)]),
    "tmd_stats_read": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_stats), _vp]),
    "tmd_batch_create": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), _u32, _vp, _u64, _vp, _vp,
                                        ctypes.POINTER(_vp), ctypes.POINTER(_u64)]),
    "tmd_batch_create_tiled": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), _u32, _vp, _u64, _vp, _vp,
                                              ctypes.POINTER(tmd_tiling), ctypes.POINTER(_vp),
                                              ctypes.POINTER(_u64)]),
    "tmd_autotune": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), _u32, _vp, ctypes.POINTER(tmd_tiling),
                                    ctypes.POINTER(ctypes.c_float)]),
    "tmd_batch_tiling": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_tiling)]),
    "tmd_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "tmd_batch_stats": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_stats), _vp]),
    "tmd_batch_destroy": (ctypes.c_int, [_vp]),
    "tmd_search_static": (ctypes.c_int, [ctypes.POINTER(tmd_job), _u32, _vp, _u64, _vp, _vp]),
    "tmd_server_create": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_server_config), ctypes.POINTER(_vp)]),
    "tmd_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), _u64]),
    "tmd_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job_result), _u32, ctypes.POINTER(_u32),
                                       _vp, _u64, ctypes.POINTER(_u64), ctypes.c_int32]),
    "tmd_server_submit_many": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_job), ctypes.POINTER(_u64),
                                              ctypes.POINTER(ctypes.c_double), _u32]),
    "tmd_server_pending": (ctypes.c_int, [_vp, ctypes.POINTER(_u64)]),
    "tmd_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(tmd_stats), ctypes.POINTER(_u64)]),
    "tmd_server_clock": (ctypes.c_double, [_vp]),
    "tmd_server_destroy": (ctypes.c_int, [_vp]),
}

_LIB = None


def lib():
    """The loaded libtmd.so (raises when it is missing: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python paper_1211_3056_gb300/build.py` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


# the declarations of include/tmd_probe.h (libtmd_probe.so)
PROBE_SIGNATURES = {
    "tmd_pipe_rates": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
}

_PROBE = None


def probe_lib():
    """The loaded libtmd_probe.so (measurement support)."""
    global _PROBE
    if _PROBE is None:
        if not os.path.exists(PROBE_PATH):
            raise ImportError(f"{PROBE_PATH} is missing: build it with `python paper_1211_3056_gb300/build.py`")
        L = ctypes.CDLL(PROBE_PATH)
        for name, (res, args) in PROBE_SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _PROBE = L
    return _PROBE


def status_str(s: int) -> str:
    try:
        return lib().tmd_status_str(int(s)).decode()
    except ImportError:
        return "unknown"


def check(status: int, where: str, ok=(TMD_OK,)):
    if status not in ok:
        raise TmdError(status, where)
    return status


def make_job(job) -> tmd_job:
    """tmd_job from any object with the descriptor fields (e.g. workloads.Job)."""
    return tmd_job(job.func, job.e_in, job.p, job.m, job.log2_N, job.d, job.log2_T, job.limbs,
                   job.start, job.count, job.flags, 0, getattr(job, "eps1", 0), getattr(job, "eps3", 0))


def job_array(jobs):
    arr = (tmd_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = make_job(j)
    return arr
