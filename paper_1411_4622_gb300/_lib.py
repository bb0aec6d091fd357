"""ctypes declarations of the libsatpila C-ABI (include/satpila.h).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation in this package.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsatpila.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_NOT_FOUND, ERR_PENDING = (-1, -2, -3, -4, -6, -7, -8)
PILA_F32, PILA_F16, PILA_U8 = 0, 1, 2
SAT_SCHED_LINEAR, SAT_SCHED_GEOMETRIC, SAT_SCHED_CUBIC = 0, 1, 2
SAT_RESIDENT_AUTO, SAT_RESIDENT_SMEM, SAT_RESIDENT_GLOBAL = 0, 1, 2
SAT_FLAG_NO_GRAPH, SAT_FLAG_AUTOTUNE, SAT_FLAG_HYBRID, SAT_FLAG_BOME_INDEPENDENT = 1, 2, 4, 8
SAT_FLAG_WINDOW_GROUPS = 16
SAT_FLAG_TEST_STALL = 32
SAT_FLAG_NEAR_TIES = 64
(SAT_PLAN_RULES, SAT_PLAN_WINDOW_SMEM, SAT_PLAN_WINDOW_GLOBAL, SAT_PLAN_WINDOW_HYBRID, SAT_PLAN_PIPE_1,
 SAT_PLAN_PIPE_2, SAT_PLAN_PIPE_4, SAT_PLAN_WINDOW_G2, SAT_PLAN_WINDOW_G4, SAT_PLAN_WINDOW_SMEM_G2,
 SAT_PLAN_WINDOW_SMEM_G4) = range(11)
SIRT_SIMULTANEOUS, SIRT_SEQUENTIAL = 0, 1
PROBE_STREAM, PROBE_SECTOR = 0, 1
SAT_SERVER_PER_CLASS = 1

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTS = ["satpila_last_error", "satpila_version", "pila_build", "pila_free", "pila_info", "pila_export",
           "pila_forward", "pila_sirt_factor", "sat_run", "sat_run_ptrs", "sat_server_create", "sat_server_submit", "sat_server_poll",
           "sat_server_wait", "sat_server_info", "sat_server_destroy", "drt_bilinear", "sat_drt_run", "fbp", "fbp_prior", "sirt_run",
           "sirt_run_noalloc", "satpila_probe_read", "satpila_probe_smem"]
NOALLOC_SCRATCH_BYTES = 8 << 20


class PilaGeom(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_angles", C.c_int32), ("n_bins", C.c_int32),
                ("angles_rad", C.POINTER(C.c_double)), ("mask", C.POINTER(C.c_uint8))]


class PilaInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_angles", C.c_int32), ("n_bins", C.c_int32), ("precision", C.c_int32),
                ("n_mask", C.c_int32), ("record_bytes", C.c_int32), ("row_records", C.c_int32),
                ("pad", C.c_int32), ("table_bytes", C.c_int64), ("entries", C.c_int64)]


class SatTraceRec(C.Structure):
    _fields_ = [("pixel", C.c_int32), ("cstar", C.c_int32), ("accepted", C.c_int32), ("pad", C.c_int32),
                ("dS", C.c_float), ("dC", C.c_float), ("fnew", C.c_float), ("pad2", C.c_float)]


class SatParams(C.Structure):
    _fields_ = [("beta", C.c_float), ("bome_k", C.c_int32), ("n_sweeps", C.c_int32),
                ("moves_per_sweep", C.c_int32), ("t0", C.c_double), ("tn", C.c_double),
                ("schedule", C.c_int32), ("t0_samples", C.c_int32), ("seed", C.c_uint64),
                ("resync_every", C.c_int32), ("residency", C.c_int32), ("flags", C.c_uint32),
                ("trace_chain", C.c_int32), ("group_warps", C.c_int32), ("pipeline_depth", C.c_int32),
                ("trace", C.c_void_p), ("sweep_cost", C.c_void_p), ("plan", C.c_int32), ("wait_ms", C.c_int32)]


class SatStats(C.Structure):
    _fields_ = [("t0", C.c_double), ("tn", C.c_double), ("initial_cost", C.c_double),
                ("final_cost", C.c_double), ("final_cost_incremental", C.c_double),
                ("max_resync_drift", C.c_double), ("accepted", C.c_int64), ("proposed", C.c_int64),
                ("t0_found", C.c_int32), ("status", C.c_int32), ("sweep_ms", C.c_double),
                ("plan", C.c_int32), ("near_ties", C.c_int32)]


class SatServerCfg(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_active", C.c_int32), ("stages_per_tick", C.c_int32),
                ("queue_limit", C.c_int32), ("mem_budget", C.c_uint64), ("flags", C.c_uint32)]


class SatRequest(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_angles", C.c_int32), ("n_bins", C.c_int32), ("precision", C.c_int32),
                ("angles_rad", C.c_void_p), ("mask", C.c_void_p), ("sino", C.c_void_p), ("image", C.c_void_p),
                ("prm", SatParams)]


class SatResult(C.Structure):
    _fields_ = [("stats", SatStats), ("submit_ms", C.c_double), ("admit_ms", C.c_double), ("done_ms", C.c_double)]


class SatServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("active", C.c_int32), ("queued", C.c_int32), ("geometries", C.c_int32), ("classes", C.c_int32),
                ("bytes_in_use", C.c_uint64), ("bytes_peak", C.c_uint64), ("mem_budget", C.c_uint64),
                ("ticks", C.c_int64), ("moves", C.c_int64)]


class SirtParams(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("mode", C.c_int32), ("relax", C.c_float), ("pad", C.c_int32)]


_lock = threading.Lock()
_lib = None


def load():
    """Load libsatpila.so (built by paper_1411_4622_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsatpila.so not found at {LIB_PATH}; run paper_1411_4622_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        V = C.c_void_p
        lib.satpila_last_error.restype = C.c_char_p
        lib.satpila_last_error.argtypes = []
        lib.satpila_version.restype = C.c_int
        lib.pila_build.argtypes = [C.POINTER(PilaGeom), C.c_int32, V, C.POINTER(V)]
        lib.pila_free.argtypes = [V]
        lib.pila_info.argtypes = [V, C.POINTER(PilaInfo)]
        lib.pila_export.argtypes = [V, V, V, V]
        lib.pila_forward.argtypes = [V, C.c_int32, V, V, V]
        lib.pila_sirt_factor.argtypes = [V, V, V]
        lib.sat_run.argtypes = [V, C.c_int32, V, V, C.POINTER(SatParams), V, V]
        lib.sat_run_ptrs.argtypes = [V, C.c_int32, V, V, C.POINTER(SatParams), V, V]
        lib.sat_server_create.argtypes = [C.POINTER(SatServerCfg), C.POINTER(V)]
        lib.sat_server_submit.argtypes = [V, C.POINTER(SatRequest), C.POINTER(C.c_uint64)]
        lib.sat_server_poll.argtypes = [V, C.c_uint64, V, C.POINTER(SatResult)]
        lib.sat_server_wait.argtypes = [V, C.c_uint64, C.c_int32, V, C.POINTER(SatResult)]
        lib.sat_server_info.argtypes = [V, C.POINTER(SatServerStats)]
        lib.sat_server_destroy.argtypes = [V]
        lib.drt_bilinear.argtypes = [C.c_int32, C.c_int32, C.c_int32, V, C.c_int32, V, V, V]
        lib.sat_drt_run.argtypes = [C.c_int32, C.c_int32, C.c_int32, V, C.c_int32, V, V, C.POINTER(SatParams), V, V]
        lib.fbp.argtypes = [C.c_int32, C.c_int32, C.c_int32, V, C.c_int32, V, V, V]
        lib.fbp_prior.argtypes = [C.c_int32, C.c_int32, V, C.c_float, V, V, V, V]
        lib.sirt_run.argtypes = [V, C.c_int32, V, V, C.POINTER(SirtParams), V, V]
        lib.sirt_run_noalloc.argtypes = [V, C.c_int32, V, V, C.POINTER(SirtParams), V, V]
        lib.satpila_probe_read.argtypes = [V, C.c_uint64, C.c_int32, C.c_uint64, C.c_uint64, C.POINTER(C.c_double), V]
        lib.satpila_probe_smem.argtypes = [C.c_int32, C.c_uint64, C.POINTER(C.c_double), V]
        for name in EXPORTS:
            if name not in ("satpila_last_error", "satpila_version"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


class SatpilaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"satpila error {code}: {msg}")
        self.code = code


def check(rc: int) -> None:
    if rc != OK:
        raise SatpilaError(rc, load().satpila_last_error().decode(errors="replace"))
