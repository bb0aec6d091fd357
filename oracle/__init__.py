"""Reference oracle for SAT with PILA (Vo, Breese & Moser): ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain single-threaded FP64 C++
restatement of the paper's method (Secs. II-A, II-B, III-B, III-D).  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may load it; the CUDA library never does, and the two share no
code.  Each function below names the passage it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["geometry.cpp", "sat.cpp", "sirt.cpp", "drt_bilinear.cpp"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHED_LINEAR, SCHED_GEOMETRIC, SCHED_CUBIC = 0, 1, 2
SIRT_SIMULTANEOUS, SIRT_SEQUENTIAL = 0, 1
BOME_SAME_PIXEL, BOME_INDEPENDENT = 0, 1
LEN_EXACT, LEN_BINARY16, LEN_BYTE180 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so from the C++ sources with g++ (portable flags;
    no fused multiply-add contraction, so every FP64 expression is evaluated
    as written, with the same roundings on every host)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_LIB_PATH) >= max(newest, os.path.getmtime(__file__)):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Geom(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_angles", C.c_int32), ("n_bins", C.c_int32),
                ("angles", C.POINTER(C.c_double))]


class SatParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("bome_k", C.c_int32), ("n_sweeps", C.c_int32),
                ("moves_per_sweep", C.c_int32), ("t0", C.c_double), ("tn", C.c_double),
                ("schedule", C.c_int32), ("t0_samples", C.c_int32), ("seed", C.c_uint64),
                ("bome_mode", C.c_int32), ("grid_levels", C.c_int32), ("length_format", C.c_int32)]


class SatStats(C.Structure):
    _fields_ = [("t0", C.c_double), ("tn", C.c_double), ("initial_cost", C.c_double),
                ("final_cost", C.c_double), ("final_cost_fresh", C.c_double),
                ("accepted", C.c_int64), ("proposed", C.c_int64), ("t0_found", C.c_int32)]


TRACE_DTYPE = np.dtype([("pixel", "<i4"), ("cstar", "<i4"), ("accepted", "<i4"), ("pad", "<i4"),
                        ("dS", "<f8"), ("dC", "<f8"), ("fnew", "<f8"), ("u_acc", "<f8"),
                        ("temp", "<f8"), ("scale_S", "<f8"), ("gap_S", "<f8")])

GPU_TRACE_DTYPE = np.dtype([("pixel", "<i4"), ("cstar", "<i4"), ("accepted", "<i4"), ("pad", "<i4"),
                            ("dS", "<f4"), ("dC", "<f4"), ("fnew", "<f4"), ("pad2", "<f4")])


class LockstepReport(C.Structure):
    _fields_ = [("moves", C.c_int64), ("near_ties", C.c_int64), ("pixel_mismatch", C.c_int64),
                ("hard_mismatch", C.c_int64), ("max_err_dS", C.c_double), ("max_err_dC", C.c_double),
                ("max_err_f", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_siddon_ray.argtypes = [C.c_int32, C.c_double, C.c_double, P, P, C.c_int32]
            lib.or_siddon_ray.restype = C.c_int
            lib.or_drt.argtypes = [C.POINTER(Geom), P, P]
            lib.or_pila.argtypes = [C.POINTER(Geom), P, P]
            lib.or_cost.argtypes = [C.c_int32, C.c_int32, P, P]
            lib.or_cost.restype = C.c_double
            lib.or_sirt_factor.argtypes = [C.POINTER(Geom), P, P]
            lib.or_round_length.argtypes = [C.c_int32, C.c_double]
            lib.or_round_length.restype = C.c_double
            lib.or_schedule_temp.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32]
            lib.or_schedule_temp.restype = C.c_double
            lib.or_sat_t0.argtypes = [C.POINTER(Geom), P, P, P, C.POINTER(SatParams), P, P]
            lib.or_sat_run.argtypes = [C.POINTER(Geom), P, P, P, C.POINTER(SatParams),
                                       C.POINTER(SatStats), P]
            lib.or_sat_lockstep.argtypes = [C.POINTER(Geom), P, P, P, C.POINTER(SatParams),
                                            C.c_double, C.c_double, P, C.c_int64, C.c_double,
                                            C.POINTER(LockstepReport)]
            lib.or_sirt_run.argtypes = [C.POINTER(Geom), P, P, P, C.c_int32, C.c_int32,
                                        C.c_double, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _geom(n, n_angles, n_bins, angles):
    g = Geom(n, n_angles, n_bins, None)
    keep = None
    if angles is not None:
        keep = _f64(angles)
        assert keep.shape == (n_angles,)
        g.angles = keep.ctypes.data_as(C.POINTER(C.c_double))
    return g, keep


def _mask(mask, n):
    if mask is None:
        return None
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(n * n)
    return m


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def siddon_ray(n, theta, s):
    """Chord lengths of one ray through the n x n grid (Sec. II-B, Siddon)."""
    cap = 4 * n + 8
    pix = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.float64)
    cnt = _load().or_siddon_ray(n, float(theta), float(s), _ptr(pix), _ptr(ln), cap)
    if cnt < 0:
        raise RuntimeError("siddon_ray: capacity exceeded")
    return pix[:cnt].copy(), ln[:cnt].copy()


def drt(image, n_angles, n_bins, angles=None):
    """Eq. (1): ray-driven discrete Radon transform of an n x n image -> [U, B]."""
    img = _f64(image)
    n = img.shape[0]
    g, keep = _geom(n, n_angles, n_bins, angles)
    out = np.zeros((n_angles, n_bins), dtype=np.float64)
    if _load().or_drt(C.byref(g), _ptr(img), _ptr(out)) != 0:
        raise RuntimeError("drt failed")
    return out


def drt_bilinear(image, n_angles, n_bins, angles=None):
    """The conventional DRT (bilinear interpolation, unit steps) -> [U, B]."""
    img = _f64(image)
    n = img.shape[0]
    g, keep = _geom(n, n_angles, n_bins, angles)
    out = np.zeros((n_angles, n_bins), dtype=np.float64)
    if _load().or_drt_bilinear(C.byref(g), _ptr(img), _ptr(out)) != 0:
        raise RuntimeError("drt_bilinear failed")
    return out


def sat_drt_run(pm, image, *, t0, tn=-1.0, beta=1.0, bome_k=1, n_sweeps=1, moves_per_sweep=0,
                schedule=SCHED_LINEAR, seed=0, mask=None, angles=None, trace=False):
    """SAT with a full bilinear DRT per estimate (Sec. III-A's baseline)."""
    pm_ = _f64(pm)
    img = _f64(image).copy()
    n = img.shape[0]
    g, keep = _geom(n, pm_.shape[0], pm_.shape[1], angles)
    m = _mask(mask, n)
    prm = _params(beta, bome_k, n_sweeps, moves_per_sweep, t0, tn, schedule, 200, seed)
    moves = moves_per_sweep if moves_per_sweep > 0 else (int(m.sum()) if m is not None else n * n)
    tr = np.zeros(n_sweeps * moves, dtype=TRACE_DTYPE) if trace else None
    st = SatStats()
    rc = _load().or_sat_drt_run(C.byref(g), _ptr(m), _ptr(pm_), _ptr(img), C.byref(prm), C.byref(st), _ptr(tr))
    if rc != 0:
        raise RuntimeError(f"sat_drt_run failed ({rc})")
    return img, {f: getattr(st, f) for f, _ in SatStats._fields_}, tr


def exhaustive_grid(pm, n, levels, beta=1.0, angles=None):
    """Least Eq. (4) cost over every n x n image with pixel values on the
    grid {0, beta/(L-1), ..., beta}: (min cost, images attaining it, first one)."""
    pm_ = _f64(pm)
    g, keep = _geom(n, pm_.shape[0], pm_.shape[1], angles)
    cost = C.c_double(0.0)
    cnt = C.c_int64(0)
    arg = np.zeros((n, n), dtype=np.float64)
    rc = _load().or_exhaustive_grid(C.byref(g), _ptr(pm_), C.c_int32(int(levels)), C.c_double(float(beta)),
                                    C.byref(cost), C.byref(cnt), _ptr(arg))
    if rc != 0:
        raise RuntimeError(f"exhaustive_grid failed ({rc})")
    return cost.value, cnt.value, arg


def pila(n, n_angles, n_bins, angles=None):
    """Eq. (5): the PILA, bins [P, U, 2] (int32, -1 = empty) and lengths [P, U, 2]."""
    g, keep = _geom(n, n_angles, n_bins, angles)
    bins = np.zeros((n * n, n_angles, 2), dtype=np.int32)
    lens = np.zeros((n * n, n_angles, 2), dtype=np.float64)
    if _load().or_pila(C.byref(g), _ptr(bins), _ptr(lens)) != 0:
        raise RuntimeError("pila: a (pixel, angle) met more than two rays")
    return bins, lens


def cost(pc, pm):
    """Eq. (4): RMS sinogram cost."""
    a, b = _f64(pc), _f64(pm)
    assert a.shape == b.shape and a.ndim == 2
    return _load().or_cost(a.shape[0], a.shape[1], _ptr(a), _ptr(b))


def sirt_factor(n, n_angles, n_bins, mask=None, angles=None):
    """Sec. III-D factor matrix: sum of squared lengths over the mask, per ray."""
    g, keep = _geom(n, n_angles, n_bins, angles)
    out = np.zeros((n_angles, n_bins), dtype=np.float64)
    m = _mask(mask, n)
    if _load().or_sirt_factor(C.byref(g), _ptr(m), _ptr(out)) != 0:
        raise RuntimeError("sirt_factor failed")
    return out


def schedule_temp(schedule, t0, tn, s, n_sweeps):
    """Eqs. (2), (8) (second form) and (9)."""
    return _load().or_schedule_temp(schedule, t0, tn, s, n_sweeps)


def _params(beta, bome_k, n_sweeps, moves_per_sweep, t0, tn, schedule, t0_samples, seed, bome_mode=0,
            grid_levels=0, length_format=0):
    return SatParams(float(beta), int(bome_k), int(n_sweeps), int(moves_per_sweep), float(t0),
                     float(tn), int(schedule), int(t0_samples), int(seed) & (2**64 - 1), int(bome_mode),
                     int(grid_levels), int(length_format))


def round_length(fmt: int, l: float) -> float:
    """A PILA length as stored in format fmt (LEN_EXACT, LEN_BINARY16, LEN_BYTE180)."""
    return _load().or_round_length(int(fmt), float(l))


def sat_t0(pm, image, *, beta=1.0, seed=0, t0_samples=200, mask=None, angles=None, length_format=0):
    """Eq. (8): initial temperature from Q uphill proposals on the initial image."""
    pm_, img = _f64(pm), _f64(image)
    n = img.shape[0]
    g, keep = _geom(n, pm_.shape[0], pm_.shape[1], angles)
    prm = _params(beta, 1, 0, 0, 0.0, -1.0, 0, t0_samples, seed, length_format=length_format)
    t0 = C.c_double(0.0)
    found = C.c_int32(0)
    rc = _load().or_sat_t0(C.byref(g), _ptr(_mask(mask, n)), _ptr(pm_), _ptr(img), C.byref(prm),
                           C.byref(t0), C.byref(found))
    if rc != 0:
        raise RuntimeError(f"sat_t0 failed ({rc})")
    return t0.value, found.value


def sat_run(pm, image, *, beta=1.0, bome_k=1, n_sweeps=1, moves_per_sweep=0, t0=-1.0, tn=-1.0,
            schedule=SCHED_LINEAR, t0_samples=200, seed=0, mask=None, angles=None, trace=False,
            bome_mode=BOME_SAME_PIXEL, grid_levels=0, length_format=0):
    """Steps 1-4 of Sec. II-A with Eqs. (6)-(7) and BoME; returns (image, stats, trace).
    length_format: the PILA's stored lengths (LEN_EXACT, LEN_BINARY16, LEN_BYTE180)."""
    pm_ = _f64(pm)
    img = _f64(image).copy()
    n = img.shape[0]
    g, keep = _geom(n, pm_.shape[0], pm_.shape[1], angles)
    m = _mask(mask, n)
    prm = _params(beta, bome_k, n_sweeps, moves_per_sweep, t0, tn, schedule, t0_samples, seed, bome_mode,
                  grid_levels, length_format)
    moves = moves_per_sweep if moves_per_sweep > 0 else (int(m.sum()) if m is not None else n * n)
    tr = np.zeros(n_sweeps * moves, dtype=TRACE_DTYPE) if trace else None
    st = SatStats()
    rc = _load().or_sat_run(C.byref(g), _ptr(m), _ptr(pm_), _ptr(img), C.byref(prm), C.byref(st),
                            _ptr(tr))
    if rc != 0:
        raise RuntimeError(f"sat_run failed ({rc})")
    stats = {f: getattr(st, f) for f, _ in SatStats._fields_}
    return img, stats, tr


def sat_lockstep(pm, image, gpu_trace, *, t0, tn, beta=1.0, bome_k=1, n_sweeps=1, moves_per_sweep=0,
                 schedule=SCHED_LINEAR, seed=0, mask=None, angles=None, tol=1e-5, bome_mode=BOME_SAME_PIXEL,
                 length_format=0):
    """Follow another implementation's move trace in FP64 (near-tie protocol)."""
    pm_ = _f64(pm)
    img = _f64(image).copy()
    n = img.shape[0]
    g, keep = _geom(n, pm_.shape[0], pm_.shape[1], angles)
    prm = _params(beta, bome_k, n_sweeps, moves_per_sweep, t0, tn, schedule, 200, seed, bome_mode,
                  length_format=length_format)
    tr = np.ascontiguousarray(gpu_trace, dtype=GPU_TRACE_DTYPE)
    rep = LockstepReport()
    rc = _load().or_sat_lockstep(C.byref(g), _ptr(_mask(mask, n)), _ptr(pm_), _ptr(img), C.byref(prm),
                                 float(t0), float(tn), _ptr(tr), len(tr), float(tol), C.byref(rep))
    if rc != 0:
        raise RuntimeError(f"sat_lockstep failed ({rc})")
    return img, {f: getattr(rep, f) for f, _ in LockstepReport._fields_}


def sirt_run(pm, image, n_iter, *, mode=SIRT_SIMULTANEOUS, relax=1.0, mask=None, angles=None):
    """Eqs. (10)-(11); returns (image, per-iteration Eq. (4) costs)."""
    pm_ = _f64(pm)
    img = _f64(image).copy()
    n = img.shape[0]
    g, keep = _geom(n, pm_.shape[0], pm_.shape[1], angles)
    costs = np.zeros(max(n_iter, 1), dtype=np.float64)
    rc = _load().or_sirt_run(C.byref(g), _ptr(_mask(mask, n)), _ptr(pm_), _ptr(img), n_iter, mode,
                             float(relax), _ptr(costs))
    if rc != 0:
        raise RuntimeError(f"sirt_run failed ({rc})")
    return img, costs[:n_iter]
