"""Python binding of the satpila C-ABI: argument marshalling only.

Every call forwards to libsatpila.so with the same name.  Arrays may be torch
tensors (CUDA or CPU) or numpy arrays; device tensors are passed as device
pointers, everything else as host pointers (the library stages host data).
Streams default to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import (PILA_F16, PILA_F32, PILA_U8, SAT_FLAG_AUTOTUNE, SAT_FLAG_BOME_INDEPENDENT, SAT_FLAG_HYBRID,  # noqa: F401
                   SAT_FLAG_NO_GRAPH, SAT_FLAG_TEST_STALL, SAT_FLAG_NEAR_TIES, ERR_TIMEOUT,
                   SAT_RESIDENT_AUTO,
                   SAT_RESIDENT_GLOBAL, SAT_RESIDENT_SMEM, SAT_SCHED_CUBIC, SAT_SCHED_GEOMETRIC,
                   SAT_SCHED_LINEAR, SIRT_SEQUENTIAL, SIRT_SIMULTANEOUS, SatpilaError)
from ._lib import ERR_BUSY, ERR_INVALID_ARG, ERR_NOT_FOUND, ERR_PENDING  # noqa: F401
from ._lib import (SAT_FLAG_WINDOW_GROUPS, SAT_PLAN_PIPE_1, SAT_PLAN_PIPE_2, SAT_PLAN_PIPE_4,  # noqa: F401
                   SAT_PLAN_RULES, SAT_PLAN_WINDOW_G2, SAT_PLAN_WINDOW_G4, SAT_PLAN_WINDOW_GLOBAL,
                   SAT_PLAN_WINDOW_HYBRID, SAT_PLAN_WINDOW_SMEM, SAT_PLAN_WINDOW_SMEM_G2, SAT_PLAN_WINDOW_SMEM_G4)
from ._lib import PROBE_SECTOR, PROBE_STREAM, SAT_SERVER_PER_CLASS  # noqa: F401

TRACE_DTYPE = np.dtype([("pixel", "<i4"), ("cstar", "<i4"), ("accepted", "<i4"), ("pad", "<i4"),
                        ("dS", "<f4"), ("dC", "<f4"), ("fnew", "<f4"), ("pad2", "<f4")])


def _is_tensor(x) -> bool:
    return hasattr(x, "data_ptr") and hasattr(x, "is_contiguous")


def _ptr(x, dtype=None):
    if x is None:
        return None
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(x.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise TypeError(f"expected {np.dtype(dtype).name}, got {x.dtype}")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype).name}, got {x.dtype}")
        return x.ctypes.data_as(C.c_void_p)
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    try:
        import torch

        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class Pila:
    """Owns a PILA handle; released by pila_free (or on garbage collection)."""

    def __init__(self, handle, n, n_angles, n_bins, precision):
        self.handle = handle
        self.n, self.n_angles, self.n_bins, self.precision = n, n_angles, n_bins, precision

    def close(self):
        if self.handle:
            L.load().pila_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pila_build(n, n_angles, n_bins, precision=PILA_F32, angles=None, mask=None, stream=None) -> Pila:
    lib = L.load()
    g = L.PilaGeom(int(n), int(n_angles), int(n_bins), None, None)
    keep = []
    if angles is not None:
        a = np.ascontiguousarray(angles, dtype=np.float64)
        keep.append(a)
        g.angles_rad = a.ctypes.data_as(C.POINTER(C.c_double))
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        keep.append(m)
        g.mask = m.ctypes.data_as(C.POINTER(C.c_uint8))
    h = C.c_void_p()
    L.check(lib.pila_build(C.byref(g), int(precision), _stream(stream), C.byref(h)))
    return Pila(h, int(n), int(n_angles), int(n_bins), int(precision))


def pila_free(p: Pila) -> None:
    p.close()


def pila_info(p: Pila) -> dict:
    info = L.PilaInfo()
    L.check(L.load().pila_info(p.handle, C.byref(info)))
    return {f: getattr(info, f) for f, _ in L.PilaInfo._fields_ if f != "pad"}


def pila_export(p: Pila, bins=None, lens=None, stream=None):
    """(bins [n*n, U, 2] int32 with -1 for empty, lens [n*n, U, 2] float32);
    bins/lens may be given (host arrays or device tensors)."""
    P = p.n * p.n
    if bins is None:
        bins = np.zeros((P, p.n_angles, 2), dtype=np.int32)
    if lens is None:
        lens = np.zeros((P, p.n_angles, 2), dtype=np.float32)
    L.check(L.load().pila_export(p.handle, _ptr(bins, np.int32), _ptr(lens, np.float32), _stream(stream)))
    return bins, lens


def pila_forward(p: Pila, images, out=None, stream=None):
    """DRT (Eq. (1)) through the PILA, float64 [n_images, U, B]."""
    n_img = int(images.shape[0]) if images.ndim == 3 else 1
    if out is None:
        if _is_tensor(images) and images.is_cuda:
            import torch

            out = torch.empty((n_img, p.n_angles, p.n_bins), dtype=torch.float64, device=images.device)
        else:
            out = np.zeros((n_img, p.n_angles, p.n_bins), dtype=np.float64)
    L.check(L.load().pila_forward(p.handle, n_img, _ptr(images, np.float32), _ptr(out, np.float64),
                                  _stream(stream)))
    return out


def pila_sirt_factor(p: Pila, stream=None) -> np.ndarray:
    w = np.zeros((p.n_angles, p.n_bins), dtype=np.float64)
    L.check(L.load().pila_sirt_factor(p.handle, _ptr(w), _stream(stream)))
    return w


def sat_params(*, beta=1.0, bome_k=1, n_sweeps=1, moves_per_sweep=0, t0=-1.0, tn=-1.0,
               schedule=SAT_SCHED_LINEAR, t0_samples=200, seed=0, resync_every=0,
               residency=SAT_RESIDENT_AUTO, flags=0, trace_chain=-1, group_warps=0, pipeline_depth=0, trace=None,
               sweep_cost=None, plan=0, wait_ms=0):
    return L.SatParams(float(beta), int(bome_k), int(n_sweeps), int(moves_per_sweep), float(t0), float(tn),
                       int(schedule), int(t0_samples), int(seed) & (2**64 - 1), int(resync_every),
                       int(residency), int(flags), int(trace_chain), int(group_warps), int(pipeline_depth), _ptr(trace),
                       _ptr(sweep_cost), int(plan), int(wait_ms))


def sat_run(p: Pila, sino_meas, images, stream=None, sync=True, **kw) -> list[dict] | None:
    """Anneal images (in place) against sino_meas; returns per-chain stats.

    sino_meas: float32 [n_chains, U, B]; images: float32 [n_chains, n, n].
    Keyword arguments are the fields of sat_params (trace: a buffer of
    TRACE_DTYPE records or a byte tensor of the same size; sweep_cost:
    float64 [n_chains, n_sweeps]).  sync=False passes no stats: with device
    tensors the call is then asynchronous on the stream and returns None."""
    n_chains = int(images.shape[0]) if images.ndim == 3 else 1
    prm = sat_params(**kw)
    stats = (L.SatStats * max(n_chains, 1))() if sync else None
    L.check(L.load().sat_run(p.handle, n_chains, _ptr(sino_meas, np.float32), _ptr(images, np.float32),
                             C.byref(prm), C.cast(stats, C.c_void_p) if sync else None, _stream(stream)))
    if not sync:
        return None
    return [{f: getattr(s, f) for f, _ in L.SatStats._fields_} for s in stats[:n_chains]]


def sat_run_ptrs(p: Pila, sinos, images, stream=None, sync=True, **kw) -> list[dict] | None:
    """sat_run over chains given one buffer each: sinos[c] float32 [U, B] and
    images[c] float32 [n, n] (annealed in place), tensors or arrays, host or
    device; the same results as sat_run on the stacked batch."""
    if len(sinos) != len(images):
        raise ValueError("one sinogram per image")
    n_chains = len(images)
    sp = (C.c_void_p * max(n_chains, 1))(*[_ptr(x, np.float32) for x in sinos])
    ip = (C.c_void_p * max(n_chains, 1))(*[_ptr(x, np.float32) for x in images])
    prm = sat_params(**kw)
    stats = (L.SatStats * max(n_chains, 1))() if sync else None
    L.check(L.load().sat_run_ptrs(p.handle, n_chains, sp, ip, C.byref(prm),
                                  C.cast(stats, C.c_void_p) if sync else None, _stream(stream)))
    if not sync:
        return None
    return [{f: getattr(s, f) for f, _ in L.SatStats._fields_} for s in stats[:n_chains]]


def drt_bilinear(images, n_angles, n_bins, stream=None):
    """Bilinear-interpolation DRT (Sec. III-A's conventional forward model) of
    device images [items, n, n] -> float32 [items, U, B] tensor."""
    import torch

    n = int(images.shape[-1])
    items = int(images.shape[0]) if images.ndim == 3 else 1
    out = torch.empty((items, n_angles, n_bins), dtype=torch.float32, device=images.device)
    L.check(L.load().drt_bilinear(n, n_angles, n_bins, None, items, _ptr(images, np.float32), _ptr(out, np.float32),
                                  _stream(stream)))
    return out


def sat_drt_run(sino_meas, images, *, mask=None, stream=None, **kw) -> list[dict]:
    """SAT with a full bilinear DRT per estimate (the baseline the PILA
    replaces); device tensors; keyword arguments as sat_params (t0 > 0)."""
    n_chains = int(images.shape[0]) if images.ndim == 3 else 1
    n = int(images.shape[-1])
    U, B = int(sino_meas.shape[-2]), int(sino_meas.shape[-1])
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    prm = sat_params(**kw)
    stats = (L.SatStats * max(n_chains, 1))()
    L.check(L.load().sat_drt_run(n, U, B, _ptr(m), n_chains, _ptr(sino_meas, np.float32), _ptr(images, np.float32),
                                 C.byref(prm), C.cast(stats, C.c_void_p), _stream(stream)))
    return [{f: getattr(s, f) for f, _ in L.SatStats._fields_} for s in stats[:n_chains]]


def fbp(sino, n, stream=None):
    """FBP images [items, n, n] (float32 tensor) of device sinograms [items, U, B]."""
    import torch

    items = int(sino.shape[0]) if sino.ndim == 3 else 1
    U, B = int(sino.shape[-2]), int(sino.shape[-1])
    out = torch.empty((items, n, n), dtype=torch.float32, device=sino.device)
    L.check(L.load().fbp(int(n), U, B, None, items, _ptr(sino, np.float32), _ptr(out, np.float32), _stream(stream)))
    return out


def fbp_prior(images, mask_frac, stream=None):
    """(init, mask, beta) from FBP images: start image, spatial constraint
    (pixels above mask_frac * max) and the pixel range beta = max."""
    import torch

    items = int(images.shape[0]) if images.ndim == 3 else 1
    n = int(images.shape[-1])
    init = torch.empty((items, n, n), dtype=torch.float32, device=images.device)
    mask = torch.empty((items, n, n), dtype=torch.uint8, device=images.device)
    beta = torch.empty((items,), dtype=torch.float32, device=images.device)
    L.check(L.load().fbp_prior(n, items, _ptr(images, np.float32), float(mask_frac), _ptr(init, np.float32),
                               _ptr(mask, np.uint8), _ptr(beta, np.float32), _stream(stream)))
    return init, mask, beta


class Server:
    """Continuous-batching annealing server (sat_server_* of include/satpila.h).

    submit() copies the request's arrays and returns a ticket; poll()/wait()
    return (image [n, n] float32, result dict) once the request is done."""

    def __init__(self, device=0, max_active=0, stages_per_tick=0, queue_limit=0, mem_budget=0, flags=0):
        cfg = L.SatServerCfg(int(device), int(max_active), int(stages_per_tick), int(queue_limit), int(mem_budget),
                             int(flags))
        h = C.c_void_p()
        L.check(L.load().sat_server_create(C.byref(cfg), C.byref(h)))
        self.handle = h
        self.sizes = {}

    def submit(self, sino, *, n, precision=PILA_F32, mask=None, image=None, angles=None, **kw) -> int:
        sino = np.ascontiguousarray(sino, dtype=np.float32)
        U, B = sino.shape
        keep = []

        def arr(x, dtype):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=dtype)
            keep.append(a)
            return a.ctypes.data_as(C.c_void_p)

        req = L.SatRequest(int(n), int(U), int(B), int(precision), arr(angles, np.float64), arr(mask, np.uint8),
                           arr(sino, np.float32), arr(image, np.float32), sat_params(**kw))
        t = C.c_uint64()
        L.check(L.load().sat_server_submit(self.handle, C.byref(req), C.byref(t)))
        self.sizes[t.value] = int(n)
        return t.value

    def _collect(self, ticket, rc, img, res):
        if rc == L.ERR_PENDING:
            return None
        L.check(rc)
        self.sizes.pop(ticket, None)
        st = {f: getattr(res.stats, f) for f, _ in L.SatStats._fields_}
        st.update(submit_ms=res.submit_ms, admit_ms=res.admit_ms, done_ms=res.done_ms)
        return img, st

    def poll(self, ticket):
        """(image, result) if done, else None."""
        n = self.sizes.get(ticket, 1)
        img = np.zeros((n, n), dtype=np.float32)
        res = L.SatResult()
        rc = L.load().sat_server_poll(self.handle, C.c_uint64(ticket), img.ctypes.data_as(C.c_void_p), C.byref(res))
        return self._collect(ticket, rc, img, res)

    def wait(self, ticket, timeout_ms=-1):
        """(image, result) once done; None if timeout_ms passes first."""
        n = self.sizes.get(ticket, 1)
        img = np.zeros((n, n), dtype=np.float32)
        res = L.SatResult()
        rc = L.load().sat_server_wait(self.handle, C.c_uint64(ticket), int(timeout_ms),
                                      img.ctypes.data_as(C.c_void_p), C.byref(res))
        return self._collect(ticket, rc, img, res)

    def info(self) -> dict:
        st = L.SatServerStats()
        L.check(L.load().sat_server_info(self.handle, C.byref(st)))
        return {f: getattr(st, f) for f, _ in L.SatServerStats._fields_}

    def close(self):
        if self.handle:
            L.load().sat_server_destroy(self.handle)
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


def sirt_run(p: Pila, sino_meas, images, *, n_iter=1, mode=SIRT_SIMULTANEOUS, relax=1.0, costs=None,
             stream=None) -> None:
    """SIRT with PILA (Eqs. (10)-(11)); images updated in place."""
    n_sl = int(images.shape[0]) if images.ndim == 3 else 1
    prm = L.SirtParams(int(n_iter), int(mode), float(relax), 0)
    L.check(L.load().sirt_run(p.handle, n_sl, _ptr(sino_meas, np.float32), _ptr(images, np.float32),
                              C.byref(prm), _ptr(costs, np.float64), _stream(stream)))


def sirt_run_noalloc(p: Pila, sino_meas, images, *, n_iter=1, mode=SIRT_SIMULTANEOUS, relax=1.0, costs=None,
                     stream=None) -> None:
    """sirt_run for callers that cannot allocate device memory: device
    tensors only, asynchronous on the stream, scratch in the library's static
    device array (see include/satpila.h)."""
    n_sl = int(images.shape[0]) if images.ndim == 3 else 1
    prm = L.SirtParams(int(n_iter), int(mode), float(relax), 0)
    L.check(L.load().sirt_run_noalloc(p.handle, n_sl, _ptr(sino_meas, np.float32), _ptr(images, np.float32),
                                      C.byref(prm), _ptr(costs, np.float64), _stream(stream)))


def probe_read(buf, kind, loads=1 << 28, region_bytes=0, stream=None) -> float:
    """Read rate (GB/s) over a device tensor: kind PROBE_STREAM
    (consecutive 16-byte loads) or PROBE_SECTOR (one 32-byte sector at a
    pseudo-random place per load, each warp inside its own region of
    region_bytes; 0: the whole buffer)."""
    if not _is_tensor(buf):
        raise TypeError("probe_read takes a device tensor")
    g = C.c_double()
    L.check(L.load().satpila_probe_read(_ptr(buf), int(buf.numel() * buf.element_size()), int(kind),
                                        int(region_bytes), int(loads), C.byref(g), _stream(stream)))
    return g.value


def probe_smem(kind, loads=1 << 30, stream=None) -> float:
    """Shared-memory 4-byte load rate (GB/s, all SMs): kind 0 conflict-free,
    1 pseudo-random words."""
    g = C.c_double()
    L.check(L.load().satpila_probe_smem(int(kind), int(loads), C.byref(g), _stream(stream)))
    return g.value
