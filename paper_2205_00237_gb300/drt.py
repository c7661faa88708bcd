"""Thin Python binding of the DRT C ABI (include/drt.h) over ctypes.

Argument marshalling only: every step of the hot path runs in libdrt.so's CUDA kernels.  PyTorch
provides device memory (tensors) and streams.  There is no CPU fallback: if the library has not been
built (``__graft_entry__.build()`` / ``paper_2205_00237_gb300.build.build()``) or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdrt.so")

DRT_OK, DRT_EINVAL, DRT_ENOMEM, DRT_ECUDA, DRT_EBUSY, DRT_ETIMEOUT, DRT_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6
FP64, FP32_BULK = 0, 1
F_FACE, F_EDGE, F_SIDE, F_NOCONV, F_DEGEN = 1, 2, 4, 8, 16

# every symbol include/drt.h declares
EXPORTS = ["drt_create", "drt_destroy", "drt_last_error", "drt_load_paths", "drt_unload", "drt_extrapolate",
           "drt_synthesize_H", "drt_synthesize_H_host", "drt_link_info", "drt_probe_peak", "drt_profile_enable",
           "drt_profile_read", "drt_synthesize_H_noalloc", "drt_batch_create", "drt_batch_run", "drt_batch_info",
           "drt_batch_destroy", "drt_serve_start", "drt_serve_stop", "drt_submit", "drt_poll", "drt_wait",
           "drt_serve_stats_read", "drt_power_profile", "drt_lifetime_windows", "drt_synthesize_H_windows",
           "drt_synthesize_H_wideband", "drt_trace_paths", "drt_synthesize_H_retraced", "drt_batch_tuning",
           "drt_profile_timeline"]
PP_DOPPLER, PP_DELAY = 0, 1


class DrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"drt error {code}: {msg}")
        self.code = code


class _Term(C.Structure):
    _fields_ = [("r", C.c_double * 3), ("v", C.c_double * 3), ("a", C.c_double * 3)]


class _Scene(C.Structure):
    _fields_ = [("tx", _Term), ("rx", _Term), ("n_bodies", C.c_int32), ("n_materials", C.c_int32),
                ("n_faces", C.c_int32), ("n_edges", C.c_int32), ("n_tiles", C.c_int32),
                ("reserved", C.c_int32), ("bodies", C.c_void_p), ("materials", C.c_void_p),
                ("faces", C.c_void_p), ("edges", C.c_void_p), ("tiles", C.c_void_p)]


class _PathSet(C.Structure):
    _fields_ = [("n_paths", C.c_int32), ("reserved", C.c_int32), ("n_int", C.c_void_p),
                ("types", C.c_void_p), ("prims", C.c_void_p), ("s0", C.c_void_p)]


class _TimeGrid(C.Structure):
    _fields_ = [("t_start", C.c_double), ("dt", C.c_double), ("n_steps", C.c_int32), ("reserved", C.c_int32)]


class _FreqGrid(C.Structure):
    _fields_ = [("fc", C.c_double), ("bandwidth", C.c_double), ("n_bins", C.c_int32), ("reserved", C.c_int32)]


class _Outputs(C.Structure):
    _fields_ = [("tau", C.c_void_p), ("amp", C.c_void_p), ("doppler", C.c_void_p), ("angles", C.c_void_p),
                ("flags", C.c_void_p), ("points", C.c_void_p)]


class _PowerGrid(C.Structure):
    _fields_ = [("steps_per_bin", C.c_int32), ("n_bins", C.c_int32), ("x0", C.c_double), ("dx", C.c_double),
                ("kind", C.c_int32), ("reserved", C.c_int32)]


class _LifetimeParams(C.Structure):
    _fields_ = [("share", C.c_double), ("min_steps", C.c_int32), ("max_steps", C.c_int32)]


class _Traced(C.Structure):
    _fields_ = [("cap", C.c_int32), ("n_found", C.c_int32), ("n_int", C.c_void_p), ("types", C.c_void_p),
                ("prims", C.c_void_p), ("s0", C.c_void_p)]


class _Request(C.Structure):
    _fields_ = [("link", C.c_uint64), ("tgrid", _TimeGrid), ("fgrid", _FreqGrid), ("H", C.c_void_p),
                ("records", _Outputs), ("precision", C.c_int32), ("reserved", C.c_int32)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("batch_requests", C.c_int32), ("t_submit", C.c_double),
                ("t_launch", C.c_double), ("t_done", C.c_double)]


class _ServeStats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("submitted", "completed", "launches", "queued", "in_flight",
                                          "arena_bytes", "arena_used", "arena_peak")]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libdrt.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(path)
        vp, st = C.c_void_p, C.c_int32
        L.drt_create.argtypes = [C.POINTER(vp), C.c_int32, C.c_uint64]
        L.drt_create.restype = st
        L.drt_destroy.argtypes = [vp]
        L.drt_destroy.restype = None
        L.drt_last_error.argtypes = []
        L.drt_last_error.restype = C.c_char_p
        L.drt_load_paths.argtypes = [vp, vp, vp, C.POINTER(C.c_uint64)]
        L.drt_load_paths.restype = st
        L.drt_unload.argtypes = [vp, C.c_uint64]
        L.drt_unload.restype = st
        L.drt_extrapolate.argtypes = [vp, C.c_uint64, vp, vp, vp, C.c_int32, vp]
        L.drt_extrapolate.restype = st
        L.drt_synthesize_H.argtypes = [vp, C.c_uint64, vp, vp, vp, C.c_int32, vp]
        L.drt_synthesize_H.restype = st
        L.drt_synthesize_H_host.argtypes = [vp, C.c_uint64, vp, vp, vp, C.c_int32, vp]
        L.drt_synthesize_H_host.restype = st
        L.drt_link_info.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int32)]
        L.drt_link_info.restype = st
        L.drt_probe_peak.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_double)]
        L.drt_probe_peak.restype = st
        L.drt_synthesize_H_noalloc.argtypes = [vp, C.c_uint64, vp, vp, vp, C.c_int32, vp]
        L.drt_synthesize_H_noalloc.restype = st
        L.drt_profile_enable.argtypes = [vp, C.c_int32]
        L.drt_profile_enable.restype = st
        L.drt_profile_read.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.drt_profile_read.restype = st
        L.drt_profile_timeline.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.drt_profile_timeline.restype = st
        L.drt_batch_create.argtypes = [vp, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(_TimeGrid),
                                       C.POINTER(_FreqGrid), C.POINTER(vp), C.c_int32, C.POINTER(vp)]
        L.drt_batch_create.restype = st
        L.drt_batch_run.argtypes = [vp, vp, C.c_int32, vp]
        L.drt_batch_run.restype = st
        L.drt_batch_info.argtypes = [vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_uint64), C.POINTER(C.c_float),
                                     C.POINTER(C.c_int64)]
        L.drt_batch_info.restype = st
        L.drt_batch_tuning.argtypes = [vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_float)]
        L.drt_batch_tuning.restype = st
        L.drt_batch_destroy.argtypes = [vp, vp]
        L.drt_batch_destroy.restype = None
        L.drt_serve_start.argtypes = [vp, C.c_uint64, C.c_int32, C.c_int32]
        L.drt_serve_start.restype = st
        L.drt_serve_stop.argtypes = [vp]
        L.drt_serve_stop.restype = st
        L.drt_submit.argtypes = [vp, C.POINTER(_Request), C.POINTER(C.c_uint64)]
        L.drt_submit.restype = st
        L.drt_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(_Result)]
        L.drt_poll.restype = st
        L.drt_wait.argtypes = [vp, C.c_uint64, C.c_uint32, C.POINTER(_Result)]
        L.drt_wait.restype = st
        L.drt_serve_stats_read.argtypes = [vp, C.POINTER(_ServeStats)]
        L.drt_serve_stats_read.restype = st
        L.drt_power_profile.argtypes = [vp, C.c_uint64, vp, vp, C.POINTER(_PowerGrid), vp, C.c_int32, vp]
        L.drt_power_profile.restype = st
        L.drt_lifetime_windows.argtypes = [vp, C.c_uint64, vp, vp, C.POINTER(_LifetimeParams), C.c_int32, vp, vp,
                                           C.c_int32, C.POINTER(C.c_int32), vp]
        L.drt_lifetime_windows.restype = st
        L.drt_synthesize_H_windows.argtypes = [vp, C.c_uint64, vp, vp, vp, C.c_int32, vp, C.c_int32, vp]
        L.drt_synthesize_H_windows.restype = st
        L.drt_synthesize_H_wideband.argtypes = [vp, C.c_uint64, vp, vp, C.c_int32, vp, C.c_int32, vp]
        L.drt_synthesize_H_wideband.restype = st
        L.drt_trace_paths.argtypes = [vp, C.c_uint64, C.c_double, C.c_int32, C.c_int32, C.POINTER(_Traced), vp]
        L.drt_trace_paths.restype = st
        L.drt_synthesize_H_retraced.argtypes = [vp, C.c_uint64, vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, vp,
                                                C.c_int32, vp]
        L.drt_synthesize_H_retraced.restype = st
        _lib = L
        return L


def _check(rc):
    if rc != DRT_OK:
        raise DrtError(rc, load_library().drt_last_error().decode())


def _tg(tg: I.TimeGrid):
    return _TimeGrid(float(tg.t_start), float(tg.dt), int(tg.n_steps), 0)


def _fg(fg: I.FreqGrid):
    return _FreqGrid(float(fg.fc), float(fg.bandwidth), int(fg.n_bins), 0)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _check_buf(X, shape, dtype, device=None, name="H"):
    """A caller-provided buffer the library writes through a raw pointer: right dtype, contiguous, at
    least `shape` elements, and on the context's device (device=None: host memory)."""
    import torch
    if not isinstance(X, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if X.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {X.dtype}")
    if not X.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    need = 1
    for d in shape:
        need *= int(d)
    if X.numel() < need:
        raise ValueError(f"{name} holds {X.numel()} elements, {need} ({'x'.join(map(str, shape))}) required")
    if device is None:
        if X.is_cuda:
            raise ValueError(f"{name} must be in host memory")
    elif not X.is_cuda or X.device.index != int(device):
        raise ValueError(f"{name} must be a CUDA tensor on device {device}")


class Context:
    """A device context: owns loaded links, scratch and the HBM budget (drt_create)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        L = load_library()
        h = C.c_void_p()
        _check(L.drt_create(C.byref(h), int(device), int(hbm_budget)))
        self._h = h
        self.device = device

    def close(self):
        if self._h:
            load_library().drt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load(self, scene: I.Scene, paths: I.PathSet) -> "Link":
        """drt_load_paths: validate, pack and copy one link's scene and chains to the device."""
        arrays = [np.ascontiguousarray(x) for x in
                  (scene.bodies, scene.materials, scene.faces, scene.edges, scene.tiles)]
        s = _Scene()
        for dst, src in ((s.tx, scene.tx), (s.rx, scene.rx)):
            for f in ("r", "v", "a"):
                getattr(dst, f)[:] = [float(x) for x in src[f]]
        s.n_bodies, s.n_materials, s.n_faces, s.n_edges, s.n_tiles = (len(a) for a in arrays)
        s.bodies, s.materials, s.faces, s.edges, s.tiles = (a.ctypes.data if len(a) else None for a in arrays)
        n_int = np.ascontiguousarray(paths.n_int, np.uint8)
        types = np.ascontiguousarray(paths.types, np.uint8)
        prims = np.ascontiguousarray(paths.prims, np.int32)
        s0 = np.ascontiguousarray(paths.s0, np.float64)
        ps = _PathSet(int(paths.n_paths), 0, n_int.ctypes.data, types.ctypes.data, prims.ctypes.data,
                      s0.ctypes.data)
        out = C.c_uint64()
        _check(load_library().drt_load_paths(self._h, C.byref(s), C.byref(ps), C.byref(out)))
        return Link(self, out.value, int(paths.n_paths))

    def profile(self, on: bool = True):
        """drt_profile_enable: bracket every kernel launch with CUDA events."""
        _check(load_library().drt_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """drt_profile_read: {kind: (launches, total ms)} since the last read.  Kinds: pose (pose
        tables), extrapolate (the per-path-step kernel), synth (H synthesis), base (FP64 warm starts,
        FP32-bulk chunk anchors and FP64 redo)."""
        counts = (C.c_int64 * 4)()
        ms = (C.c_double * 4)()
        _check(load_library().drt_profile_read(self._h, counts, ms))
        names = ("pose", "extrapolate", "synth", "base")
        return {names[k]: (int(counts[k]), float(ms[k])) for k in range(4)}

    def profile_timeline(self, cap: int = 256):
        """drt_profile_timeline: [(kind name, start ms, end ms)] of the bracketed launch groups since
        the last profile_read, in issue order, times after the start of the first; keeps the record."""
        n = C.c_int32(0)
        kind = (C.c_int32 * cap)()
        t0 = (C.c_double * cap)()
        t1 = (C.c_double * cap)()
        _check(load_library().drt_profile_timeline(self._h, int(cap), C.byref(n), kind, t0, t1))
        names = ("pose", "extrapolate", "synth", "base")
        return [(names[kind[i]], float(t0[i]), float(t1[i])) for i in range(min(cap, n.value))]

    def batch(self, links, tgrids, fgrids, Hs, precision: int = FP32_BULK) -> "Batch":
        """drt_batch_create: one batched synthesis plan over loaded links; Hs are complex64 CUDA
        tensors [T_i][F_i] (kept referenced by the plan).  Autotunes on the device (synchronous)."""
        import torch
        n = len(links)
        for i, (t, f, h) in enumerate(zip(tgrids, fgrids, Hs)):
            _check_buf(h, (t.n_steps, f.n_bins), torch.complex64, self.device, name=f"Hs[{i}]")
        ids = (C.c_uint64 * n)(*[lk.handle for lk in links])
        tgs = (_TimeGrid * n)(*[_tg(t) for t in tgrids])
        fgs = (_FreqGrid * n)(*[_fg(f) for f in fgrids])
        hs = (C.c_void_p * n)(*[h.data_ptr() for h in Hs])
        out = C.c_void_p()
        _check(load_library().drt_batch_create(self._h, n, ids, tgs, fgs, hs, int(precision), C.byref(out)))
        return Batch(self, out, list(Hs))

    def serve_start(self, pool_bytes: int = 0, n_slots: int = 4, max_batch: int = 256):
        """drt_serve_start: start the serving loop with an arena of pool_bytes (0 = default)."""
        _check(load_library().drt_serve_start(self._h, int(pool_bytes), int(n_slots), int(max_batch)))

    def serve_stop(self):
        """drt_serve_stop: finish every submitted request and end the serving loop."""
        _check(load_library().drt_serve_stop(self._h))

    def submit(self, link: "Link", tg: I.TimeGrid, fg: I.FreqGrid, H, records: dict | None = None,
               precision: int = FP32_BULK) -> int:
        """drt_submit: queue one prediction request; H (complex64 CUDA tensor [T][F]) and the optional
        record tensors must stay alive until the request is done.  Returns the ticket."""
        import torch
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, self.device)
        rec = records or {}
        req = _Request(link.handle, _tg(tg), _fg(fg), H.data_ptr(),
                       _Outputs(*(_dptr(rec.get(k)) for k in ("tau", "amp", "doppler", "angles", "flags", "points"))),
                       int(precision), 0)
        t = C.c_uint64()
        _check(load_library().drt_submit(self._h, C.byref(req), C.byref(t)))
        return t.value

    @staticmethod
    def _result(r: _Result) -> dict:
        return dict(status=r.status, batch_requests=r.batch_requests, t_submit=r.t_submit, t_launch=r.t_launch,
                    t_done=r.t_done, latency=r.t_done - r.t_submit)

    def poll(self, ticket: int):
        """drt_poll: None while pending, else the result dict (the ticket is then retired)."""
        done, r = C.c_int32(), _Result()
        _check(load_library().drt_poll(self._h, int(ticket), C.byref(done), C.byref(r)))
        return self._result(r) if done.value else None

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        """drt_wait: block until the request is done (raises DrtError DRT_ETIMEOUT on expiry)."""
        r = _Result()
        _check(load_library().drt_wait(self._h, int(ticket), int(timeout_ms), C.byref(r)))
        return self._result(r)

    def serve_stats(self) -> dict:
        st = _ServeStats()
        _check(load_library().drt_serve_stats_read(self._h, C.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in _ServeStats._fields_}

    def probe_peak(self, kind: int, blocks: int = 152 * 16) -> float:
        f = C.c_double()
        _check(load_library().drt_probe_peak(self._h, int(kind), int(blocks), C.byref(f)))
        return f.value


class Link:
    """One loaded link (scene + chains resident on the device)."""

    def __init__(self, ctx: Context, handle: int, n_paths: int):
        self.ctx, self.handle, self.n_paths = ctx, handle, n_paths

    def unload(self):
        if self.handle:
            _check(load_library().drt_unload(self.ctx._h, self.handle))
            self.handle = 0

    def extrapolate(self, tg: I.TimeGrid, fg: I.FreqGrid, precision: int = FP64, points: bool = False,
                    out: dict | None = None, stream=None) -> dict:
        """drt_extrapolate into torch CUDA tensors ([T][P] in the caller's path order)."""
        import torch
        T, P = int(tg.n_steps), self.n_paths
        dev = torch.device("cuda", self.ctx.device)
        if out is None:
            ft = torch.float64 if precision == FP64 else torch.float32
            out = dict(tau=torch.empty((T, P), dtype=torch.float64, device=dev),
                       amp=torch.empty((T, P, 2), dtype=ft, device=dev),
                       doppler=torch.empty((T, P), dtype=ft, device=dev),
                       angles=torch.empty((T, P, 4), dtype=torch.float32, device=dev),
                       flags=torch.empty((T, P), dtype=torch.uint8, device=dev),
                       points=torch.empty((T, P, 4, 3), dtype=torch.float64, device=dev) if points else None)
        o = _Outputs(*(_dptr(out.get(k)) for k in ("tau", "amp", "doppler", "angles", "flags", "points")))
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_extrapolate(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs), C.byref(o),
                                               int(precision), _stream_ptr(stream)))
        return out

    def synthesize_H(self, tg: I.TimeGrid, fg: I.FreqGrid, precision: int = FP64, H=None, stream=None):
        """drt_synthesize_H into a complex64 CUDA tensor [T][F]."""
        import torch
        if H is None:
            H = torch.empty((int(tg.n_steps), int(fg.n_bins)), dtype=torch.complex64,
                            device=torch.device("cuda", self.ctx.device))
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, self.ctx.device)
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_synthesize_H(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs), _dptr(H),
                                               int(precision), _stream_ptr(stream)))
        return H

    def synthesize_H_host(self, tg: I.TimeGrid, fg: I.FreqGrid, precision: int = FP64, H=None, stream=None):
        """drt_synthesize_H_host into a (pinned) host complex64 tensor [T][F]; synchronous."""
        import torch
        if H is None:
            H = torch.empty((int(tg.n_steps), int(fg.n_bins)), dtype=torch.complex64, pin_memory=True)
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, None)
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_synthesize_H_host(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs),
                                                    _dptr(H), int(precision), _stream_ptr(stream)))
        return H

    def power_profile(self, tg: I.TimeGrid, fg: I.FreqGrid, steps_per_bin: int, x0: float, dx: float, n_bins: int,
                      kind: int = PP_DOPPLER, precision: int = FP64, P=None, stream=None):
        """drt_power_profile: power-Doppler (kind PP_DOPPLER) or power-delay (PP_DELAY) profile into a
        float64 CUDA tensor [ceil(T / steps_per_bin)][n_bins]."""
        import torch
        n_t = -(-int(tg.n_steps) // int(steps_per_bin)) if int(steps_per_bin) > 0 else 0   # the call rejects < 1
        if P is None:
            P = torch.empty((n_t, int(n_bins)), dtype=torch.float64, device=torch.device("cuda", self.ctx.device))
        _check_buf(P, (n_t, max(int(n_bins), 0)), torch.float64, self.ctx.device, name="P")
        g = _PowerGrid(int(steps_per_bin), int(n_bins), float(x0), float(dx), int(kind), 0)
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_power_profile(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs), C.byref(g),
                                                _dptr(P), int(precision), _stream_ptr(stream)))
        return P

    def lifetime_windows(self, tg: I.TimeGrid, fg: I.FreqGrid, share: float, min_steps: int = 1,
                         max_steps: int | None = None, precision: int = FP64, stream=None):
        """drt_lifetime_windows: (window starts as a list of steps, per-step major-change flags as a
        numpy bool array) of the multipath-lifetime plan."""
        T = int(tg.n_steps)
        lp = _LifetimeParams(float(share), int(min_steps), int(max_steps if max_steps is not None else max(T, 1)))
        major = np.zeros(max(T, 1), dtype=np.uint8)
        cap = max(T, 1)
        starts = np.zeros(cap, dtype=np.int32)
        nw = C.c_int32(0)
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_lifetime_windows(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs), C.byref(lp),
                                                   int(precision), major.ctypes.data, starts.ctypes.data, cap,
                                                   C.byref(nw), _stream_ptr(stream)))
        return [int(x) for x in starts[:nw.value]], major[:T].astype(bool)

    def synthesize_H_windows(self, tg: I.TimeGrid, fg: I.FreqGrid, starts, precision: int = FP64, H=None,
                             stream=None):
        """drt_synthesize_H_windows: H over the T_C windows starting at `starts` (steps)."""
        import torch
        if H is None:
            H = torch.empty((int(tg.n_steps), int(fg.n_bins)), dtype=torch.complex64,
                            device=torch.device("cuda", self.ctx.device))
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, self.ctx.device)
        st_ = np.ascontiguousarray(np.asarray(starts, dtype=np.int32))
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_synthesize_H_windows(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs),
                                                       st_.ctypes.data if st_.size else None, int(st_.size),
                                                       _dptr(H), int(precision), _stream_ptr(stream)))
        return H

    def synthesize_H_wideband(self, tg: I.TimeGrid, fg: I.FreqGrid, n_sub: int, precision: int = FP64, H=None,
                              stream=None):
        """drt_synthesize_H_wideband: H with field coefficients per sub-band (n_sub sub-bands)."""
        import torch
        if H is None:
            H = torch.empty((int(tg.n_steps), int(fg.n_bins)), dtype=torch.complex64,
                            device=torch.device("cuda", self.ctx.device))
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, self.ctx.device)
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_synthesize_H_wideband(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs),
                                                        int(n_sub), _dptr(H), int(precision), _stream_ptr(stream)))
        return H

    def trace_paths(self, t: float, max_order: int = 2, with_tiles: bool = True, cap: int = 1 << 16,
                    stream=None) -> I.PathSet:
        """drt_trace_paths: conventional ray tracing at instant t over this link's scene; the rays found,
        in enumeration order, as a PathSet (edge parameters at t in s0)."""
        while True:
            n_int = np.zeros(cap, np.uint8)
            types = np.zeros((cap, 4), np.uint8)
            prims = np.zeros((cap, 4), np.int32)
            s0 = np.zeros((cap, 4), np.float64)
            tr = _Traced(int(cap), 0, n_int.ctypes.data, types.ctypes.data, prims.ctypes.data, s0.ctypes.data)
            _check(load_library().drt_trace_paths(self.ctx._h, self.handle, float(t), int(max_order),
                                                  1 if with_tiles else 0, C.byref(tr), _stream_ptr(stream)))
            if tr.n_found <= cap:
                n = tr.n_found
                return I.PathSet(n_int[:n].copy(), types[:n].copy(), prims[:n].copy(), s0[:n].copy())
            cap = tr.n_found

    def synthesize_H_retraced(self, tg: I.TimeGrid, fg: I.FreqGrid, starts, max_order: int = 2,
                              with_tiles: bool = True, precision: int = FP64, H=None, stream=None):
        """drt_synthesize_H_retraced: H over T_C windows with a ray-tracing run at every window start."""
        import torch
        if H is None:
            H = torch.empty((int(tg.n_steps), int(fg.n_bins)), dtype=torch.complex64,
                            device=torch.device("cuda", self.ctx.device))
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, self.ctx.device)
        st_ = np.ascontiguousarray(np.asarray(starts, dtype=np.int32))
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_synthesize_H_retraced(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs),
                                                        st_.ctypes.data if st_.size else None, int(st_.size),
                                                        int(max_order), 1 if with_tiles else 0, _dptr(H),
                                                        int(precision), _stream_ptr(stream)))
        return H

    def synthesize_H_noalloc(self, tg: I.TimeGrid, fg: I.FreqGrid, H, precision: int = FP64, stream=None):
        """drt_synthesize_H_noalloc: the same H as synthesize_H without any device allocation, for
        callers that cannot allocate at call time; H is a caller-provided complex64 CUDA tensor."""
        import torch
        _check_buf(H, (tg.n_steps, fg.n_bins), torch.complex64, self.ctx.device)
        tgs, fgs = _tg(tg), _fg(fg)
        _check(load_library().drt_synthesize_H_noalloc(self.ctx._h, self.handle, C.byref(tgs), C.byref(fgs),
                                                       _dptr(H), int(precision), _stream_ptr(stream)))
        return H


class Batch:
    """A batched synthesis plan (drt_batch_create) over several loaded links."""

    def __init__(self, ctx: Context, handle, Hs):
        self.ctx, self._h, self.Hs = ctx, handle, Hs

    def run(self, use_graph: bool = True, stream=None):
        """drt_batch_run: every stage of the batch on `stream` (replayed from a CUDA graph)."""
        _check(load_library().drt_batch_run(self.ctx._h, self._h, 1 if use_graph else 0, _stream_ptr(stream)))

    def info(self, redo: bool = False) -> dict:
        v, b, ms, r = C.c_int32(), C.c_uint64(), C.c_float(), C.c_int64()
        _check(load_library().drt_batch_info(self.ctx._h, self._h, C.byref(v), C.byref(b), C.byref(ms),
                                             C.byref(r) if redo else None))
        out = dict(variant=v.value, scratch_bytes=b.value, tune_ms=ms.value)
        if redo:
            out["redo_steps"] = r.value
        div, cms = C.c_int32(), (C.c_float * 3)()
        _check(load_library().drt_batch_tuning(self.ctx._h, self._h, C.byref(div), cms))
        out["chunk_div"] = div.value
        out["chunk_ns_per_step"] = [float(x) for x in cms]
        return out

    def close(self):
        if self._h:
            load_library().drt_batch_destroy(self.ctx._h, self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
