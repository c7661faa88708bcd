"""FP64 CPU oracle of the DRT hot path (ctypes binding of drt_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  Nothing here is shared with the CUDA library; the two meet only
through the seeded inputs of ``paper_2205_00237_gb300.inputs``.

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdrt_oracle.so")
_lock = threading.Lock()
_lib = None

METHOD_DRT, METHOD_RESOLVE = 0, 1
F_FACE, F_EDGE, F_SIDE, F_NOCONV, F_DEGEN = 1, 2, 4, 8, 16
MAX_INT = 4


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc -O2 (no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm",
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Term(C.Structure):
    _fields_ = [("r", C.c_double * 3), ("v", C.c_double * 3), ("a", C.c_double * 3)]


class _Scene(C.Structure):
    _fields_ = [("tx", _Term), ("rx", _Term), ("n_bodies", C.c_int32), ("n_materials", C.c_int32),
                ("n_faces", C.c_int32), ("n_edges", C.c_int32), ("n_tiles", C.c_int32),
                ("pad_", C.c_int32), ("bodies", C.c_void_p), ("mats", C.c_void_p),
                ("faces", C.c_void_p), ("edges", C.c_void_p), ("tiles", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_extrapolate.restype = C.c_int
            L.or_extrapolate.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_double,
                                         C.c_int32, C.c_int32] + [C.c_void_p] * 8
            L.or_synthesize_H.restype = C.c_int
            L.or_synthesize_H.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_void_p]
            L.or_fresnel_coeffs.argtypes = [C.c_double] * 5 + [dp]
            L.or_fresnel_G_ri.argtypes = [C.c_double, dp]
            L.or_transition_F_ri.argtypes = [C.c_double, dp]
            L.or_utd_ri.argtypes = [C.c_double] * 10 + [dp]
            L.or_er_norm.restype = C.c_double
            L.or_er_norm.argtypes = [C.c_double, C.c_double]
            L.or_er_amp.restype = C.c_double
            L.or_er_amp.argtypes = [C.c_double] * 5
            L.or_body_point.argtypes = [C.c_void_p, dp, C.c_double, dp]
            L.or_frame_roundtrip.argtypes = [C.c_void_p, C.c_int32, C.c_double, dp, dp, dp]
            L.or_ref_point_local.argtypes = [dp, dp, dp]
            L.or_diff_point_local.argtypes = [dp, dp, dp]
            L.or_trace_candidates.restype = C.c_int64
            L.or_trace_candidates.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
            L.or_trace.restype = C.c_int32
            L.or_trace.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_int32] + \
                [C.c_void_p] * 7
            L.or_doppler_chain.restype = C.c_double
            L.or_doppler_chain.argtypes = [C.c_int32, dp, dp, C.c_double]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _SceneHandle:
    """Keeps the contiguous arrays alive while the C structure points at them."""

    def __init__(self, scene):
        self.arrays = [np.ascontiguousarray(x) for x in
                       (scene.bodies, scene.materials, scene.faces, scene.edges, scene.tiles)]
        s = _Scene()
        for dst, src in ((s.tx, scene.tx), (s.rx, scene.rx)):
            for f in ("r", "v", "a"):
                getattr(dst, f)[:] = [float(x) for x in src[f]]
        s.n_bodies, s.n_materials, s.n_faces, s.n_edges, s.n_tiles = (len(a) for a in self.arrays)
        s.bodies, s.mats, s.faces, s.edges, s.tiles = (a.ctypes.data if len(a) else None
                                                      for a in self.arrays)
        self.s = s

    @property
    def ref(self):
        return C.byref(self.s)


def extrapolate(scene, paths, tgrid, fc, method=METHOD_DRT, n_threads=1, points=False,
                velocities=False):
    """Per-(step, path) records over the time grid; dict of [T][P] numpy arrays."""
    L = lib()
    T, P = int(tgrid.n_steps), paths.n_paths
    out = dict(tau=np.empty((T, P)), amp=np.empty((T, P, 2)), fd=np.empty((T, P)),
               ang=np.empty((T, P, 4)), flags=np.empty((T, P), np.uint8), margin=np.empty((T, P)))
    out["pts"] = np.empty((T, P, MAX_INT, 3)) if points else None
    out["vel"] = np.empty((T, P, MAX_INT + 2, 3)) if velocities else None
    h = _SceneHandle(scene)
    n_int = np.ascontiguousarray(paths.n_int, np.uint8)
    types = np.ascontiguousarray(paths.types, np.uint8)
    prims = np.ascontiguousarray(paths.prims, np.int32)
    s0 = np.ascontiguousarray(paths.s0, np.float64)
    rc = L.or_extrapolate(h.ref, P, _ptr(n_int), _ptr(types), _ptr(prims), _ptr(s0),
                          float(tgrid.t_start), float(tgrid.dt), T, float(fc), int(method),
                          int(n_threads), _ptr(out["tau"]), _ptr(out["amp"]), _ptr(out["fd"]),
                          _ptr(out["ang"]), _ptr(out["flags"]), _ptr(out["margin"]),
                          _ptr(out["pts"]), _ptr(out["vel"]))
    if rc != 0:
        raise RuntimeError(f"or_extrapolate failed: {rc}")
    out["a"] = out["amp"][..., 0] + 1j * out["amp"][..., 1]
    return out


def synthesize_H(rec, fgrid, n_threads=1):
    """Direct FP64 sum H[t][k] over the valid paths of an extrapolate() record."""
    L = lib()
    T, P = rec["tau"].shape
    H = np.empty((T, int(fgrid.n_bins), 2))
    tau = np.ascontiguousarray(rec["tau"])
    amp = np.ascontiguousarray(rec["amp"])
    flags = np.ascontiguousarray(rec["flags"])
    L.or_synthesize_H(T, P, _ptr(tau), _ptr(amp), _ptr(flags), float(fgrid.fc),
                      float(fgrid.bandwidth), int(fgrid.n_bins), int(n_threads), _ptr(H))
    return H[..., 0] + 1j * H[..., 1]


# ---------------------------------------------------------------------------- unit-level calls
PP_DOPPLER, PP_DELAY = 0, 1


def power_profile(rec, steps_per_bin, x0, dx, n_bins, kind=PP_DOPPLER):
    """Power-Doppler (PDfP, Sec. IV-A) or power-delay (PDP, Sec. IV-B) profile of an extrapolate()
    record: the incoherent sum of |a_p(t)|^2 over the valid path-steps whose instant falls in time
    bin i (steps_per_bin consecutive steps) and whose Doppler shift (Hz) or delay (s) falls in bin
    j = floor((x - x0) / dx), 0 <= j < n_bins.  Returns P[n_time_bins][n_bins] (FP64)."""
    T, P = rec["tau"].shape
    n_t = -(-T // steps_per_bin)
    out = np.zeros((n_t, n_bins))
    x = rec["fd"] if kind == PP_DOPPLER else rec["tau"]
    pw = np.abs(rec["a"]) ** 2
    for t in range(T):                      # plain loops: the definition, nothing fused
        for p in range(P):
            if rec["flags"][t, p] != 0:
                continue
            j = int(np.floor((x[t, p] - x0) / dx))
            if 0 <= j < n_bins:
                out[t // steps_per_bin, j] += pw[t, p]
    return out


def subbands(n_bins, n_sub):
    """Bin ranges [k0, k1) of n_sub near-equal sub-bands: k0 = s N / n_sub (integer division)."""
    return [(s * n_bins // n_sub, (s + 1) * n_bins // n_sub) for s in range(n_sub)]


def synthesize_H_wideband(scene, paths, tgrid, fgrid, n_sub, n_threads=1):
    """H(t, f) with the field coefficients (Fresnel, UTD, ER, lambda / 4 pi) evaluated per sub-band
    instead of once at fc: sub-band [k0, k1) spans [f_k0, f_k0 + (k1 - k0) df) of the grid
    f_k = fc - B/2 + k B/N and its coefficients are taken at the centre of that interval (one
    sub-band is the narrowband case, coefficients at fc).  Each sub-band is a plain extrapolation
    at its centre frequency and a direct sum over its own bins."""
    from types import SimpleNamespace
    T, N = int(tgrid.n_steps), int(fgrid.n_bins)
    df = fgrid.bandwidth / N
    H = np.empty((T, N), dtype=np.complex128)
    for k0, k1 in subbands(N, n_sub):
        n = k1 - k0
        fs = SimpleNamespace(fc=fgrid.fc - fgrid.bandwidth / 2 + (k0 + n / 2) * df, bandwidth=n * df, n_bins=n)
        rec = extrapolate(scene, paths, tgrid, fs.fc, n_threads=n_threads)
        H[:, k0:k1] = synthesize_H(rec, fs, n_threads=n_threads)
    return H


def lifetime_toggles(rec, share):
    """Expiry criterion of the multipath lifetime T_C (Sec. II: the time during which no major path
    appears or disappears).  major[n] (n >= 1) is True when some path is valid at one of the instants
    n - 1, n and not at the other while, at the instant where it is valid, its |a|^2 is at least
    `share` of the total |a|^2 of the valid paths of that instant."""
    T, P = rec["flags"].shape
    valid = rec["flags"] == 0
    pw = np.abs(rec["a"]) ** 2
    tot = np.zeros(T)
    for n in range(T):
        for p in range(P):
            if valid[n, p]:
                tot[n] += pw[n, p]
    major = np.zeros(T, dtype=bool)
    for n in range(1, T):
        for p in range(P):
            if valid[n, p] != valid[n - 1, p]:
                m = n if valid[n, p] else n - 1
                if pw[m, p] >= share * tot[m]:
                    major[n] = True
    return major


def plan_windows(major, min_steps, max_steps):
    """Segmentation of the span into T_C windows (Sec. IV-B divides its span into T_C windows, longer
    where the multipath is stable, shorter near LoS/NLoS transitions): a window starting at step s
    ends at the first major change n with s + min_steps <= n <= s + max_steps, else after max_steps
    steps.  Returns the first step of every window, starting with 0."""
    T = len(major)
    starts = [0]
    s = 0
    while True:
        nxt = s + max_steps
        for n in range(s + min_steps, min(s + max_steps, T - 1) + 1):
            if major[n]:
                nxt = n
                break
        if nxt >= T:
            return starts
        starts.append(nxt)
        s = nxt


def synthesize_H_windows(rec, starts, fgrid, n_threads=1):
    """H(t, f) of DRT over a span divided into T_C windows: every window re-initialises the multipath
    at its first instant (the chains valid there, as a ray-tracing run at that instant returns them)
    and extrapolates only those chains until the next window; a chain that appears inside a window is
    not seen until the next one (Sec. II, Sec. IV-B)."""
    T, P = rec["flags"].shape
    flags = rec["flags"].copy()
    bounds = list(starts) + [T]
    for k in range(len(starts)):
        s0, s1 = bounds[k], bounds[k + 1]
        for p in range(P):
            if rec["flags"][s0, p] != 0:        # not in the chain set of this window
                flags[s0:s1, p] |= np.uint8(0x80)
    r = dict(rec)
    r["flags"] = flags
    return synthesize_H(r, fgrid, n_threads=n_threads)


def fresnel(eps_r, sigma, pec, fc, cos_theta):
    o = np.empty(4)
    lib().or_fresnel_coeffs(eps_r, sigma, float(pec), fc, cos_theta, _dp(o))
    return o[0] + 1j * o[1], o[2] + 1j * o[3]


def fresnel_G(x):
    o = np.empty(2)
    lib().or_fresnel_G_ri(x, _dp(o))
    return o[0] + 1j * o[1]


def transition_F(X):
    o = np.empty(2)
    lib().or_transition_F_ri(X, _dp(o))
    return o[0] + 1j * o[1]


def utd(n, phi, phip, sinb0, L, k, eps_r=1.0, sigma=0.0, pec=True, fc=1e9):
    o = np.empty(4)
    lib().or_utd_ri(n, phi, phip, sinb0, L, k, eps_r, sigma, float(pec), fc, _dp(o))
    return o[0] + 1j * o[1], o[2] + 1j * o[3]


def er_norm(alpha, cos_theta_i):
    return lib().or_er_norm(alpha, cos_theta_i)


def er_amp(alpha, S, area, cos_theta_i, cos_psi):
    return lib().or_er_amp(alpha, S, area, cos_theta_i, cos_psi)


def body_point(body_rec, p0, t):
    b = np.ascontiguousarray(np.array(body_rec))
    o = np.empty(9)
    p = np.ascontiguousarray(p0, np.float64)
    lib().or_body_point(_ptr(b), _dp(p), t, _dp(o))
    return o.reshape(3, 3)


def frame_roundtrip(scene, face, t, state9):
    h = _SceneHandle(scene)
    i = np.ascontiguousarray(state9, np.float64)
    loc, out = np.empty(9), np.empty(9)
    lib().or_frame_roundtrip(h.ref, face, t, _dp(i), _dp(loc), _dp(out))
    return loc.reshape(3, 3), out.reshape(3, 3)


def ref_point_local(t9, r9):
    q = np.empty(9)
    lib().or_ref_point_local(_dp(np.ascontiguousarray(t9, float)), _dp(np.ascontiguousarray(r9, float)), _dp(q))
    return q.reshape(3, 3)


def diff_point_local(t9, r9):
    q = np.empty(9)
    lib().or_diff_point_local(_dp(np.ascontiguousarray(t9, float)), _dp(np.ascontiguousarray(r9, float)), _dp(q))
    return q.reshape(3, 3)


def doppler_chain(pos, vel, fc):
    pos = np.ascontiguousarray(pos, float)
    vel = np.ascontiguousarray(vel, float)
    return lib().or_doppler_chain(pos.shape[0] - 2, _dp(pos), _dp(vel), fc)


def trace(scene, t, max_order=2, with_tiles=True, report=1e-9, n_threads=8):
    """Conventional ray tracing at instant t (drt_oracle.c or_trace): the chains that are rays, as a
    PathSet in enumeration order (edge parameters at t in s0), plus the candidates a run at t could
    decide either way (decision margin below `report` m): dict(paths, index, margin, ambiguous)."""
    from paper_2205_00237_gb300 import inputs as I
    L = lib()
    h = _SceneHandle(scene)
    cap = 1 << 16
    while True:
        index = np.empty(cap, np.int64)
        found = np.empty(cap, np.uint8)
        margin = np.empty(cap)
        n_int = np.empty(cap, np.uint8)
        types = np.empty((cap, MAX_INT), np.uint8)
        prims = np.empty((cap, MAX_INT), np.int32)
        s0 = np.empty((cap, MAX_INT))
        n = L.or_trace(h.ref, float(t), int(max_order), int(bool(with_tiles)), float(report), int(n_threads), cap,
                       *[_ptr(a) for a in (index, found, margin, n_int, types, prims, s0)])
        if n <= cap:
            break
        cap = n
    o = np.argsort(index[:n], kind="stable")
    index, found, margin = index[:n][o], found[:n][o].astype(bool), margin[:n][o]
    ps = I.PathSet(n_int[:n][o].copy(), types[:n][o].copy(), prims[:n][o].copy(), s0[:n][o].copy())
    rays = ps.subset(np.nonzero(found)[0])
    return dict(paths=rays, index=index[found], margin=margin[found],
                ambiguous=index[(~found) | (margin < report)], candidates=int(L.or_trace_candidates(h.ref, int(max_order),
                                                                                                    int(bool(with_tiles)))))



def trace_chain(scene, index, with_tiles=True):
    """The chain of enumeration index `index` of or_trace (line of sight; faces, edges, tiles; ordered
    pairs of faces / edges): (n, types, prims), or None for an excluded pair."""
    from paper_2205_00237_gb300 import inputs as I
    nf, ne = len(scene.faces), len(scene.edges)
    NP, NT = nf + ne, (len(scene.tiles) if with_tiles else 0)

    def one(c):
        return (I.T_R, c) if c < nf else (I.T_D, c - nf) if c < NP else (I.T_S, c - NP)
    if index == 0:
        return []
    j = index - 1
    if j < NP + NT:
        return [one(j)]
    q = j - NP - NT
    a, b = q // NP, q % NP
    return None if a == b else [one(a), one(b)]


def synthesize_H_retraced(scene, tgrid, fgrid, starts, chains_at, n_threads=1):
    """DRT over T_C windows with a ray-tracing run at every window start: window w extrapolates the
    PathSet chains_at(w) (the rays at its first instant) over its instants.  H [T][F]."""
    from paper_2205_00237_gb300 import inputs as I
    T = int(tgrid.n_steps)
    H = np.zeros((T, int(fgrid.n_bins)), np.complex128)
    bounds = list(starts) + [T]
    for w in range(len(starts)):
        k0, k1 = bounds[w], bounds[w + 1]
        sub = I.TimeGrid(tgrid.t_start + k0 * tgrid.dt, tgrid.dt, k1 - k0)
        ps = chains_at(w)
        if ps.n_paths == 0:
            continue
        rec = extrapolate(scene, ps, sub, fgrid.fc, n_threads=n_threads)
        H[k0:k1] = synthesize_H(rec, fgrid, n_threads=n_threads)
    return H
