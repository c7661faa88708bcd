"""Multipath-lifetime (T_C) management on the GPU against the oracle (Sec. II, Sec. IV-B).

drt_lifetime_windows must find the oracle's major changes and window plan; drt_synthesize_H_windows
must give the oracle's windowed H.  A decision may go either way only where the form's geometry may
decide a path's validity either way (within the flags band of a face or edge boundary, at the change
itself or at a window start) or where a path's power share sits within the amplitude bar of the
threshold; such changes and windows are allowed to differ and bound the H difference by their
amplitudes, as in the plain H comparison.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_gpu_parity import band_amplitude, compare_H_band
from test_oracle_lifetime import DT, FC, N_IN, N_OUT, T as T_WALL
from test_oracle_pins import wall_scene

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BAND = {"fp64": 1e-9, "fp32": 1e-9}
A_TOL = {"fp64": 1e-9, "fp32": 5e-3}


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    c = drt.Context(0)
    yield c
    c.close()


def prec_of(form):
    from paper_2205_00237_gb300 import drt
    return drt.FP64 if form == "fp64" else drt.FP32_BULK


def windowed_record(r, starts, band):
    """The oracle record with every path outside its window's multipath flagged; a path whose
    validity at a window start is within `band` of a boundary may be selected either way, so its
    margin is set to 0 over that window (it then only bounds the difference)."""
    T, P = r["flags"].shape
    flags, margin = r["flags"].copy(), r["margin"].copy()
    b = list(starts) + [T]
    for k in range(len(starts)):
        s0, s1 = b[k], b[k + 1]
        for p in range(P):
            if r["margin"][s0, p] < band:
                margin[s0:s1, p] = 0.0
            if r["flags"][s0, p] != 0:
                flags[s0:s1, p] |= np.uint8(0x80)
    w = dict(r)
    w["flags"], w["margin"] = flags, margin
    return w


def ambiguous_changes(r, share, band, a_tol):
    """Steps whose major-change decision may go either way in a form: a path within `band` of a
    boundary at n - 1 or n, or a validity change whose power share is within the amplitude bar of
    the threshold."""
    valid = r["flags"] == 0
    pw = np.abs(r["a"]) ** 2
    tot = np.where(valid, pw, 0.0).sum(axis=1)
    v0, v1 = valid[:-1], valid[1:]
    near = np.minimum(r["margin"][1:], r["margin"][:-1]) < band
    x = np.where(v1, pw[1:], pw[:-1])
    thr = share * np.where(v1, tot[1:, None], tot[:-1, None])
    close = np.abs(x - thr) <= 3 * a_tol * np.maximum(x, thr)
    amb = np.zeros(valid.shape[0], bool)
    amb[1:] = (near | ((v0 != v1) & close)).any(axis=1)
    return amb


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_wall_case_windows_and_H(ctx, form):
    """The hand-solved wall case: the reflection appears at step 436 and leaves at 1008."""
    sc = wall_scene([-60, 0, 2], [-41, 0, 2], vrx=(20.0, 0, 0), pec=True)
    ps = I.chains_to_pathset([[], [(I.T_R, 0)]])
    tg, fg = I.TimeGrid(0.0, DT, T_WALL), I.FreqGrid(FC, 100e6, 64)
    link = ctx.load(sc, ps)
    prec = prec_of(form)
    starts, major = link.lifetime_windows(tg, fg, 0.1, precision=prec)
    assert starts == [0, N_IN, N_OUT]
    assert list(np.flatnonzero(major)) == [N_IN, N_OUT]
    assert link.lifetime_windows(tg, fg, 0.1, 1, 400, precision=prec)[0] == [0, 400, N_IN, N_IN + 400, N_OUT]
    assert link.lifetime_windows(tg, fg, 0.1, 500, 2000, precision=prec)[0] == [0, N_OUT]
    assert link.lifetime_windows(tg, fg, 0.6, 1, 400, precision=prec)[0] == [0, 400, 800]
    r = O.extrapolate(sc, ps, tg, FC)
    for st in ([0, N_IN, N_OUT], [0], [0, 500]):
        H = link.synthesize_H_windows(tg, fg, st, prec).cpu().numpy()
        compare_H_band(H, windowed_record(r, st, BAND[form]), fg, tol=1e-4 if form == "fp64" else 1e-3)
    link.unload()


@pytest.mark.parametrize("form", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["tiny0", "canyon"])
def test_lifetime_plan_and_windowed_H(ctx, which, form):
    if which == "canyon":
        sc = I.scene_canyon(0)
        ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))
        tg, fg = I.TimeGrid(0.0, 0.5e-3, 1000), I.FreqGrid(60e9, 1e9, 256)
        # 102 validity changes over these 0.5 s, 8 of them above 1e-5 of the power (the largest 3.6e-3)
        share, mn, mx = 1e-5, 20, 300
    else:
        sc = I.scene_tiny(0)
        ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed0.npz"))
        tg, fg = I.TimeGrid(0.0, 1e-3, 1000), I.FreqGrid(28e9, 400e6, 256)
        share, mn, mx = 0.01, 50, 400
    prec = prec_of(form)
    link = ctx.load(sc, ps)
    r = O.extrapolate(sc, ps, tg, fg.fc, n_threads=8)
    starts, major = link.lifetime_windows(tg, fg, share, mn, mx, precision=prec)
    want = O.lifetime_toggles(r, share)
    amb = ambiguous_changes(r, share, BAND[form], A_TOL[form])
    assert np.array_equal(major[~amb], want[~amb])
    assert want.any()                      # the case has major changes to find
    # the host planner is the oracle's planner applied to the GPU's change flags
    assert starts == O.plan_windows(major, mn, mx)
    if np.array_equal(major, want):
        assert starts == O.plan_windows(want, mn, mx)
    H = link.synthesize_H_windows(tg, fg, starts, prec).cpu().numpy()
    compare_H_band(H, windowed_record(r, starts, BAND[form]), fg, tol=1e-4 if form == "fp64" else 1e-3)
    link.unload()


def test_window_at_every_step_is_the_plain_synthesis(ctx):
    from paper_2205_00237_gb300 import drt
    sc = I.scene_tiny(1)
    ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed1.npz"))
    tg, fg = I.TimeGrid(0.0, 1e-3, 300), I.FreqGrid(28e9, 400e6, 64)
    link = ctx.load(sc, ps)
    Hw = link.synthesize_H_windows(tg, fg, list(range(300)), drt.FP64).cpu().numpy()
    H = link.synthesize_H(tg, fg, drt.FP64).cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(H) ** 2, axis=1)) + 1e-300
    assert (np.abs(Hw - H).max(axis=1) / rms).max() < 1e-6
    link.unload()


def test_lifetime_edges_and_errors(ctx):
    from paper_2205_00237_gb300 import drt
    import torch
    sc = I.scene_tiny(0)
    ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed0.npz"))
    tg, fg = I.TimeGrid(0.0, 1e-3, 40), I.FreqGrid(28e9, 400e6, 16)
    link = ctx.load(sc, ps)
    assert link.lifetime_windows(I.TimeGrid(0.0, 1e-3, 0), fg, 0.1)[0] == []
    e = ctx.load(sc, I.empty_paths(0))
    st, mj = e.lifetime_windows(tg, fg, 0.1, 1, 10)
    assert st == [0, 10, 20, 30] and not mj.any()
    He = e.synthesize_H_windows(tg, fg, st).cpu().numpy()
    assert (He == 0).all()
    e.unload()
    for share, mn, mx in ((-1.0, 1, 10), (float("nan"), 1, 10), (0.1, 0, 10), (0.1, 5, 4)):
        with pytest.raises(drt.DrtError) as ei:
            link.lifetime_windows(tg, fg, share, mn, mx)
        assert ei.value.code == drt.DRT_EINVAL
    H = torch.empty((40, 16), dtype=torch.complex64, device="cuda")
    for bad in ([], [1], [0, 0], [0, 5, 3], [0, 40]):
        with pytest.raises(drt.DrtError) as ei:
            link.synthesize_H_windows(tg, fg, bad, H=H)
        assert ei.value.code == drt.DRT_EINVAL
    link.unload()


def test_canyon_full_size_plan(ctx):
    """The benchmarked configuration (canyon, 2000 x 0.5 ms, share 1e-5, windows of 10-150 ms), FP64."""
    from paper_2205_00237_gb300 import drt
    sc = I.scene_canyon(0)
    ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))
    tg, fg = I.grids("canyon")
    link = ctx.load(sc, ps)
    starts, major = link.lifetime_windows(tg, fg, 1e-5, 20, 300, precision=drt.FP64)
    r = O.extrapolate(sc, ps, tg, fg.fc, n_threads=16)
    want = O.lifetime_toggles(r, 1e-5)
    amb = ambiguous_changes(r, 1e-5, BAND["fp64"], A_TOL["fp64"])
    assert np.array_equal(major[~amb], want[~amb])
    assert starts == O.plan_windows(major, 20, 300) and len(starts) > 2
    link.unload()
