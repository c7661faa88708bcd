"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances, FP64 form: delay 1e-12 relative; complex amplitude 1e-9 relative; Doppler 1e-3 Hz
(the oracle evaluates the product formula directly, ~1e-5 Hz of rounding at 60 GHz); angles 2e-6 rad
(stored as FP32); interaction points 1e-8 m; flags exact except within 1e-9 m of a face or edge
boundary; H(t, f) within 1e-4 of RMS_f |H_ref(t, .)| per time step (FP32 synthesis from FP64-reduced
phases).

FP32-bulk form (FP32 deltas on FP64 anchors every 16 steps): carrier phase 2 pi fc tau within 1e-3
rad on valid path-steps; delay 1e-8 relative on valid path-steps (1e-7 on all well-sided ones); amplitude 5e-3 relative; Doppler 0.1 Hz; angles 2e-6
rad; points 1e-3 m; flags exact except within 1e-9 m of a boundary (the FP32 kernels hand every
step whose validity margin is within their position-error bound to the FP64 redo); |H| within 1e-4
and H within 1e-3 of RMS_f |H_ref(t, .)|.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    c = drt.Context(0)
    yield c
    c.close()


def canyon():
    return I.scene_canyon(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))


def compare_records(g, r, where=None, min_ray_frac=0.5):
    """g: GPU dict (torch tensors), r: oracle dict (numpy)."""
    tau = g["tau"].cpu().numpy()
    flags = g["flags"].cpu().numpy()
    amp = g["amp"].cpu().numpy().astype(np.float64)
    a = amp[..., 0] + 1j * amp[..., 1]
    fd = g["doppler"].cpu().numpy().astype(np.float64)
    ang = g["angles"].cpu().numpy().astype(np.float64)
    # Flags are compared everywhere outside the 1e-9 m boundary band.  Geometry is compared where
    # the chain is still a ray up to leaving a finite face or edge: with a vertex on the wrong side
    # of a wall or wedge no stationary path exists and the image construction can be arbitrarily
    # ill-conditioned (grazing), so those path-steps only carry their flags.
    far = r["margin"] > 1e-9
    if where is not None:
        far &= where
    assert np.array_equal(flags[far], r["flags"][far])
    ok = (r["flags"] & (O.F_DEGEN | O.F_SIDE | O.F_NOCONV)) == 0
    if where is not None:
        ok &= where
    assert ok.sum() >= min_ray_frac * ok.size
    rel = np.abs(tau - r["tau"]) / r["tau"]
    assert rel[ok].max() < 1e-12
    valid = ok & (r["flags"] == 0)
    assert (np.abs(a - r["a"]) <= 1e-9 * np.abs(r["a"]) + 1e-30)[valid].all()
    assert np.abs(fd - r["fd"])[ok].max() < 1e-3
    dang = np.abs(np.angle(np.exp(1j * (ang - r["ang"]))))
    assert dang[ok].max() < 2e-6
    if g.get("points") is not None and r.get("pts") is not None:
        pts = g["points"].cpu().numpy()
        d = np.abs(pts - r["pts"])[ok]
        assert np.nanmax(d) < 1e-8
        assert np.array_equal(np.isnan(pts[ok]), np.isnan(r["pts"][ok]))


def compare_H(Hg, Href, tol=1e-4, mag_tol=None):
    Hg = np.asarray(Hg, np.complex128)
    rms = np.sqrt(np.mean(np.abs(Href) ** 2, axis=1, keepdims=True))
    nz = rms[:, 0] > 0
    err = np.abs(Hg - Href)[nz] / rms[nz]
    assert err.max() < tol, err.max()
    if mag_tol is not None:
        emag = np.abs(np.abs(Hg) - np.abs(Href))[nz] / rms[nz]
        assert emag.max() < mag_tol, emag.max()
    assert np.all(np.abs(Hg[~nz]) == 0)


def band_amplitude(r):
    """|a| of each path-step, widened to its neighbouring instants: the bound on what a path-step
    that may be decided either way can contribute (at a degenerate instant, where a path leaves its
    face through a corner, the oracle's own amplitude is zero but the limit from either side is not)."""
    a = np.abs(r["a"])
    if a.shape[0] > 1:
        a = np.maximum(a, np.maximum(np.vstack([a[1:], a[-1:]]), np.vstack([a[:1], a[:-1]])))
    return a


def compare_H_band(Hg, r, fg, tol=1e-3, mag_tol=1e-4, band=1e-9):
    """H against the oracle.  A path-step within `band` m of a validity boundary (face or edge rim,
    side plane; 1e-9 m in both forms) may be decided either way, so the oracle sum leaves those
    path-steps out and each row may differ from it by at most tol (and mag_tol for |H|) of the row
    RMS plus the summed magnitude of their amplitudes."""
    Hg = np.asarray(Hg, np.complex128)
    near = r["margin"] < band
    r_far = dict(r)
    r_far["flags"] = np.where(near, np.uint8(0x80), r["flags"]).astype(np.uint8)
    Href = O.synthesize_H(r_far, fg, n_threads=8)
    Hall = O.synthesize_H(r, fg, n_threads=8)
    rms = np.sqrt(np.mean(np.abs(Hall) ** 2, axis=1))
    slack = np.where(near, band_amplitude(r), 0.0).sum(axis=1)
    nz = rms > 0
    err = (np.abs(Hg - Href).max(axis=1) - slack)[nz] / rms[nz]
    assert err.max() < tol, err.max()
    emag = (np.abs(np.abs(Hg) - np.abs(Href)).max(axis=1) - slack)[nz] / rms[nz]
    assert emag.max() < mag_tol, emag.max()
    assert np.all(np.abs(Hg[~nz]) <= slack[~nz, None] * (1 + 1e-6))
    return int(near.sum())


def compare_H_pair(H1, H2, r, tol=2e-4, band=1e-9):
    """Two FP32-bulk results of the same link (e.g. different chunk lengths): equal within tol of the
    row RMS plus the amplitudes of the path-steps either may decide differently (near a boundary)."""
    H1, H2 = np.asarray(H1, np.complex128), np.asarray(H2, np.complex128)
    slack = np.where(r["margin"] < band, band_amplitude(r), 0.0).sum(axis=1)
    rms = np.sqrt(np.mean(np.abs(H2) ** 2, axis=1)) + 1e-300
    err = (np.abs(H1 - H2).max(axis=1) - slack) / rms
    assert err.max() < tol, err.max()


def compare_records_bulk(g, r, fc):
    """FP32-bulk records against the oracle (see the module docstring for the bars)."""
    tau = g["tau"].cpu().numpy()
    flags = g["flags"].cpu().numpy()
    amp = g["amp"].cpu().numpy().astype(np.float64)
    a = amp[..., 0] + 1j * amp[..., 1]
    fd = g["doppler"].cpu().numpy().astype(np.float64)
    ang = g["angles"].cpu().numpy().astype(np.float64)
    far = r["margin"] > 1e-9
    assert np.array_equal(flags[far], r["flags"][far])
    ok = (r["flags"] & (O.F_DEGEN | O.F_SIDE | O.F_NOCONV)) == 0
    valid = ok & (r["flags"] == 0)
    assert valid.sum() > 0.5 * valid.size
    rel = np.abs(tau - r["tau"]) / r["tau"]
    assert rel[valid].max() < 1e-8 and rel[ok].max() < 1e-7
    assert (2 * np.pi * fc * np.abs(tau - r["tau"]))[valid].max() < 1e-3
    # FP32 coefficients: 5e-3 relative, except near a null of the path's own amplitude (the UTD
    # terms and the ER lobe cancel there), where the bar is 1e-5 of the path's peak over the horizon
    peak = np.where(valid, np.abs(r["a"]), 0.0).max(axis=0, keepdims=True)
    assert (np.abs(a - r["a"]) <= 5e-3 * np.abs(r["a"]) + 1e-5 * peak)[valid].all()
    assert np.abs(fd - r["fd"])[ok].max() < 0.1
    assert np.abs(np.angle(np.exp(1j * (ang - r["ang"]))))[ok].max() < 2e-6
    if g.get("points") is not None and r.get("pts") is not None:
        d = np.abs(g["points"].cpu().numpy() - r["pts"])[ok]
        assert np.nanmax(d) < 1e-3


@pytest.mark.parametrize("seed", [0, 1])
def test_tiny_scene_full_horizon(ctx, seed):
    """28 GHz tiny scene, 1000 x 1 ms, 256 bins over 400 MHz: every output against the oracle."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc = I.scene_tiny(seed)
    ps = I.PathSet.from_npz(os.path.join(GOLD, f"pathset_tiny_seed{seed}.npz"))
    tg, fg = I.grids("tiny")
    link = ctx.load(sc, ps)
    g = link.extrapolate(tg, fg, drt.FP64, points=True)
    H = link.synthesize_H(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    r = O.extrapolate(sc, ps, tg, fg.fc, points=True, n_threads=8)
    compare_records(g, r)
    compare_H(H.cpu().numpy(), O.synthesize_H(r, fg, n_threads=8))
    link.unload()


def test_tiny_candidates_flags_and_geometry(ctx):
    """All 50 candidate chains of order <= 2 (most of them not valid rays): flags and geometry."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc = I.scene_tiny(0)
    ps = I.chains_tiny(sc)
    tg, fg = I.TimeGrid(0.0, 0.01, 100), I.FreqGrid(28e9, 400e6, 256)
    link = ctx.load(sc, ps)
    g = link.extrapolate(tg, fg, drt.FP64, points=True)
    H = link.synthesize_H(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    r = O.extrapolate(sc, ps, tg, fg.fc, points=True, n_threads=8)
    compare_records(g, r, min_ray_frac=0.05)
    compare_H(H.cpu().numpy(), O.synthesize_H(r, fg, n_threads=8))
    link.unload()


def test_canyon_sampled_horizon(ctx):
    """Full-3D canyon (512 chains with R, D, S and multi-diffraction segments, 60 GHz, 512 bins over
    1 GHz) at 48 instants spread over the 1 s horizon, with a ragged path count (509)."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc, ps = canyon()
    ps = ps.subset(np.arange(3, 512))
    fg = I.FreqGrid(60e9, 1e9, 512)
    tg = I.TimeGrid(0.0, 0.5e-3 * 41, 48)
    link = ctx.load(sc, ps)
    g = link.extrapolate(tg, fg, drt.FP64, points=True)
    H = link.synthesize_H(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    r = O.extrapolate(sc, ps, tg, fg.fc, points=True, n_threads=8)
    compare_records(g, r)
    compare_H(H.cpu().numpy(), O.synthesize_H(r, fg, n_threads=8))
    link.unload()


def test_canyon_full_size_sampled_rows(ctx):
    """The benchmark's launch: 512 chains x 2000 steps x 512 bins in one call; 16 sampled time rows
    checked against the oracle (records and H)."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc, ps = canyon()
    tg, fg = I.grids("canyon")
    link = ctx.load(sc, ps)
    g = link.extrapolate(tg, fg, drt.FP64)
    H = link.synthesize_H(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    rows = np.linspace(0, tg.n_steps - 1, 16).astype(int)
    for t in rows:
        r = O.extrapolate(sc, ps, I.TimeGrid(t * tg.dt, tg.dt, 1), fg.fc, n_threads=8)
        gi = {k: (v[t:t + 1] if v is not None else None) for k, v in g.items()}
        compare_records(gi, r)
        compare_H(H[t:t + 1].cpu().numpy(), O.synthesize_H(r, fg))
    link.unload()


@pytest.mark.parametrize("n_bins", [1, 17, 100])
def test_ragged_frequency_tiles(ctx, n_bins):
    from paper_2205_00237_gb300 import drt
    import torch
    sc, ps = canyon()
    ps = ps.subset(np.arange(0, 70))
    tg, fg = I.TimeGrid(0.1, 0.01, 5), I.FreqGrid(60e9, 1e9 * n_bins / 512, n_bins)
    link = ctx.load(sc, ps)
    H = link.synthesize_H(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    r = O.extrapolate(sc, ps, tg, fg.fc, n_threads=8)
    compare_H(H.cpu().numpy(), O.synthesize_H(r, fg))
    link.unload()


def test_empty_and_degenerate_inputs(ctx):
    """No paths (H = 0), no steps, and a line-of-sight-only link."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc = I.scene_tiny(0)
    fg = I.FreqGrid(28e9, 400e6, 64)
    link = ctx.load(sc, I.empty_paths(0))
    H = link.synthesize_H(I.TimeGrid(0, 1e-3, 4), fg, drt.FP64)
    torch.cuda.synchronize()
    assert torch.all(H == 0)
    link.unload()
    los = I.chains_to_pathset([[]])
    link = ctx.load(sc, los)
    out = link.extrapolate(I.TimeGrid(0, 1e-3, 0), fg, drt.FP64)
    assert out["tau"].numel() == 0
    tg = I.TimeGrid(0.0, 1e-3, 10)
    g = link.extrapolate(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    d = np.linalg.norm(np.asarray(sc.rx["r"]) + np.outer(np.arange(10) * 1e-3, sc.rx["v"]) - sc.tx["r"], axis=1)
    lam = I.C0 / fg.fc
    a = g["amp"].cpu().numpy()[:, 0]
    assert np.allclose(a[:, 0], lam / (4 * math.pi * d), rtol=1e-12, atol=0) and np.all(a[:, 1] == 0)
    link.unload()


def test_invalid_inputs_are_rejected(ctx):
    from paper_2205_00237_gb300 import drt
    sc = I.scene_tiny(0)
    bad = I.chains_to_pathset([[(I.T_R, 99)]])
    with pytest.raises(drt.DrtError) as e:
        ctx.load(sc, bad)
    assert e.value.code == drt.DRT_EINVAL
    sc2 = I.scene_tiny(0)
    sc2.faces["n"][1] = [0.0, 0.0, 2.0]
    with pytest.raises(drt.DrtError):
        ctx.load(sc2, I.chains_to_pathset([[]]))
    link = ctx.load(sc, I.chains_to_pathset([[]]))
    with pytest.raises(drt.DrtError):
        link.synthesize_H(I.TimeGrid(0, 1e-3, 4), I.FreqGrid(28e9, 400e6, 0), drt.FP64)
    with pytest.raises(drt.DrtError):
        link.extrapolate(I.TimeGrid(0, 1e-3, 4), I.FreqGrid(28e9, 400e6, 8), 7)
    link.unload()
    with pytest.raises(drt.DrtError) as e:
        link.handle = 12345
        link.unload()
    assert e.value.code == drt.DRT_ENOTFOUND


def test_host_output_entry_point(ctx):
    """drt_synthesize_H_host (host buffers, copies inside the call) equals the device entry point."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc, ps = canyon()
    tg, fg = I.TimeGrid(0.0, 1e-3, 64), I.FreqGrid(60e9, 1e9, 512)
    link = ctx.load(sc, ps)
    Hd = link.synthesize_H(tg, fg, drt.FP64)
    Hh = link.synthesize_H_host(tg, fg, drt.FP64)
    torch.cuda.synchronize()
    assert torch.equal(Hd.cpu(), Hh)
    link.unload()


def test_hbm_budget_is_enforced():
    from paper_2205_00237_gb300 import drt
    sc, ps = canyon()
    with drt.Context(0, hbm_budget=1 << 16) as c:
        with pytest.raises(drt.DrtError) as e:
            c.load(sc, ps)
        assert e.value.code == drt.DRT_ENOMEM


@pytest.mark.parametrize("which", ["tiny0", "tiny1", "canyon"])
def test_fp32_bulk_form(ctx, which):
    """FP32-bulk form over a full horizon: records and H against the FP64 oracle."""
    from paper_2205_00237_gb300 import drt
    import torch
    if which == "canyon":
        sc, ps = canyon()
        tg, fg = I.grids("canyon")
    else:
        seed = int(which[-1])
        sc = I.scene_tiny(seed)
        ps = I.PathSet.from_npz(os.path.join(GOLD, f"pathset_tiny_seed{seed}.npz"))
        tg, fg = I.grids("tiny")
    link = ctx.load(sc, ps)
    g = link.extrapolate(tg, fg, drt.FP32_BULK, points=True)
    H = link.synthesize_H(tg, fg, drt.FP32_BULK)
    torch.cuda.synchronize()
    r = O.extrapolate(sc, ps, tg, fg.fc, points=True, n_threads=8)
    compare_records_bulk(g, r, fg.fc)
    compare_H_band(H.cpu().numpy(), r, fg)
    link.unload()


def test_fp32_bulk_ragged_grid(ctx):
    """A time grid that starts off t0 and ends inside a 16-step chunk, ragged path count."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc, ps = canyon()
    ps = ps.subset(np.arange(0, 45))
    tg, fg = I.TimeGrid(0.0123, 0.5e-3, 37), I.FreqGrid(60e9, 1e9, 100)
    link = ctx.load(sc, ps)
    g = link.extrapolate(tg, fg, drt.FP32_BULK)
    H = link.synthesize_H(tg, fg, drt.FP32_BULK)
    torch.cuda.synchronize()
    r = O.extrapolate(sc, ps, tg, fg.fc, n_threads=8)
    compare_records_bulk(g, r, fg.fc)
    compare_H_band(H.cpu().numpy(), r, fg)
    link.unload()

