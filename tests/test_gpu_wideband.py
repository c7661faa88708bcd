"""Wideband coefficients on the GPU (drt_synthesize_H_wideband) against the oracle's per-sub-band sum.

Every sub-band of the GPU result must match the oracle's extrapolation at that sub-band's centre
frequency, synthesised over the sub-band's bins, within the form's H bars, taken against the RMS of
the whole row (FP64: 1e-4; FP32-bulk: 1e-3, magnitude 1e-4, boundary path-steps bounded by their
amplitudes).
"""
import os
from types import SimpleNamespace

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_gpu_parity import band_amplitude

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BAND = {"fp64": 1e-9, "fp32": 1e-9}


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    c = drt.Context(0)
    yield c
    c.close()


def case(which):
    if which == "canyon":
        return (I.scene_canyon(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz")),
                I.TimeGrid(0.0, 0.5e-3, 600), I.FreqGrid(60e9, 4e9, 256))
    seed = int(which[-1])
    return (I.scene_tiny(seed), I.PathSet.from_npz(os.path.join(GOLD, f"pathset_tiny_seed{seed}.npz")),
            I.TimeGrid(0.0, 1e-3, 1000), I.FreqGrid(28e9, 2e9, 100))


def compare_wideband(Hg, sc, ps, tg, fg, n_sub, tol, band, mag_tol=1e-4):
    """Row error over the whole band, normalised by the row's RMS over all bins (the narrowband H
    metric); in each sub-band the path-steps within `band` of a boundary are left out of the oracle
    sum and bound the difference by their amplitudes."""
    df = fg.bandwidth / fg.n_bins
    T, N = Hg.shape
    Href, Hall = np.empty((T, N), complex), np.empty((T, N), complex)
    err, emag = np.zeros(T), np.zeros(T)
    for k0, k1 in O.subbands(N, n_sub):
        n = k1 - k0
        fs = SimpleNamespace(fc=fg.fc - fg.bandwidth / 2 + (k0 + n / 2) * df, bandwidth=n * df, n_bins=n)
        r = O.extrapolate(sc, ps, tg, fs.fc, n_threads=8)
        near = r["margin"] < band
        r_far = dict(r)
        r_far["flags"] = np.where(near, np.uint8(0x80), r["flags"]).astype(np.uint8)
        Href[:, k0:k1] = O.synthesize_H(r_far, fs, n_threads=8)
        Hall[:, k0:k1] = O.synthesize_H(r, fs, n_threads=8)
        slack = np.where(near, band_amplitude(r), 0.0).sum(axis=1)
        d = Hg[:, k0:k1] - Href[:, k0:k1]
        err = np.maximum(err, np.abs(d).max(axis=1) - slack)
        emag = np.maximum(emag, np.abs(np.abs(Hg[:, k0:k1]) - np.abs(Href[:, k0:k1])).max(axis=1) - slack)
    rms = np.sqrt(np.mean(np.abs(Hall) ** 2, axis=1))
    nz = rms > 0
    assert (err[nz] / rms[nz]).max() < tol, (err[nz] / rms[nz]).max()
    assert (emag[nz] / rms[nz]).max() < mag_tol, (emag[nz] / rms[nz]).max()


@pytest.mark.parametrize("form", ["fp64", "fp32"])
@pytest.mark.parametrize("which,n_sub", [("tiny0", 3), ("tiny1", 100), ("canyon", 4), ("canyon", 5)])
def test_wideband_matches_oracle_per_subband(ctx, which, n_sub, form):
    from paper_2205_00237_gb300 import drt
    import torch
    sc, ps, tg, fg = case(which)
    prec = drt.FP64 if form == "fp64" else drt.FP32_BULK
    link = ctx.load(sc, ps)
    H = link.synthesize_H_wideband(tg, fg, n_sub, prec)
    torch.cuda.synchronize()
    compare_wideband(H.cpu().numpy().astype(np.complex128), sc, ps, tg, fg, n_sub,
                     tol=1e-4 if form == "fp64" else 1e-3, band=BAND[form])
    link.unload()


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_one_subband_is_the_plain_synthesis(ctx, form):
    from paper_2205_00237_gb300 import drt
    sc, ps, tg, fg = case("canyon")
    prec = drt.FP64 if form == "fp64" else drt.FP32_BULK
    link = ctx.load(sc, ps)
    Hw = link.synthesize_H_wideband(tg, fg, 1, prec).cpu().numpy()
    H = link.synthesize_H(tg, fg, prec).cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(H) ** 2, axis=1)) + 1e-300
    assert (np.abs(Hw - H).max(axis=1) / rms).max() < 1e-6   # FP32 redo additions: order only
    link.unload()


def test_wideband_rejects_bad_subband_counts(ctx):
    from paper_2205_00237_gb300 import drt
    sc, ps, tg, fg = case("tiny0")
    link = ctx.load(sc, ps)
    for n_sub in (0, -1, fg.n_bins + 1):
        with pytest.raises(drt.DrtError) as ei:
            link.synthesize_H_wideband(tg, fg, n_sub)
        assert ei.value.code == drt.DRT_EINVAL
    link.unload()


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_canyon_full_size_sampled_rows(ctx, form):
    """The benchmarked configuration (canyon, 2000 x 0.5 ms, 512 bins over 1 GHz, 4 sub-bands):
    sampled rows of the GPU result against the oracle's per-sub-band sums at those instants."""
    from paper_2205_00237_gb300 import drt
    import torch
    sc = I.scene_canyon(0)
    ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))
    tg, fg = I.grids("canyon")
    prec = drt.FP64 if form == "fp64" else drt.FP32_BULK
    link = ctx.load(sc, ps)
    H = link.synthesize_H_wideband(tg, fg, 4, prec)
    torch.cuda.synchronize()
    rows = [0, 777, 1500, tg.n_steps - 1]
    Hg = H[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.complex128)
    for j, t in enumerate(rows):
        compare_wideband(Hg[j:j + 1], sc, ps, I.TimeGrid(tg.t_start + t * tg.dt, tg.dt, 1), fg, 4,
                         tol=1e-4 if form == "fp64" else 1e-3, band=BAND[form])
    link.unload()
