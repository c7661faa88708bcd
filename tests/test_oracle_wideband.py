"""Pins of the oracle's wideband synthesis: field coefficients per sub-band (the narrowband reading
evaluates Fresnel, UTD, ER and lambda / 4 pi once at fc).

Sub-band [k0, k1) of the grid f_k = fc - B/2 + k B/N spans [f_k0, f_k0 + (k1 - k0) df); its
coefficients are taken at the centre of that span.  Checked against Friis (LoS and a PEC reflection:
|a| = c / (4 pi f_s d)), against the textbook TE Fresnel coefficient of a lossy wall at each
sub-band's centre (eps_c = eps_r - j sigma / (2 pi f eps0)), and against the narrowband sum for one
sub-band.
"""
import math
import os

import numpy as np

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_oracle_pins import wall_scene

C0 = I.C0
EPS0 = 8.8541878128e-12
FC, B, N = 28e9, 4e9, 64       # a wide band so that the per-sub-band coefficients differ visibly
TX, RX = [-30, 0, 2], [10, 0, 2]


def centres(n_sub):
    df = B / N
    return [(k0, k1, FC - B / 2 + (k0 + (k1 - k0) / 2) * df) for k0, k1 in O.subbands(N, n_sub)]


def test_subband_split():
    assert O.subbands(64, 4) == [(0, 16), (16, 32), (32, 48), (48, 64)]
    assert O.subbands(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert O.subbands(5, 5) == [(k, k + 1) for k in range(5)]


def test_one_subband_is_the_narrowband_sum():
    sc = I.scene_tiny(1)
    ps = I.PathSet.from_npz(os.path.join(os.path.dirname(__file__), "golden", "pathset_tiny_seed1.npz"))
    tg, fg = I.TimeGrid(0.0, 1e-3, 50), I.FreqGrid(FC, 400e6, 32)
    Hw = O.synthesize_H_wideband(sc, ps, tg, fg, 1)
    H = O.synthesize_H(O.extrapolate(sc, ps, tg, FC), fg)
    assert np.allclose(Hw, H, rtol=1e-13, atol=0)


def run(chains, pec=True):
    sc = wall_scene(TX, RX, pec=pec)
    ps = I.chains_to_pathset(chains)
    tg = I.TimeGrid(0.0, 1e-3, 3)
    return sc, ps, tg, I.FreqGrid(FC, B, N)


def test_los_friis_per_subband():
    sc, ps, tg, fg = run([[]])
    d = 40.0
    for n_sub in (1, 4, 5, N):
        H = O.synthesize_H_wideband(sc, ps, tg, fg, n_sub)
        for k0, k1, fs in centres(n_sub):
            assert np.allclose(np.abs(H[:, k0:k1]), C0 / (4 * np.pi * fs * d), rtol=1e-12)
            if k1 - k0 > 1:   # phase step across a sub-band: exp(-j 2 pi df tau)
                r = H[:, k0 + 1:k1] / H[:, k0:k1 - 1]
                assert np.allclose(r, np.exp(-2j * np.pi * (B / N) * d / C0), rtol=1e-9, atol=0)


def test_pec_reflection_friis_per_subband():
    sc, ps, tg, fg = run([[(I.T_R, 0)]])
    dr = math.hypot(40.0, 20.0)
    H = O.synthesize_H_wideband(sc, ps, tg, fg, 4)
    for k0, k1, fs in centres(4):
        assert np.allclose(np.abs(H[:, k0:k1]), C0 / (4 * np.pi * fs * dr), rtol=1e-12)


def test_lossy_reflection_follows_fresnel_per_subband():
    """A lossy wall (eps_r 4, sigma 0.02 S/m): |a_s| = c / (4 pi f_s d_R) |R_TE(f_s)|, the conductivity
    term of eps_c falling as 1 / f_s across the band."""
    sc, ps, tg, fg = run([[(I.T_R, 0)]], pec=False)
    eps_r, sigma = float(sc.materials[0]["eps_r"]), float(sc.materials[0]["sigma"])
    dr = math.hypot(40.0, 20.0)
    ct = 20.0 / dr
    H = O.synthesize_H_wideband(sc, ps, tg, fg, 8)
    mags = []
    for k0, k1, fs in centres(8):
        ec = eps_r - 1j * sigma / (2 * np.pi * fs * EPS0)
        root = np.sqrt(ec - (1 - ct * ct))
        rte = (ct - root) / (ct + root)
        want = C0 / (4 * np.pi * fs * dr) * abs(rte)
        assert np.allclose(np.abs(H[:, k0:k1]), want, rtol=1e-12)
        mags.append(abs(rte))
    assert mags[0] != mags[-1]
