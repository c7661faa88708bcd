"""Pins of the oracle's multipath-lifetime (T_C) management: expiry criterion, window planner and
windowed H (Sec. II multipath lifetime, Sec. IV-B segmentation into T_C windows).

Worked case, solved by hand: a PEC wall on the plane y = 10 spanning x in [-20, 20]; TX fixed at
(-60, 0, 2), RX at (-41 + 20 t, 0, 2).  Both terminals are 10 m in front of the wall, so the
reflection point is their midpoint, x_Q = -50.5 + 10 t: it enters the wall at t = 3.05 s and leaves
it at t = 7.05 s.  With 7 ms steps that makes step 436 the first valid instant of the reflection and
1008 the first invalid one.  LoS length d_L = 19 + 20 t, reflected length d_R = sqrt(d_L^2 + 20^2);
the vertical polarisation is TE on the vertical wall, so |a| = lambda / (4 pi d) on both paths
(Friis, |Gamma| = 1) and the reflection's share of the power is d_L^2 / (d_L^2 + d_R^2) ~ 0.49.
"""
import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_oracle_pins import wall_scene

C0 = I.C0
FC = 5.9e9
DT, T = 7e-3, 1200
N_IN, N_OUT = 436, 1008


@pytest.fixture(scope="module")
def run():
    sc = wall_scene([-60, 0, 2], [-41, 0, 2], vrx=(20.0, 0, 0), pec=True)
    ps = I.chains_to_pathset([[], [(I.T_R, 0)]])
    tg = I.TimeGrid(0.0, DT, T)
    return O.extrapolate(sc, ps, tg, FC), tg


def hand_power(n):
    t = n * DT
    lam = C0 / FC
    dl = 19 + 20 * t
    dr = np.hypot(dl, 20.0)
    return (lam / (4 * np.pi * dl)) ** 2, (lam / (4 * np.pi * dr)) ** 2


def test_reflection_enters_and_leaves_the_wall_on_the_hand_steps(run):
    r, _ = run
    n = np.arange(T)
    assert (r["flags"][:, 0] == 0).all()
    assert (r["flags"][(n >= N_IN) & (n < N_OUT), 1] == 0).all()
    assert (r["flags"][(n < N_IN) | (n >= N_OUT), 1] & O.F_FACE).all()
    pl, pr = hand_power(n[N_IN:N_OUT])
    assert np.allclose(np.abs(r["a"][N_IN:N_OUT, 0]) ** 2, pl, rtol=1e-9)
    assert np.allclose(np.abs(r["a"][N_IN:N_OUT, 1]) ** 2, pr, rtol=1e-9)


def test_major_changes_are_the_hand_steps(run):
    r, _ = run
    major = O.lifetime_toggles(r, 0.1)
    assert list(np.flatnonzero(major)) == [N_IN, N_OUT]
    # a share above the reflection's (~0.49) makes neither change major
    assert not O.lifetime_toggles(r, 0.6).any()


def test_share_is_taken_at_the_valid_instant(run):
    """Appearance: the share is the reflection's at step 436 (where it is valid); disappearance: at
    step 1007.  Thresholds just below and above the hand shares switch each change on and off."""
    r, _ = run
    for n_valid, n_change in ((N_IN, N_IN), (N_OUT - 1, N_OUT)):
        pl, pr = hand_power(n_valid)
        share = pr / (pl + pr)
        assert O.lifetime_toggles(r, share * (1 - 1e-7))[n_change]
        assert not O.lifetime_toggles(r, share * (1 + 1e-7))[n_change]


def test_window_planner(run):
    r, _ = run
    major = O.lifetime_toggles(r, 0.1)
    assert O.plan_windows(major, 1, 10000) == [0, N_IN, N_OUT]
    assert O.plan_windows(major, 1, 400) == [0, 400, N_IN, N_IN + 400, N_OUT]
    assert O.plan_windows(major, 500, 2000) == [0, N_OUT]
    assert O.plan_windows(np.zeros(T, bool), 1, 400) == [0, 400, 800]
    assert O.plan_windows(np.zeros(T, bool), 1, T) == [0]
    assert O.plan_windows(np.ones(T, bool), 1, 1) == list(range(T))
    last = np.zeros(T, bool)
    last[T - 1] = True                  # a change at the last instant opens a one-step window
    assert O.plan_windows(last, 1, 10000) == [0, T - 1]
    assert O.plan_windows(last, T, 10000) == [0]


def los_only_rows(H, rows, fg):
    """LoS alone: |H| = lambda / (4 pi d_L) in every bin, phase step exp(-j 2 pi df d_L / c)."""
    lam = C0 / FC
    df = fg.bandwidth / fg.n_bins
    for n in rows:
        dl = 19 + 20 * n * DT
        assert np.allclose(np.abs(H[n]), lam / (4 * np.pi * dl), rtol=1e-9)
        ratio = H[n, 1:] / H[n, :-1]
        assert np.allclose(ratio, np.exp(-2j * np.pi * df * dl / C0), rtol=1e-9, atol=0)


def test_windowed_H(run):
    r, _ = run
    fg = I.FreqGrid(FC, 100e6, 64)
    Hfull = O.synthesize_H(r, fg)
    n = np.arange(T)
    # windows at the major changes: the reflection is tracked exactly while it exists
    H = O.synthesize_H_windows(r, [0, N_IN, N_OUT], fg)
    los_only_rows(H, n[(n < N_IN) | (n >= N_OUT)][::37], fg)
    assert np.allclose(H[N_IN:N_OUT], Hfull[N_IN:N_OUT], rtol=1e-12, atol=0)
    # one window from t = 0: the reflection is not in its chain set, so it is never seen
    H0 = O.synthesize_H_windows(r, [0], fg)
    los_only_rows(H0, n[::29], fg)
    # a window boundary after the reflection appears: missed until step 500
    H5 = O.synthesize_H_windows(r, [0, 500], fg)
    los_only_rows(H5, np.r_[n[N_IN:500:9], n[N_OUT::23]], fg)
    assert np.allclose(H5[500:N_OUT], Hfull[500:N_OUT], rtol=1e-12, atol=0)
    assert np.abs(H5[N_IN:500] - Hfull[N_IN:500]).min() > 0
    # a window at every instant is the per-instant method
    Hall = O.synthesize_H_windows(r, list(range(T)), fg)
    assert np.allclose(Hall, Hfull, rtol=1e-12, atol=0)
