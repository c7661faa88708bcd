"""Conventional ray tracing at an instant on the GPU (drt_trace_paths) and DRT with a ray-tracing run at
every window start (drt_synthesize_H_retraced), against the oracle.

The GPU's rays at an instant must be the oracle's rays, except candidates whose decision margin
(validity or occlusion) is below 1e-9 m, which either side may decide either way; their diffraction
parameters must agree to 1e-8 m.  The re-traced H must equal the oracle's extrapolation and synthesis
of the same windows' chains (the GPU's own ray sets, checked against the oracle above) within the
H bars of the form.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_gpu_parity import compare_H, compare_H_band

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


def chain_key(ps, p):
    n = int(ps.n_int[p])
    return tuple(zip(ps.types[p, :n].tolist(), ps.prims[p, :n].tolist()))


def compare_rays(gps, scene, t, max_order, with_tiles):
    r = O.trace(scene, t, max_order, with_tiles=with_tiles)
    want = {chain_key(r["paths"], p): p for p in range(r["paths"].n_paths)}
    amb = set()
    for k in r["ambiguous"]:
        ch = O.trace_chain(scene, int(k), with_tiles)
        if ch is not None:
            amb.add(tuple(ch))
    got = {chain_key(gps, p): p for p in range(gps.n_paths)}
    sure = {k for k, p in want.items() if r["margin"][p] >= 1e-9}
    assert sure <= set(got), sorted(sure - set(got))[:5]
    assert set(got) <= set(want) | amb, sorted(set(got) - set(want) - amb)[:5]
    for k in set(got) & set(want):
        pg, pw = got[k], want[k]
        for j in range(len(k)):
            if k[j][0] == I.T_D:
                assert abs(gps.s0[pg, j] - r["paths"].s0[pw, j]) < 1e-8
    return len(got), len(want)


@pytest.mark.parametrize("which,t", [("tiny", 0.0), ("tiny", 0.6), ("canyon", 0.0), ("canyon", 0.4),
                                     ("link", 1.3)])
def test_traced_rays_match_the_oracle(ctx, which, t):
    if which == "tiny":
        sc, tiles = I.scene_tiny(0), False
        ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed0.npz"))
    elif which == "canyon":
        sc, tiles = I.scene_canyon(0), True
        ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))
    else:
        sc, tiles = I.scene_link(2), True
        ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_link_seed2.npz"))
    link = ctx.load(sc, ps)
    gps = link.trace_paths(t, 2, with_tiles=tiles)
    n_got, n_want = compare_rays(gps, sc, t, 2, tiles)
    assert n_got > 3
    link.unload()


def test_shoebox_room_lattice_on_the_gpu(ctx):
    from test_oracle_trace import shoebox
    sc = shoebox([2.0, 3.0, 1.2], [7.5, 1.7, 2.05])
    link = ctx.load(sc, I.chains_to_pathset([[]]))
    gps = link.trace_paths(0.0, 2, with_tiles=False)
    assert gps.n_paths == 1 + 6 + 18
    compare_rays(gps, sc, 0.0, 2, False)
    link.unload()


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_retraced_windows_match_the_oracle(ctx, form):
    """Tiny 28 GHz case over 1000 x 1 ms in three windows with reflections and diffractions up to order
    two; the canyon over 600 x 0.5 ms in three windows with tiles."""
    from paper_2205_00237_gb300 import drt
    prec = drt.FP64 if form == "fp64" else drt.FP32_BULK
    for sc, ps, tg, fg, tiles, starts in (
            (I.scene_tiny(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed0.npz")),
             I.TimeGrid(0.0, 1e-3, 1000), I.FreqGrid(28e9, 400e6, 256), False, [0, 300, 700]),
            (I.scene_canyon(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz")),
             I.TimeGrid(0.0, 0.5e-3, 600), I.FreqGrid(60e9, 1e9, 512), True, [0, 250, 400])):
        link = ctx.load(sc, ps)
        H = link.synthesize_H_retraced(tg, fg, starts, 2, with_tiles=tiles, precision=prec).cpu().numpy()
        sets = [link.trace_paths(tg.t_start + k * tg.dt, 2, with_tiles=tiles) for k in starts]
        Href = O.synthesize_H_retraced(sc, tg, fg, starts, lambda w: sets[w], n_threads=8)
        if form == "fp64":
            compare_H(H, Href)
        else:
            rows = []
            bounds = starts + [tg.n_steps]
            for w in range(len(starts)):
                sub = I.TimeGrid(tg.t_start + bounds[w] * tg.dt, tg.dt, bounds[w + 1] - bounds[w])
                rows.append((bounds[w], bounds[w + 1], O.extrapolate(sc, sets[w], sub, fg.fc, n_threads=8)))
            for k0, k1, r in rows:
                compare_H_band(H[k0:k1], r, fg)
        link.unload()
