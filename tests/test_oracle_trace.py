"""Pins of the oracle's conventional ray tracing at an instant (the run DRT starts from, Sec. II, and
re-runs at every multipath-lifetime boundary, Sec. IV-B): brute-force image-tree enumeration with
validity and occlusion tests.

* In a rectangular (shoebox) room the image sources form a lattice, one image per lattice point, all
  visible from every interior receiver (the property the image method for rectangular rooms relies
  on).  Up to two reflections there are 1 + 6 + 18 lattice points: two per axis of order two (the
  ordered pairs of opposite walls) and four per pair of axes (reflections on perpendicular walls
  commute, so of the two orderings of each pair of adjacent walls exactly one is a ray).  The tracer
  must return exactly those 25 chains, each of the length |RX - lattice image|, wherever TX and RX
  stand inside.
* A rectangular screen between TX and RX blocks the line of sight exactly while the straight segment
  crosses the screen's rectangle; with the screen in the plane x = 0 and the terminals at x = -5 and
  x = +5, the crossing point is the midpoint, so the line of sight reopens when the receiver's lateral
  offset passes twice the screen's half-width.
* Every chain the tracer returns is valid for the DRT extrapolation at the same instant (flags 0) and
  its diffraction parameters give the extrapolation's points.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I


def shoebox(tx, rx, dims=(10.0, 7.0, 3.0)):
    """Six walls with inward normals: the room [0, a] x [0, b] x [0, c]."""
    a, b, c = dims
    B = I._Builder("shoebox")
    m = B.material(4.0, 0.02)
    B.face(0, m, [0, b / 2, c / 2], [1, 0, 0], [0, 1, 0], b / 2, c / 2)
    B.face(0, m, [a, b / 2, c / 2], [-1, 0, 0], [0, 1, 0], b / 2, c / 2)
    B.face(0, m, [a / 2, 0, c / 2], [0, 1, 0], [1, 0, 0], a / 2, c / 2)
    B.face(0, m, [a / 2, b, c / 2], [0, -1, 0], [1, 0, 0], a / 2, c / 2)
    B.face(0, m, [a / 2, b / 2, 0], [0, 0, 1], [1, 0, 0], a / 2, b / 2)
    B.face(0, m, [a / 2, b / 2, c], [0, 0, -1], [1, 0, 0], a / 2, b / 2)
    return B.build((tx, [0, 0, 0], [0, 0, 0]), (rx, [0, 0, 0], [0, 0, 0]))


def test_shoebox_room_every_image_source_of_order_two_is_visible():
    rng = np.random.default_rng(3)
    for _ in range(6):
        tx = rng.uniform([0.5, 0.5, 0.3], [9.5, 6.5, 2.7])
        rx = rng.uniform([0.5, 0.5, 0.3], [9.5, 6.5, 2.7])
        r = O.trace(shoebox(tx, rx), 0.0, 2, with_tiles=False)
        assert r["candidates"] == 1 + 6 + 36
        assert r["paths"].n_paths == 1 + 6 + 18
        assert len(r["ambiguous"]) == 0
        pairs = {tuple(r["paths"].prims[p, :2]) for p in range(r["paths"].n_paths) if r["paths"].n_int[p] == 2}
        for a in range(6):
            for b in range(a + 1, 6):
                if a // 2 == b // 2:             # opposite walls: both orderings
                    assert (a, b) in pairs and (b, a) in pairs
                else:                            # perpendicular walls: exactly one ordering
                    assert ((a, b) in pairs) != ((b, a) in pairs)
        # each returned chain is the image-method ray: its length is |RX - image of TX|
        rec = O.extrapolate(shoebox(tx, rx), r["paths"], I.TimeGrid(0, 1, 1), 3e9, points=True)
        assert (rec["flags"] == 0).all()
        for p in range(r["paths"].n_paths):
            img = np.array(tx, float)
            for w in r["paths"].prims[p, :r["paths"].n_int[p]]:
                axis, val = [(0, 0.0), (0, 10.0), (1, 0.0), (1, 7.0), (2, 0.0), (2, 3.0)][w]
                img[axis] = 2 * val - img[axis]
            d = np.linalg.norm(np.asarray(rx) - img)
            assert abs(rec["tau"][0, p] * I.C0 - d) < 1e-9


def screen_scene(rx_y):
    B = I._Builder("screen")
    m = B.material(5.0, 0.05)
    B.face(0, m, [0, 0, 1.75], [1, 0, 0], [0, 1, 0], 1.0, 1.25)     # x = 0, |y| <= 1, 0.5 <= z <= 3
    return B.build(([-5, 0, 1.5], [0, 0, 0], [0, 0, 0]), ([5, rx_y, 1.5], [0, 0, 0], [0, 0, 0]))


def has_los(r):
    return any(int(r["paths"].n_int[p]) == 0 for p in range(r["paths"].n_paths))


def test_screen_blocks_line_of_sight_until_the_closed_form_offset():
    assert not has_los(O.trace(screen_scene(0.0), 0.0, 1, with_tiles=False))
    assert has_los(O.trace(screen_scene(4.0), 0.0, 1, with_tiles=False))
    lo, hi = 0.0, 4.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if has_los(O.trace(screen_scene(mid), 0.0, 1, with_tiles=False)):
            hi = mid
        else:
            lo = mid
    assert abs(0.5 * (lo + hi) - 2.0) < 1e-9          # crossing at y = rx_y / 2 = the half-width 1
    # the screen's own reflection needs both terminals on its front side: never a ray here
    r = O.trace(screen_scene(4.0), 0.0, 1, with_tiles=False)
    assert all(not (r["paths"].n_int[p] == 1 and r["paths"].types[p, 0] == I.T_R) for p in range(r["paths"].n_paths))


@pytest.mark.parametrize("which", ["tiny", "canyon"])
def test_traced_chains_are_valid_rays_for_the_extrapolation(which):
    if which == "tiny":
        sc, t, fc, tiles = I.scene_tiny(0), 0.3, 28e9, False
    else:
        sc, t, fc, tiles = I.scene_canyon(0), 0.4, 60e9, True
    r = O.trace(sc, t, 2, with_tiles=tiles)
    ps = r["paths"]
    assert ps.n_paths > 3
    rec = O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), fc, points=True, n_threads=8)
    assert (rec["flags"][0] == 0).all()
    # the diffraction parameters returned by the tracer reproduce the extrapolation's points
    for p in range(ps.n_paths):
        for j in range(int(ps.n_int[p])):
            if ps.types[p, j] == I.T_D:
                E = sc.edges[ps.prims[p, j]]
                e = (E["b"] - E["a"]) / np.linalg.norm(E["b"] - E["a"])
                q = rec["pts"][0, p, j]
                body = sc.bodies[E["body"]]
                if np.allclose(body["v"], 0) and np.allclose(body["a"], 0) and body["w0"] == 0:
                    assert abs((q - E["a"]) @ e - ps.s0[p, j]) < 1e-9
