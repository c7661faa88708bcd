"""Oracle pins of cascaded edge diffraction (two diffractions in one segment between point sources).

Sec. III-B extends DRT to diffraction with the UTD of Kouyoumjian and Pathak.  For a diffraction whose
incident wave was itself diffracted by an earlier edge, the incident wavefront is astigmatic (one
caustic on the earlier edge, the other behind it), and the UTD prescribes both the spreading of the
new diffracted ray, sqrt(rho / (s (rho + s))) with rho the incident wavefront's radius of curvature in
the plane of the incident ray and the edge, and the distance parameter L of the transition function.
Two independent pins:

* continuity: as the receiver crosses the second edge's incident shadow boundary for the field
  diffracted by the first edge, the singly diffracted ray is blocked by the second wedge while the
  doubly diffracted ray's transition function jumps; their sum must stay continuous.  That holds only
  when both the spreading and L of the second diffraction follow the incident wavefront, for parallel
  and for skew edges, soft and hard polarisation.  (The first edge's coefficient enters the two rays
  with slightly different distance parameters, the receiver and the second edge being its observers;
  the geometry keeps that diffraction far from its own shadow boundaries, at 60 GHz, with the receiver
  0.1 m beyond the second edge, so this O(1 / (k L a)) difference stays near 1e-7 of the field.)
* closed form: for parallel edges and rays normal to them, the doubly diffracted amplitude of a point
  source is (lambda / 4 pi) |D_1| |D_2| / sqrt(s0 s1 s2 (s0 + s1 + s2)) (the spreading factors
  telescope), with L_1 = s0 s1 / (s0 + s1) and L_2 = s1 s2 / (s1 + s2).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

C0 = I.C0
FC = 60e9
K = 2 * math.pi * FC / C0


def _frame(kind):
    """World axes (u, v, w) of the 2D construction: w is the first edge's direction."""
    if kind == "vertical":          # edges along z: E (vertical) parallel to the edges -> soft
        return np.eye(3)
    if kind == "horizontal":        # edges along x, rays in the y-z plane: E normal to the edges -> hard
        return np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    # skew: a generic rotation of the whole construction; the second wedge is tilted further below
    R = I._rot_axis([0.3, -0.5, 0.8], 0.7)
    return R


def two_wedge_scene(kind, tilt=0.0, tx_w=0.0, rx_w=0.0, rx_u=10.1, rx_v0=-2.0, vrx=-0.05):
    """Two metal right-angled wedges in the frame (u, v, w) (columns of `_frame(kind)`):
    wedge A fills u <= 0, v <= 0 (edge 1 on the w axis), wedge B fills u <= 10, v <= -2 (edge 2 through
    (10, -2)), optionally rotated by `tilt` about the u axis through its edge.  TX at (-1, 10, tx_w);
    RX at (rx_u, rx_v0 + vrx t, rx_w).  In the plane w = 0 the second edge's incident shadow boundary
    for waves from edge 1 is the line v = -u / 5."""
    F = _frame(kind)
    u, v, w = F[:, 0], F[:, 1], F[:, 2]
    world = lambda p: p[0] * u + p[1] * v + p[2] * w
    b = I._Builder(f"two-wedges-{kind}")
    metal = b.material(1.0, 0.0, pec=True)
    b.edge(0, metal, world([0, 0, -20]), world([0, 0, 20]), v, u)                    # edge 1
    Rt = I._rot_axis(u, tilt)
    c2 = world([10, -2, 0])
    b.edge(0, metal, c2 + Rt @ (-20 * w), c2 + Rt @ (20 * w), Rt @ v, Rt @ u)        # edge 2
    tx = world([-1.0, 10.0, tx_w])
    rx = world([rx_u, rx_v0, rx_w])
    sc = b.build((tx, [0, 0, 0], [0, 0, 0]), (rx, vrx * v, [0, 0, 0]))
    ps = I.chains_to_pathset([[(I.T_D, 0)], [(I.T_D, 0), (I.T_D, 1)]])
    ps.s0[:, :2] = 20.0
    return sc, ps, F


def _edge_angle(sc, e, X, Q):
    """Angle of X about edge e at its point Q, from the 0-face towards the 0-face normal."""
    E = sc.edges[e]
    ed = (E["b"] - E["a"]) / np.linalg.norm(E["b"] - E["a"])
    x, y = np.cross(E["n0"], ed), E["n0"]
    r = X - Q
    r = r - ed * (r @ ed)
    return math.atan2(r @ y, r @ x) % (2 * math.pi)


def _lit_measure(sc, r):
    """phi - phi' - pi at edge 2 of the doubly diffracted path: negative where the singly diffracted ray
    passes the second wedge (lit), positive in its shadow, zero on the incident shadow boundary."""
    pts = r["pts"][0, 1]
    d1, d2 = pts[0], pts[1]
    rx = np.asarray(sc.rx["r"]) + np.asarray(sc.rx["v"]) * r["t"]
    return _edge_angle(sc, 1, rx, d2) - _edge_angle(sc, 1, d1, d2) - math.pi


def _run(sc, ps, t):
    r = O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), FC, points=True)
    r["t"] = t
    return r


@pytest.mark.parametrize("kind,tilt,tx_w,rx_w", [("vertical", 0.0, 0.0, 0.0), ("horizontal", 0.0, 0.0, 0.0),
                                                 ("skew", 0.35, 2.0, -0.03), ("skew", -0.5, -1.0, 0.04)])
def test_double_diffraction_continuous_across_second_shadow_boundary(kind, tilt, tx_w, rx_w):
    sc, ps, _ = two_wedge_scene(kind, tilt, tx_w, rx_w)
    lo, hi = 0.0, 0.8
    assert _lit_measure(sc, _run(sc, ps, lo)) < 0 < _lit_measure(sc, _run(sc, ps, hi))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _lit_measure(sc, _run(sc, ps, mid)) < 0:
            lo = mid
        else:
            hi = mid
    tc = 0.5 * (lo + hi)

    def parts(t):
        r = _run(sc, ps, t)
        assert (r["flags"][0] == 0).all()
        f = r["a"][0] * np.exp(-1j * K * r["tau"][0] * C0)
        lit = _lit_measure(sc, r) < 0
        return (f[0] if lit else 0.0), f[1], lit

    s_m, dd_m, lit_m = parts(tc - 1e-9)
    s_p, dd_p, lit_p = parts(tc + 1e-9)
    assert lit_m and not lit_p
    ref = abs(s_m)
    assert ref > 0
    # the doubly diffracted ray takes over exactly what the blocked singly diffracted ray carried
    assert abs((s_m + dd_m) - (s_p + dd_p)) < 1e-6 * ref
    # not vacuous: each part jumps by about half the incident field there
    assert abs(dd_m - dd_p) > 0.5 * ref


@pytest.mark.parametrize("kind", ["vertical", "horizontal"])
def test_double_diffraction_parallel_edges_closed_form(kind):
    sc, ps, _ = two_wedge_scene(kind, rx_u=14.0, rx_v0=-0.5, vrx=0.0)
    r = _run(sc, ps, 0.0)
    assert r["flags"][0, 1] == 0
    tx, rx = np.asarray(sc.tx["r"]), np.asarray(sc.rx["r"])
    d1, d2 = r["pts"][0, 1, 0], r["pts"][0, 1, 1]
    s0, s1, s2 = np.linalg.norm(d1 - tx), np.linalg.norm(d2 - d1), np.linalg.norm(rx - d2)
    # the rays lie in the plane w = 0, normal to both edges
    assert abs(r["tau"][0, 1] * C0 - (s0 + s1 + s2)) < 1e-9
    pol = 0 if kind == "vertical" else 1          # soft (E along the edges) or hard coefficient
    D1 = O.utd(1.5, _edge_angle(sc, 0, d2, d1), _edge_angle(sc, 0, tx, d1), 1.0, s0 * s1 / (s0 + s1), K)[pol]
    D2 = O.utd(1.5, _edge_angle(sc, 1, rx, d2), _edge_angle(sc, 1, d1, d2), 1.0, s1 * s2 / (s1 + s2), K)[pol]
    lam = C0 / FC
    ref = lam / (4 * math.pi) * abs(D1) * abs(D2) / math.sqrt(s0 * s1 * s2 * (s0 + s1 + s2))
    assert abs(abs(r["a"][0, 1]) - ref) < 1e-12 * ref


def test_double_diffraction_crossed_edges_closed_form():
    """Edge 2 perpendicular to edge 1 and to the ray between them: the incident wavefront's radius in
    the plane of the ray and edge 2 is the one whose caustic lies on edge 1, rho_e = s1, so the amplitude
    is (lambda / 4 pi) |D_s1| |D_h2| (1 / s0) sqrt(s0 / (s1 (s0 + s1))) sqrt(s1 / (s2 (s1 + s2))) with
    L_1 = s0 s1 / (s0 + s1) and L_2 = s2 (s0 + s1) / (s0 + s1 + s2).  With the parallel case this pins
    rho_e at both ends of its range (rho1 and rho2 of the incident wavefront).  Vertical polarisation
    along edge 1 is the soft case there and the hard case at the horizontal edge 2."""
    b = I._Builder("crossed-wedges")
    metal = b.material(1.0, 0.0, pec=True)
    z = np.array([0.0, 0.0, 1.0])
    b.edge(0, metal, [0, 0, -20], [0, 0, 20], [0, 1, 0], [1, 0, 0])            # edge 1 along z
    c2 = np.array([10.0, -2.0, 0.0])
    rh = c2 / np.linalg.norm(c2)                                                # ray direction edge 1 -> 2
    e2 = np.cross(z, rh)
    c45 = math.sqrt(0.5)
    # wedge B below edge 2 in the (rh, z) plane, faces at -45 and -135 degrees from rh
    b.edge(0, metal, c2 - 20 * e2, c2 + 20 * e2, c45 * rh + c45 * z, -c45 * rh + c45 * z)
    tx = np.array([-1.0, 10.0, 0.0])
    s2_ = 5.0
    rx = c2 + s2_ * (math.cos(math.radians(30)) * rh + math.sin(math.radians(30)) * z)
    sc = b.build((tx, [0, 0, 0], [0, 0, 0]), (rx, [0, 0, 0], [0, 0, 0]))
    ps = I.chains_to_pathset([[(I.T_D, 0), (I.T_D, 1)]])
    ps.s0[0, :2] = 20.0
    r = _run(sc, ps, 0.0)
    assert r["flags"][0, 0] == 0
    d1, d2 = r["pts"][0, 0, 0], r["pts"][0, 0, 1]
    assert np.abs(d1).max() < 1e-9 and np.abs(d2 - c2).max() < 1e-9
    s0, s1, s2 = np.linalg.norm(d1 - tx), np.linalg.norm(d2 - d1), s2_
    D1 = O.utd(1.5, _edge_angle(sc, 0, d2, d1), _edge_angle(sc, 0, tx, d1), 1.0, s0 * s1 / (s0 + s1), K)[0]
    L2 = s2 * (s0 + s1) / (s0 + s1 + s2)
    D2 = O.utd(1.5, _edge_angle(sc, 1, rx, d2), _edge_angle(sc, 1, d1, d2), 1.0, L2, K)[1]
    lam = C0 / FC
    spread = (1 / s0) * math.sqrt(s0 / (s1 * (s0 + s1))) * math.sqrt(s1 / (s2 * (s1 + s2)))
    ref = lam / (4 * math.pi) * abs(D1) * abs(D2) * spread
    assert abs(abs(r["a"][0, 0]) - ref) < 1e-12 * ref
