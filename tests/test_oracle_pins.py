"""Pins of the FP64 oracle against facts the paper and the mathematics fix (CPU only, no GPU).

Each test pins the oracle to something other than itself: closed forms, the reflection law and the
Keller cone, brute-force minimisation, finite differences, the paper's own validation (DRT against a
snapshot re-solve, Sec. IV-A.2), reciprocity, textbook limits of the Fresnel and UTD coefficients,
scipy's Fresnel integrals, continuity of GO + diffracted field across shadow boundaries, closed-form
hemispheric integrals of the ER lobe, and properties of H(t, f).
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2205_00237_gb300 import inputs as I

C0 = I.C0
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def canyon():
    return I.scene_canyon(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))


def posed_rotation(body, t):
    th = body["w0"] * t + 0.5 * body["wdot"] * t * t
    return Rotation.from_rotvec(np.asarray(body["k"]) * th).as_matrix()


def posed_origin(body, t):
    return np.asarray(body["o"]) + np.asarray(body["v"]) * t + 0.5 * np.asarray(body["a"]) * t * t


def posed(body, p0, t):
    return posed_origin(body, t) + posed_rotation(body, t) @ (np.asarray(p0) - np.asarray(body["o"]))


def wall_scene(tx, rx, vtx=(0, 0, 0), vrx=(0, 0, 0), body_kin=None, pec=False):
    """One rectangular wall on the plane y = 10 (normal -y, 40 m x 20 m) and its edges."""
    b = I._Builder("wall")
    mat = b.material(1.0, 0.0, pec=True) if pec else b.material(4.0, 0.02)
    body = 0
    if body_kin is not None:
        body = b.body(**body_kin)
    b.face(body, mat, [0, 10, 5], [0, -1, 0], [1, 0, 0], 20.0, 10.0)
    b.edge(body, mat, [20, 10, 0], [20, 10, 10], [0, -1, 0], [1, 0, 0])   # vertical corner at x = 20
    return b.build((tx, vtx, [0, 0, 0]), (rx, vrx, [0, 0, 0]))


# ------------------------------------------------------------------------------------------------
# reflection geometry
# ------------------------------------------------------------------------------------------------
def test_single_reflection_closed_form_and_brute_force():
    """Eq. ref_point: the path length equals |RX - image(TX)| and the point minimises the length."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        tx = [rng.uniform(-15, 15), rng.uniform(-5, 8), rng.uniform(0.5, 8)]
        rx = [rng.uniform(-15, 15), rng.uniform(-5, 8), rng.uniform(0.5, 8)]
        sc = wall_scene(tx, rx)
        ps = I.chains_to_pathset([[(I.T_R, 0)]])
        r = O.extrapolate(sc, ps, I.TimeGrid(0, 1, 1), 3e9, points=True)
        img = np.array([tx[0], 20.0 - tx[1], tx[2]])
        d_img = np.linalg.norm(np.array(rx) - img)
        assert abs(r["tau"][0, 0] * C0 - d_img) < 1e-12 * d_img
        q = r["pts"][0, 0, 0]
        assert abs(q[1] - 10.0) < 1e-12
        # brute-force: dense grid then local refinement of |TX-Q| + |Q-RX| over the plane y = 10
        f = lambda x, z: (np.hypot(np.hypot(x - tx[0], 10 - tx[1]), z - tx[2])
                          + np.hypot(np.hypot(x - rx[0], 10 - rx[1]), z - rx[2]))
        xs, zs = np.meshgrid(np.linspace(-40, 40, 801), np.linspace(-20, 30, 501))
        k = np.argmin(f(xs, zs))
        x0, z0 = xs.flat[k], zs.flat[k]
        for h in (0.1, 0.01, 1e-3, 1e-4, 1e-5, 1e-6):
            g = np.linspace(-10, 10, 21) * h
            X, Z = np.meshgrid(x0 + g, z0 + g)
            k = np.argmin(f(X, Z))
            x0, z0 = X.flat[k], Z.flat[k]
        assert abs(q[0] - x0) < 1e-5 and abs(q[2] - z0) < 1e-5


def test_reflection_law_and_keller_cone_on_canyon():
    """All reflection points obey the reflection law and coplanarity; all diffraction points lie on
    the Keller cone (equal angles with the edge), to 1e-12, at several instants."""
    sc, ps = canyon()
    for t in (0.0, 0.37, 0.81):
        r = O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), 60e9, points=True, n_threads=4)
        tx = np.asarray(sc.tx["r"]) + np.asarray(sc.tx["v"]) * t + 0.5 * np.asarray(sc.tx["a"]) * t * t
        rx = np.asarray(sc.rx["r"]) + np.asarray(sc.rx["v"]) * t + 0.5 * np.asarray(sc.rx["a"]) * t * t
        n_checked = 0
        for p in range(ps.n_paths):
            n = int(ps.n_int[p])
            if r["flags"][0, p] & (O.F_DEGEN | O.F_SIDE | O.F_NOCONV):
                continue                  # the laws hold for rays on the correct sides only
            V = [tx] + [r["pts"][0, p, j] for j in range(n)] + [rx]
            for j in range(n):
                kin = V[j + 1] - V[j]
                kin /= np.linalg.norm(kin)
                kout = V[j + 2] - V[j + 1]
                kout /= np.linalg.norm(kout)
                ty, pr = ps.types[p, j], ps.prims[p, j]
                if ty == I.T_R:
                    f = sc.faces[pr]
                    nv = posed_rotation(sc.bodies[f["body"]], t) @ f["n"]
                    assert abs(np.dot(nv, kin) + np.dot(nv, kout)) < 1e-12
                    assert abs(np.dot(np.cross(kin, nv), kout)) < 1e-12
                    n_checked += 1
                elif ty == I.T_D:
                    e = sc.edges[pr]
                    ev = posed_rotation(sc.bodies[e["body"]], t) @ ((e["b"] - e["a"]) / np.linalg.norm(e["b"] - e["a"]))
                    assert abs(np.dot(kin, ev) - np.dot(kout, ev)) < 1e-12
                    # and the point is on the (moving) edge line
                    a = posed(sc.bodies[e["body"]], e["a"], t)
                    w = V[j + 1] - a
                    assert np.linalg.norm(w - np.dot(w, ev) * ev) < 1e-9
                    n_checked += 1
        assert n_checked > 500


def test_tiny_scene_exit_time_worked_example():
    """Tiny scene, seed 0: ground-then-rear-face reflection.  By hand (images in the ground and in the
    rear plane x = x_f(t) = 71 + 15 t, RX at x_R(t) = 50 + 10 t), the point's height on the face is
    z = -5 + 6.5 x_f / (2 x_f - x_R); it leaves the bottom of the face (z < 0) when
    x_f / (2 x_f - x_R) = 5 / 6.5, i.e. at t* = (5/6.5 * 92 - 71) / (15 - 5/6.5 * 20)."""
    sc = I.scene_tiny(0)
    ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed0.npz"))
    j = [p for p in range(ps.n_paths) if ps.n_int[p] == 2][0]
    lam = 5 / 6.5
    t_star = (lam * 92 - 71) / (15 - lam * 20)
    r = O.extrapolate(sc, ps, I.TimeGrid(0, 1e-3, 1000), 28e9, points=True)
    n_star = t_star / 1e-3                       # = 600 up to rounding: the exit falls on a step
    steps = np.arange(1000)
    assert (r["flags"][steps < n_star - 1e-6, j] == 0).all()
    assert (r["flags"][steps > n_star + 1e-6, j] & O.F_FACE).all()
    on = np.abs(steps - n_star) < 1e-6
    assert (r["margin"][on, j] < 1e-9).all()      # the step on the boundary is a boundary case
    # height of the point on the face before exit matches the hand formula
    for n in (0, 250, 500):
        t = n * 1e-3
        xf, xr = 71 + 15 * t, 50 + 10 * t
        z = -5 + 6.5 * xf / (2 * xf - xr)
        assert abs(r["pts"][n, j, 1, 2] - z) < 1e-12


# ------------------------------------------------------------------------------------------------
# the paper's own validation: DRT equals a snapshot re-solve (Sec. IV-A.2, "virtually zero" error)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["tiny0", "tiny1", "canyon"])
def test_drt_equals_snapshot_resolve(which):
    if which.startswith("tiny"):
        seed = int(which[-1])
        sc = I.scene_tiny(seed)
        ps = I.chains_tiny(sc)            # all 50 candidates, valid or not
        tg, fc = I.TimeGrid(0.0, 0.05, 20), 28e9
    else:
        sc, ps = canyon()
        tg, fc = I.TimeGrid(0.0, 0.05, 20), 60e9
    a = O.extrapolate(sc, ps, tg, fc, O.METHOD_DRT, n_threads=8, points=True, velocities=True)
    b = O.extrapolate(sc, ps, tg, fc, O.METHOD_RESOLVE, n_threads=8, points=True, velocities=True)
    # Where a ray has a neighbour on the wrong side of a wall or wedge (side flag), the image
    # construction is no longer a stationary path and the two solvers legitimately differ; impossible
    # candidates can also end on a kink where two vertices meet (degenerate flag).
    ok = ((a["flags"] | b["flags"]) & (O.F_DEGEN | O.F_NOCONV | O.F_SIDE)) == 0
    assert ok.sum() > (60 if which.startswith("tiny") else 0.9 * ok.size)
    rel = np.abs(a["tau"] - b["tau"]) / b["tau"]
    assert rel[ok].max() < 1e-12
    dp = np.abs(a["pts"] - b["pts"])[ok]
    assert np.nanmax(dp) < 1e-8
    # 5-point finite differences of the re-solve (h = 1 ms) truncate at ~1e-5 of the point's own
    # speed where a diffraction point slides fast (hundreds of m/s near grazing)
    dv = np.abs(a["vel"] - b["vel"])[ok]
    vmag = np.maximum(1.0, np.abs(b["vel"]))[ok]
    assert np.nanmax(dv / vmag) < 1e-5
    far = ok & (np.minimum(a["margin"], b["margin"]) > 1e-9)
    assert np.array_equal(a["flags"][far], b["flags"][far])
    va = ok & (a["flags"] == 0)
    assert (np.abs(a["a"] - b["a"])[va] <= 1e-8 * np.abs(b["a"])[va]).all()
    assert np.abs(a["fd"] - b["fd"])[va].max() < 1e-3


# ------------------------------------------------------------------------------------------------
# Doppler (App. A)
# ------------------------------------------------------------------------------------------------
def test_doppler_los_closed_form():
    """LoS: f' = f0 (c - v_RX.k)/(c - v_TX.k) exactly; head-on to first order f0 (v_T + v_R)/c."""
    fc = 5.9e9
    vt, vr = np.array([13.9, 0, 0]), np.array([-10.0, 0, 0])
    sc = wall_scene([0, 0, 1.75], [200, 0, 1.75], vt, vr)
    ps = I.chains_to_pathset([[]])
    r = O.extrapolate(sc, ps, I.TimeGrid(0, 1, 1), fc)
    k = np.array([1.0, 0, 0])
    exact = fc * ((C0 - vr @ k) / (C0 - vt @ k) - 1)
    assert abs(r["fd"][0, 0] - exact) < 1e-6
    assert abs(r["fd"][0, 0] - fc * (13.9 + 10.0) / C0) < 1e-3 * fc * 23.9 / C0


def test_doppler_equals_minus_path_length_rate():
    """For every canyon path, f_D = -(f0/c) dd/dt to O((v/c)^2): the rate of the re-solved length by a
    Richardson-extrapolated central difference."""
    sc, ps = canyon()
    fc, t = 60e9, 0.3
    d = {}
    for h in (1e-3, 5e-4):
        for s in (-1, 1):
            r = O.extrapolate(sc, ps, I.TimeGrid(t + s * h, 1, 1), fc, O.METHOD_RESOLVE, n_threads=8)
            d[(h, s)] = r["tau"][0] * C0
    rate = lambda h: (d[(h, 1)] - d[(h, -1)]) / (2 * h)
    ddt = (4 * rate(5e-4) - rate(1e-3)) / 3
    r = O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), fc, n_threads=8)
    ok = (r["flags"][0] & (O.F_DEGEN | O.F_NOCONV | O.F_SIDE)) == 0
    assert ok.sum() > 400
    err = np.abs(r["fd"][0] + fc / C0 * ddt)[ok]
    assert err.max() < 2e-2                      # f0 (v/c)^2 ~ 1e-3 Hz plus the difference error
    assert np.abs(r["fd"][0][ok]).max() > 1000   # the check is not vacuous


def test_doppler_sign_flip_when_terminals_pass():
    """LoS Doppler changes sign when TX and RX pass each other (Sec. IV-A.1)."""
    sc = wall_scene([0, -3, 1.75], [40, 3, 1.75], [13.9, 0, 0], [-10.0, 0, 0])
    ps = I.chains_to_pathset([[]])
    r = O.extrapolate(sc, ps, I.TimeGrid(0, 0.1, 40), 3e9)
    fd = r["fd"][:, 0]
    assert fd[0] > 0 and fd[-1] < 0
    t_pass = 40 / 23.9
    k = int(np.argmax(fd < 0))
    assert abs(k * 0.1 - t_pass) <= 0.1


def test_rotating_reflector_changes_doppler():
    """A reflector that starts rotating turns a near-zero reflection Doppler into a non-zero one
    (Sec. IV-A.3)."""
    kin_still = dict(o=[20, 10, 5], v=[0, 0, 0], a=[0, 0, 0], k=[0, 0, 1], w0=0.0, wdot=0.0)
    kin_rot = dict(kin_still, w0=math.pi / 6)
    ps = I.chains_to_pathset([[(I.T_R, 0)]])
    res = []
    for kin in (kin_still, kin_rot):
        sc = wall_scene([-5, 0, 1.75], [5, 0, 1.75], [7.8, 0, 0], [8.3, 0, 0], body_kin=kin)
        res.append(O.extrapolate(sc, ps, I.TimeGrid(0, 1, 1), 3e9)["fd"][0, 0])
    assert abs(res[0]) < 0.05 * abs(res[1])
    assert abs(res[1]) > 50.0


# ------------------------------------------------------------------------------------------------
# kinematics and frames (Eqs. Taylor, RigidBodyMotion, coordinate_transf, relative_vel/acc)
# ------------------------------------------------------------------------------------------------
def test_rigid_body_point_velocity_and_acceleration():
    rng = np.random.default_rng(3)
    body = np.zeros((), I.BODY)
    body["o"] = rng.normal(size=3)
    body["v"] = rng.normal(size=3) * 10
    body["a"] = rng.normal(size=3)
    k = rng.normal(size=3)
    body["k"] = k / np.linalg.norm(k)
    body["w0"], body["wdot"] = 0.7, -0.3
    p0 = rng.normal(size=3) * 3
    t, h = 0.8, 1e-4
    s = O.body_point(body, p0, t)
    pos = lambda tt: O.body_point(body, p0, tt)[0]
    v_fd = (pos(t - 2 * h) - 8 * pos(t - h) + 8 * pos(t + h) - pos(t + 2 * h)) / (12 * h)
    a_fd = (-pos(t - 2 * h) + 16 * pos(t - h) - 30 * pos(t) + 16 * pos(t + h) - pos(t + 2 * h)) / (12 * h * h)
    assert np.abs(s[1] - v_fd).max() < 1e-8
    assert np.abs(s[2] - a_fd).max() < 1e-4
    assert np.abs(s[0] - posed(body, p0, t)).max() < 1e-12


def test_relative_motion_round_trip_and_local_derivatives():
    """to_local then from_local is the identity; the local velocity/acceleration of Eqs.
    relative_vel/relative_acc are the time derivatives of the local coordinates (a missing Euler,
    Coriolis or centrifugal term fails the second check)."""
    kin = dict(o=[1, 12, 5], v=[3, -1, 0.5], a=[0.2, 0.1, -0.3], k=[0.3, 0.2, 0.93], w0=0.8, wdot=0.4)
    sc = wall_scene([0, 0, 1], [5, 0, 1], body_kin=kin)
    x0, v0, a0 = np.array([2.0, 1, 3]), np.array([10.0, -3, 1]), np.array([1.0, 2, -1])
    state = lambda tt: np.concatenate([x0 + v0 * tt + 0.5 * a0 * tt * tt, v0 + a0 * tt, a0])
    t, h = 0.6, 1e-4
    loc, back = O.frame_roundtrip(sc, 0, t, state(t))
    assert np.abs(back.ravel() - state(t)).max() < 1e-12
    lp = lambda tt: O.frame_roundtrip(sc, 0, tt, state(tt))[0][0]
    v_fd = (lp(t - 2 * h) - 8 * lp(t - h) + 8 * lp(t + h) - lp(t + 2 * h)) / (12 * h)
    a_fd = (-lp(t - 2 * h) + 16 * lp(t - h) - 30 * lp(t) + 16 * lp(t + h) - lp(t + 2 * h)) / (12 * h * h)
    assert np.abs(loc[1] - v_fd).max() < 1e-8
    assert np.abs(loc[2] - a_fd).max() < 1e-4


def test_appendix_b_and_c_partials():
    """App. B partial derivatives of Eq. ref_point (with the corrected d x_Q / d y_RX) and App. C's
    d z_QD / dt match finite differences; the printed form of d x_Q / d y_RX does not."""
    xT, yT, xR, yR = 1.3, 2.1, 7.7, 0.9
    xq = lambda xT, yT, xR, yR: xT + (xR - xT) * yT / (yR + yT)
    h = 1e-6
    fd = lambda i: (xq(*[v + h * (j == i) for j, v in enumerate((xT, yT, xR, yR))])
                    - xq(*[v - h * (j == i) for j, v in enumerate((xT, yT, xR, yR))])) / (2 * h)
    s = yT + yR
    assert abs(fd(0) - (1 - yT / s)) < 1e-8
    assert abs(fd(1) - yR * (xR - xT) / s ** 2) < 1e-8
    assert abs(fd(2) - yT / s) < 1e-8
    assert abs(fd(3) - (-yT * (xR - xT) / s ** 2)) < 1e-8           # corrected
    assert abs(fd(3) - (-yR * (xR - xT) / s ** 2)) > 1e-2           # printed (typo) form
    # the oracle's jets give the same velocity for unit rates of each coordinate
    for i, expect in enumerate([1 - yT / s, yR * (xR - xT) / s ** 2, yT / s, -yT * (xR - xT) / s ** 2]):
        T9 = np.array([xT, yT, 0.0, 0, 0, 0, 0, 0, 0])
        R9 = np.array([xR, yR, 0.0, 0, 0, 0, 0, 0, 0])
        (T9 if i < 2 else R9)[3 + (i % 2)] = 1.0
        q = O.ref_point_local(T9, R9)
        assert abs(q[1, 0] - expect) < 1e-12
    # App. C: z_QD velocity for moving terminals, against a finite difference of Eq. diff_point
    T = lambda t: np.array([2.0 + 3 * t, 1.0 - t, 4.0 + 2 * t])
    R = lambda t: np.array([-3.0 + t, -2.0 + 0.5 * t, -1.0 - t])
    zq = lambda t: (R(t)[2] + np.hypot(*R(t)[:2]) * (T(t)[2] - R(t)[2])
                    / (np.hypot(*T(t)[:2]) + np.hypot(*R(t)[:2])))
    q = O.diff_point_local(np.concatenate([T(0), [3, -1, 2], [0, 0, 0]]),
                           np.concatenate([R(0), [1, 0.5, -1], [0, 0, 0]]))
    assert abs(q[0, 2] - zq(0)) < 1e-12
    assert abs(q[1, 2] - (zq(1e-6) - zq(-1e-6)) / 2e-6) < 1e-7
    assert abs(q[2, 2] - (zq(1e-4) - 2 * zq(0) + zq(-1e-4)) / 1e-8) < 1e-4


# ------------------------------------------------------------------------------------------------
# reciprocity
# ------------------------------------------------------------------------------------------------
def test_reciprocity_of_reflection_and_diffraction_chains():
    """Swapping TX and RX and reversing a chain of reflections and perfectly conducting wedge
    diffractions leaves the length, the delay and the complex amplitude unchanged.  (Luebbers'
    lossy-wedge heuristic weights the two reflection terms by face coefficients taken at the source
    and observer angles respectively, so it is not reciprocal; those chains are left out.)"""
    total = 0
    cases = [canyon() + (60e9,)] + [(I.scene_link(k), I.PathSet.from_npz(
        os.path.join(GOLD, f"pathset_link_seed{k}.npz")), 28e9) for k in range(I.LINK_SCENES)]
    for sc, ps, fc in cases:
        keep = [p for p in range(ps.n_paths) if ps.n_int[p] > 0 and T_S_free(ps, p) and pec_wedges(sc, ps, p)]
        sub = ps.subset(keep)
        rev = I.empty_paths(sub.n_paths)
        for p in range(sub.n_paths):
            n = int(sub.n_int[p])
            rev.n_int[p] = n
            rev.types[p, :n] = sub.types[p, :n][::-1]
            rev.prims[p, :n] = sub.prims[p, :n][::-1]
            rev.s0[p, :n] = sub.s0[p, :n][::-1]
        sw = I.Scene(sc.name, sc.rx.copy(), sc.tx.copy(), sc.bodies, sc.materials, sc.faces, sc.edges, sc.tiles)
        a = O.extrapolate(sc, sub, I.TimeGrid(0.2, 1, 1), fc, n_threads=8)
        b = O.extrapolate(sw, rev, I.TimeGrid(0.2, 1, 1), fc, n_threads=8)
        ok = (a["flags"][0] == 0) & (b["flags"][0] == 0)
        total += ok.sum()
        assert np.abs(a["tau"][0] - b["tau"][0])[ok].max() < 1e-12 * a["tau"][0].max()
        assert (np.abs(a["a"][0] - b["a"][0]) <= 1e-9 * np.abs(a["a"][0]))[ok].all()
    assert total > 150


def T_S_free(ps, p):
    return not np.any(ps.types[p, :ps.n_int[p]] == I.T_S)


def pec_wedges(sc, ps, p):
    return all(sc.materials[sc.edges[ps.prims[p, j]]["material"]]["pec"] != 0
               for j in range(int(ps.n_int[p])) if ps.types[p, j] == I.T_D)


# ------------------------------------------------------------------------------------------------
# Fresnel, UTD, ER
# ------------------------------------------------------------------------------------------------
def test_fresnel_limits():
    rte, rtm = O.fresnel(1, 0, True, 3e9, 0.3)
    assert rte == -1 and rtm == 1
    er = 5.3
    rte, rtm = O.fresnel(er, 0.0, False, 3e9, 1.0)
    n = math.sqrt(er)
    assert abs(rte - (1 - n) / (1 + n)) < 1e-14 and abs(rtm + rte) < 1e-14
    cb = math.cos(math.atan(n))            # Brewster angle of a lossless dielectric: R_par = 0
    assert abs(O.fresnel(er, 0.0, False, 3e9, cb)[1]) < 1e-14
    rte, rtm = O.fresnel(er, 0.1, False, 3e9, 1e-9)   # grazing -> -1 for both
    assert abs(rte + 1) < 1e-8 and abs(rtm + 1) < 1e-8
    rte, rtm = O.fresnel(er, 1e9, False, 3e9, 0.6)    # good conductor -> PEC limit
    assert abs(rte + 1) < 1e-3 and abs(rtm - 1) < 1e-3
    for ct in np.linspace(0.01, 1, 50):               # passive: |R| <= 1
        rte, rtm = O.fresnel(er, 0.05, False, 60e9, ct)
        assert abs(rte) <= 1 and abs(rtm) <= 1


def test_fresnel_integral_against_scipy():
    from scipy.special import fresnel as sp_fresnel
    for x in [0.0, 0.01, 0.3, 1.0, 1.7, 2.5, 3.3, 5.0, 9.0, 20.0, 60.0]:
        u = x * math.sqrt(2 / math.pi)
        S, Cf = sp_fresnel(u)
        ref = math.sqrt(math.pi / 2) * ((0.5 - Cf) - 1j * (0.5 - S))
        assert abs(O.fresnel_G(x) - ref) < 1e-13


def test_transition_function_limits():
    for X in (200.0, 1e3, 1e5):
        F = O.transition_F(X)
        # asymptotic series 1 + j/(2X) - 3/(4X^2) - 15j/(8X^3) + ..., error below the next term
        assert abs(F - (1 + 0.5j / X - 0.75 / X ** 2 - 15j / (8 * X ** 3))) < 2 * 105 / (16 * X ** 4) + 1e-13
    for X in (1e-6, 1e-4):
        F = O.transition_F(X)
        assert abs(F - math.sqrt(math.pi * X) * np.exp(1j * math.pi / 4)) < 3 * X


def _wedge_fields(n, phi, phip, sp, s, k, pol, mat=(1.0, 0.0, True), fc=1e9):
    """2D (beta0 = pi/2) scalar GO + UTD field of a point source at (sp, phip) around a wedge edge on
    the z axis, observer at (s, phi); face 0 on phi = 0."""
    src = sp * np.array([math.cos(phip), math.sin(phip)])
    obs = s * np.array([math.cos(phi), math.sin(phi)])
    u = 0j
    if phi < math.pi + phip:                                   # lit by the incident wave
        R = np.linalg.norm(obs - src)
        u += np.exp(-1j * k * R) / R
    if phi < math.pi - phip:                                   # reflected by face 0
        img = sp * np.array([math.cos(-phip), math.sin(-phip)])
        R = np.linalg.norm(obs - img)
        rte, rtm = O.fresnel(mat[0], mat[1], mat[2], fc, math.sin(phip))
        u += (rte if pol == "s" else rtm) * np.exp(-1j * k * R) / R
    L = s * sp / (s + sp)
    Ds, Dh = O.utd(n, phi, phip, 1.0, L, k, *mat, fc=fc)
    D = Ds if pol == "s" else Dh
    ud = np.exp(-1j * k * sp) / sp * D * math.sqrt(sp / (s * (sp + s))) * np.exp(-1j * k * s)
    return u, ud


@pytest.mark.parametrize("n", [1.5, 1.8])
@pytest.mark.parametrize("pol", ["s", "h"])
@pytest.mark.parametrize("mat", [(1.0, 0.0, True), (5.3, 0.1, False)])
def test_utd_restores_continuity_across_shadow_boundaries(n, pol, mat):
    """GO + diffracted field is continuous across the incident and reflection shadow boundaries
    (Kouyoumjian-Pathak); with Luebbers' coefficients also for a lossy wedge at the RSB."""
    k = 2 * math.pi * 1e9 / C0
    phip, sp, s = 0.6, 7.0, 11.0
    boundaries = [math.pi - phip] + ([math.pi + phip] if mat[2] else [])
    for b in boundaries:
        go_m, d_m = _wedge_fields(n, b - 1e-9, phip, sp, s, k, pol, mat)
        go_p, d_p = _wedge_fields(n, b + 1e-9, phip, sp, s, k, pol, mat)
        u_go = 1 / (s + sp)
        assert abs((go_m + d_m) - (go_p + d_p)) < 1e-6 * u_go
        # the check is not vacuous: GO and the diffracted field each jump there
        assert abs(go_m - go_p) > 0.1 * u_go and abs(d_m - d_p) > 0.1 * u_go


def test_er_lobe_normalisation_closed_form():
    """int_hemisphere ((1 + cos psi)/2)^alpha dOmega for alpha = 2, 4 from the binomial expansion
    with I_j = 2 pi/(j+1) (j even), pi cos(ti) (j = 1), pi/4 cos(ti)(3 - cos^2 ti) (j = 3)."""
    for ct in (1.0, 0.8, 0.5, 0.2, 0.05):
        Ij = {0: 2 * math.pi, 1: math.pi * ct, 2: 2 * math.pi / 3, 3: math.pi / 4 * ct * (3 - ct * ct),
              4: 2 * math.pi / 5}
        for a in (2, 4):
            ref = sum(math.comb(a, j) * Ij[j] for j in range(a + 1)) / 2 ** a
            assert abs(O.er_norm(a, ct) - ref) < 1e-12 * ref


def test_er_scattered_power_balance():
    """The ER lobe radiates S^2 times the power intercepted by the tile (adaptive quadrature)."""
    from scipy.integrate import dblquad
    S, area = 0.4, 4.0
    for alpha in (2.0, 4.0):
        for ti in (0.2, 0.9):
            ct = math.cos(ti)
            kspec = np.array([math.sin(ti), 0, ct])

            def f(ph, th):
                s = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
                return O.er_amp(alpha, S, area, ct, float(s @ kspec)) ** 2 * math.sin(th)
            P, _ = dblquad(f, 0, math.pi / 2, 0, 2 * math.pi, epsabs=1e-12, epsrel=1e-10)
            assert abs(P - S * S * area * ct) < 1e-7 * P


def test_free_space_and_single_tile_amplitude():
    """LoS gives lambda/(4 pi d) (Friis); a TX-tile-RX chain in a horizontal plane (vertical
    polarisation kept) gives lambda/(4 pi) x er_amp / (r_i r_s) with the tile's phase."""
    fc = 28e9
    lam = C0 / fc
    b = I._Builder("tile")
    mat = b.material(5.0, 0.01)
    b.tile(0, mat, [0, 10, 2], [0, -1, 0], 4.0, 0.35, 4.0, 0.7)
    sc = b.build(([-6, 0, 2], [0, 0, 0], [0, 0, 0]), ([9, 1, 2], [0, 0, 0], [0, 0, 0]))
    ps = I.chains_to_pathset([[], [(I.T_S, 0)]])
    r = O.extrapolate(sc, ps, I.TimeGrid(0, 1, 1), fc)
    d = math.dist([-6, 0, 2], [9, 1, 2])
    assert abs(r["a"][0, 0] - lam / (4 * math.pi * d)) < 1e-15
    ri, rs = math.dist([-6, 0, 2], [0, 10, 2]), math.dist([0, 10, 2], [9, 1, 2])
    kin = np.array([6.0, 10, 0]) / ri
    kout = np.array([9.0, -9, 0]) / rs
    ct = kin[1]
    kspec = kin - 2 * kin[1] * np.array([0, 1.0, 0])
    ref = lam / (4 * math.pi) * O.er_amp(4.0, 0.35, 4.0, ct, float(kspec @ kout)) / (ri * rs) * np.exp(0.7j)
    assert abs(r["a"][0, 1] - ref) < 1e-12 * abs(ref)


# ------------------------------------------------------------------------------------------------
# validity flags
# ------------------------------------------------------------------------------------------------
def _winding_inside(pt2, poly):
    wn = 0
    for i in range(len(poly)):
        a, b = poly[i], poly[(i + 1) % len(poly)]
        cross = (b[0] - a[0]) * (pt2[1] - a[1]) - (pt2[0] - a[0]) * (b[1] - a[1])
        if a[1] <= pt2[1] < b[1] and cross > 0:
            wn += 1
        elif b[1] <= pt2[1] < a[1] and cross < 0:
            wn -= 1
    return wn != 0


def test_face_flags_against_winding_number():
    """The in-face flag of a path is set exactly when one of its reflection points falls outside its
    face by a winding-number test on the face's corners."""
    sc, ps = canyon()
    n_cmp = 0
    for t in (0.1, 0.5, 0.95):
        r = O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), 60e9, points=True, n_threads=8)
        for p in range(ps.n_paths):
            if r["margin"][0, p] < 1e-9 or not np.any(ps.types[p] == I.T_R):
                continue
            any_out = False
            for j in range(int(ps.n_int[p])):
                if ps.types[p, j] != I.T_R:
                    continue
                f = sc.faces[ps.prims[p, j]]
                if not np.isfinite(f["hu"]):
                    continue
                R = posed_rotation(sc.bodies[f["body"]], t)
                c = posed(sc.bodies[f["body"]], f["c"], t)
                u, n = R @ f["u"], R @ f["n"]
                w = np.cross(u, n)
                corners = [(-f["hu"], -f["hw"]), (f["hu"], -f["hw"]), (f["hu"], f["hw"]), (-f["hu"], f["hw"])]
                q = r["pts"][0, p, j] - c
                any_out |= not _winding_inside((q @ u, q @ w), corners)
            assert bool(int(r["flags"][0, p]) & O.F_FACE) == any_out
            n_cmp += 1
    assert n_cmp > 600


# ------------------------------------------------------------------------------------------------
# H(t, f)
# ------------------------------------------------------------------------------------------------
def test_H_single_path_properties():
    """One path: |H(t, .)| = |a| flat across the band, phase slope -2 pi tau, and the inverse DFT over
    frequency peaks at the delay bin."""
    sc = wall_scene([0, 0, 2], [120, 3, 2])
    ps = I.chains_to_pathset([[]])
    fg = I.FreqGrid(28e9, 400e6, 256)
    r = O.extrapolate(sc, ps, I.TimeGrid(0, 1, 1), fg.fc)
    H = O.synthesize_H(r, fg)[0]
    a, tau = r["a"][0, 0], r["tau"][0, 0]
    assert np.abs(np.abs(H) - abs(a)).max() < 1e-12 * abs(a)
    dphi = np.angle(H[1:] / H[:-1])
    df = fg.bandwidth / fg.n_bins
    assert np.abs(dphi - np.angle(np.exp(-2j * math.pi * df * tau))).max() < 1e-9
    h = np.fft.ifft(H * np.exp(2j * math.pi * (fg.fc - fg.bandwidth / 2) * tau))
    assert int(np.argmax(np.abs(h))) == int(round(tau * fg.bandwidth)) % fg.n_bins


def test_H_is_linear_over_valid_paths():
    """H of a path set is the sum of the H of its valid paths; invalid paths add nothing."""
    sc = I.scene_tiny(0)
    ps = I.chains_tiny(sc)
    fg = I.FreqGrid(28e9, 400e6, 64)
    r = O.extrapolate(sc, ps, I.TimeGrid(0, 0.1, 8), fg.fc)
    H = O.synthesize_H(r, fg)
    acc = np.zeros_like(H)
    for p in range(ps.n_paths):
        rp = {k: (v[:, p:p + 1] if v is not None else None) for k, v in r.items()}
        acc += O.synthesize_H(rp, fg)
    assert np.abs(H - acc).max() < 1e-13 * np.abs(H).max()
    assert (r["flags"] != 0).any()


@pytest.mark.parametrize("edge_kind", ["vertical", "horizontal"])
def test_reflection_plus_diffraction_continuous_at_path_level(edge_kind):
    """A receiver that moves so that a reflection point slides off a metal face across one of the
    face's edges: the reflected path disappears (face flag) exactly where the edge-diffracted path
    takes over, and reflected + diffracted contributions a exp(-jkd) are continuous there.  This
    pins the polarisation bases of the Fresnel and UTD dyads against each other."""
    fc = 3e9
    k = 2 * math.pi * fc / C0
    b = I._Builder("box")
    metal = b.material(1.0, 0.0, pec=True)
    b.box(0, metal, [0, 0, 0.75], np.eye(3), (4.0, 2.0, 1.5))
    if edge_kind == "vertical":
        tx, rx, vrx = [-6.0, 5.0, 1.0], [4.0, 6.0, 1.2], [4.0, 0, 0]
    else:
        tx, rx, vrx = [0.5, 5.0, 0.6], [-0.3, 7.0, 0.2], [0, 0, 2.0]
    sc = b.build((tx, [0, 0, 0], [0, 0, 0]), (rx, vrx, [0, 0, 0]))
    face = [i for i in range(len(sc.faces)) if np.allclose(sc.faces[i]["n"], [0, 1, 0])][0]
    want_dir = [0, 0, 1] if edge_kind == "vertical" else [1, 0, 0]
    cands = []
    for e in range(len(sc.edges)):
        E = sc.edges[e]
        d = (E["b"] - E["a"]) / np.linalg.norm(E["b"] - E["a"])
        touches = any(np.allclose(E[nm], [0, 1, 0]) for nm in ("n0", "nn"))
        if touches and abs(abs(d @ want_dir) - 1) < 1e-12:
            cands.append(e)
    ps = I.chains_to_pathset([[(I.T_R, face)]] + [[(I.T_D, e)] for e in cands])
    ps.s0[1:, 0] = 0.5
    flag_at = lambda t: O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), fc)["flags"][0, 0]
    lo, hi = 0.0, 3.0
    assert flag_at(lo) == 0 and flag_at(hi) & O.F_FACE
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if flag_at(mid) == 0:
            lo = mid
        else:
            hi = mid
    tc = 0.5 * (lo + hi)

    def total(t):
        r = O.extrapolate(sc, ps, I.TimeGrid(t, 1, 1), fc)
        ok = r["flags"][0] == 0
        return np.sum((r["a"][0] * np.exp(-1j * k * r["tau"][0] * C0))[ok]), r
    s_m, r_m = total(tc - 1e-9)
    s_p, r_p = total(tc + 1e-9)
    a_r = abs(r_m["a"][0, 0])
    assert r_m["flags"][0, 0] == 0 and r_p["flags"][0, 0] & O.F_FACE
    assert abs(s_m - s_p) < 1e-4 * a_r
    assert np.abs(r_m["a"][0, 1:]).max() > 0.1 * a_r      # the diffracted path is a real contribution


# ------------------------------------------------------------------------------------------------
# Power-Doppler and power-delay profiles (Sec. IV-A, IV-B)
# ------------------------------------------------------------------------------------------------
def _los_run(fc=5.9e9):
    """LoS only: TX fixed at (0, 0, 5), RX from (50, 0, 5) receding along +x at 20 m/s, so the
    delay is (50 + 20 t)/c, the Doppler shift -20 fc / c and |a| = lambda / (4 pi d) (Friis)."""
    sc = wall_scene([0, 0, 5], [50, 0, 5], vrx=(20.0, 0, 0))
    ps = I.chains_to_pathset([[]])
    tg = I.TimeGrid(0.0, 0.01, 100)
    return O.extrapolate(sc, ps, tg, fc), tg, fc


def test_power_doppler_profile_closed_form():
    rec, tg, fc = _los_run()
    lam = C0 / fc
    t = tg.t_start + tg.dt * np.arange(tg.n_steps)
    pw = (lam / (4 * np.pi * (50 + 20 * t))) ** 2
    fd = -20 * fc / C0
    x0, dx, nb = -1000.0, 14.34, 100
    P = O.power_profile(rec, 20, x0, dx, nb, O.PP_DOPPLER)
    j = int(np.floor((fd - x0) / dx))
    want = np.zeros_like(P)
    want[:, j] = pw.reshape(5, 20).sum(axis=1)
    assert P.shape == (5, nb)
    assert np.allclose(P, want, rtol=1e-9, atol=0)


def test_power_delay_profile_closed_form():
    rec, tg, fc = _los_run()
    lam = C0 / fc
    t = tg.t_start + tg.dt * np.arange(tg.n_steps)
    d = 50 + 20 * t
    x0, dx, nb = 1.0e-7, 1.0e-9, 200
    P = O.power_profile(rec, 7, x0, dx, nb, O.PP_DELAY)   # a ragged last time bin (100 = 14 x 7 + 2)
    want = np.zeros((15, nb))
    for k in range(tg.n_steps):
        want[k // 7, int(np.floor((d[k] / C0 - x0) / dx))] += (lam / (4 * np.pi * d[k])) ** 2
    assert np.allclose(P, want, rtol=1e-9, atol=0)


def test_power_profile_keeps_only_valid_path_steps_in_range():
    """Total power equals the sum of |a|^2 over valid path-steps whose Doppler is in range; a path
    that leaves its face (tiny scene, seed 0: ground-then-box point from t = 0.6 s) stops counting."""
    sc = I.scene_tiny(0)
    ps = I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed0.npz"))
    tg = I.TimeGrid(0.0, 1e-3, 1000)
    rec = O.extrapolate(sc, ps, tg, 28e9, n_threads=8)
    x0, dx, nb = -3000.0, 14.34, 420
    P = O.power_profile(rec, 200, x0, dx, nb, O.PP_DOPPLER)
    valid = rec["flags"] == 0
    inr = (rec["fd"] >= x0) & (rec["fd"] < x0 + dx * nb)
    pw = np.abs(rec["a"]) ** 2
    assert np.isclose(P.sum(), pw[valid & inr].sum(), rtol=1e-12)
    assert (~valid).any() and (pw[~valid] > 0).any()        # invalid path-steps carry power, excluded
    per_bin = np.where(valid & inr, pw, 0).reshape(5, 200, -1).sum(axis=(1, 2))
    assert np.allclose(P.sum(axis=1), per_bin, rtol=1e-12)
