"""Seeded synthetic inputs for the DRT hot path: dynamic environment database + candidate ray chains.

This module is shared by the CUDA product path, the FP64 oracle and the tests.  It holds none of the
method's arithmetic: it draws scenes (bodies, faces, edges, scattering tiles, terminal kinematics) and
candidate interaction sequences, nothing else.  Whether a candidate chain is a valid ray at t0 is
decided elsewhere (the ray-tracing run at t0 is external to DRT, Sec. II).

Scene model (Sec. II, "dynamic environment database"):
  * geometry at t0 in world coordinates: planar rectangular faces, straight wedge edges and
    diffuse-scattering tiles (Sec. III-C), each attached to a rigid body;
  * dynamics: per body a reference point o (rotation centre) with velocity v and constant
    acceleration a (Eq. Taylor), a fixed unit rotation axis k with angular speed w0 and constant
    angular acceleration wdot (Sec. III-A, theta(t) = w0*dt + wdot*dt^2/2); per terminal r, v, a.

Every record layout below is little-endian with natural alignment; the C structures of the library
(include/drt.h) and of the oracle mirror these byte layouts.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------------------------
# Record layouts (one numpy dtype per C structure)
# ----------------------------------------------------------------------------------------------
BODY = np.dtype([("o", "<f8", 3), ("v", "<f8", 3), ("a", "<f8", 3), ("k", "<f8", 3),
                 ("w0", "<f8"), ("wdot", "<f8")])                                  # 112 B
TERMINAL = np.dtype([("r", "<f8", 3), ("v", "<f8", 3), ("a", "<f8", 3)])           # 72 B
MATERIAL = np.dtype([("eps_r", "<f8"), ("sigma", "<f8"), ("rough_s", "<f8"),
                     ("pec", "<f8")])                                              # 32 B
FACE = np.dtype([("body", "<i4"), ("material", "<i4"), ("c", "<f8", 3), ("n", "<f8", 3),
                 ("u", "<f8", 3), ("hu", "<f8"), ("hw", "<f8")])                   # 96 B
EDGE = np.dtype([("body", "<i4"), ("material", "<i4"), ("a", "<f8", 3), ("b", "<f8", 3),
                 ("n0", "<f8", 3), ("nn", "<f8", 3), ("wedge_n", "<f8")])          # 112 B
TILE = np.dtype([("body", "<i4"), ("material", "<i4"), ("c", "<f8", 3), ("n", "<f8", 3),
                 ("area", "<f8"), ("s", "<f8"), ("alpha_r", "<f8"), ("phase", "<f8")])  # 88 B

assert BODY.itemsize == 112 and TERMINAL.itemsize == 72 and MATERIAL.itemsize == 32
assert FACE.itemsize == 96 and EDGE.itemsize == 112 and TILE.itemsize == 88

# interaction type codes of a chain vertex
T_NONE, T_R, T_D, T_S = 0, 1, 2, 3
MAX_INT = 4          # at most 2R + 1D + 1S per chain in the paper's measured case (Sec. IV-B)
C0 = 299792458.0     # speed of light, m/s


@dataclasses.dataclass
class Scene:
    """Dynamic environment database of one link at t0 (all arrays are numpy structured arrays)."""
    name: str
    tx: np.ndarray          # TERMINAL, shape ()
    rx: np.ndarray          # TERMINAL, shape ()
    bodies: np.ndarray      # BODY [B]; body 0 is the static world
    materials: np.ndarray   # MATERIAL [M]
    faces: np.ndarray       # FACE [NF]
    edges: np.ndarray       # EDGE [NE]
    tiles: np.ndarray       # TILE [NT]


@dataclasses.dataclass
class PathSet:
    """Interaction chains of one link, as produced by a ray-tracing run at t0 (Sec. II, Fig. 1)."""
    n_int: np.ndarray       # uint8 [P]       number of interactions (0 = line of sight)
    types: np.ndarray       # uint8 [P, 4]    T_R / T_D / T_S per vertex, T_NONE past n_int
    prims: np.ndarray       # int32 [P, 4]    face / edge / tile index per vertex, -1 past n_int
    s0: np.ndarray          # float64 [P, 4]  edge parameter (m from edge point a) of D vertices at t0

    @property
    def n_paths(self) -> int:
        return int(self.n_int.shape[0])

    def subset(self, idx) -> "PathSet":
        idx = np.asarray(idx)
        return PathSet(self.n_int[idx].copy(), self.types[idx].copy(), self.prims[idx].copy(),
                       self.s0[idx].copy())

    @staticmethod
    def concat(sets) -> "PathSet":
        return PathSet(np.concatenate([s.n_int for s in sets]), np.concatenate([s.types for s in sets]),
                       np.concatenate([s.prims for s in sets]), np.concatenate([s.s0 for s in sets]))

    def to_npz(self, path):
        np.savez_compressed(path, n_int=self.n_int, types=self.types, prims=self.prims, s0=self.s0)

    @staticmethod
    def from_npz(path) -> "PathSet":
        z = np.load(path)
        return PathSet(z["n_int"].astype(np.uint8), z["types"].astype(np.uint8),
                       z["prims"].astype(np.int32), z["s0"].astype(np.float64))


@dataclasses.dataclass
class TimeGrid:
    """t_n = t0 + t_start + n*dt, n = 0..n_steps-1 (times relative to t0 in seconds)."""
    t_start: float
    dt: float
    n_steps: int


@dataclasses.dataclass
class FreqGrid:
    """f_k = fc - bandwidth/2 + k*bandwidth/n_bins, k = 0..n_bins-1; coefficients are taken at fc."""
    fc: float
    bandwidth: float
    n_bins: int


def empty_paths(n: int) -> PathSet:
    return PathSet(np.zeros(n, np.uint8), np.zeros((n, MAX_INT), np.uint8),
                   np.full((n, MAX_INT), -1, np.int32), np.zeros((n, MAX_INT), np.float64))


def chains_to_pathset(chains) -> PathSet:
    """chains: list of [(type, prim), ...] (empty list = line of sight)."""
    ps = empty_paths(len(chains))
    for i, ch in enumerate(chains):
        ps.n_int[i] = len(ch)
        for j, (ty, pr) in enumerate(ch):
            ps.types[i, j] = ty
            ps.prims[i, j] = pr
    return ps


# ----------------------------------------------------------------------------------------------
# Scene builders
# ----------------------------------------------------------------------------------------------
def _unit(x):
    x = np.asarray(x, np.float64)
    return x / np.linalg.norm(x)


def _rot_z(yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _rot_axis(k, ang):
    k = _unit(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


class _Builder:
    def __init__(self, name):
        self.name = name
        self.bodies = [dict(o=[0, 0, 0], v=[0, 0, 0], a=[0, 0, 0], k=[0, 0, 1], w0=0.0, wdot=0.0)]
        self.materials = []
        self.faces, self.edges, self.tiles = [], [], []

    def material(self, eps_r, sigma, rough_s=0.0, pec=False):
        self.materials.append((eps_r, sigma, rough_s, 1.0 if pec else 0.0))
        return len(self.materials) - 1

    def body(self, o, v, a, k=(0, 0, 1), w0=0.0, wdot=0.0):
        self.bodies.append(dict(o=o, v=v, a=a, k=_unit(k), w0=w0, wdot=wdot))
        return len(self.bodies) - 1

    def face(self, body, mat, c, n, u, hu, hw):
        self.faces.append((body, mat, c, _unit(n), _unit(u), hu, hw))
        return len(self.faces) - 1

    def edge(self, body, mat, p, q, n0, nn):
        """Wedge edge between the 0-face (outward normal n0) and the n-face (outward normal nn).

        The endpoints are ordered so that (b - a) is parallel to n0 x nn; the exterior wedge
        parameter is n = 1 + angle(n0, nn)/pi (n = 1.5 for a right-angled corner)."""
        n0, nn = _unit(n0), _unit(nn)
        e = np.cross(n0, nn)
        p, q = np.asarray(p, float), np.asarray(q, float)
        a, b = (p, q) if np.dot(q - p, e) > 0 else (q, p)
        wn = 1.0 + math.acos(max(-1.0, min(1.0, float(np.dot(n0, nn))))) / math.pi
        self.edges.append((body, mat, a, b, n0, nn, wn))
        return len(self.edges) - 1

    def tile(self, body, mat, c, n, area, s, alpha_r, phase):
        self.tiles.append((body, mat, c, _unit(n), area, s, alpha_r, phase))

    def box(self, body, mat, centre, R, dims, with_faces=True, with_edges=True):
        """Axis-aligned (in body frame R) box: 6 faces and 12 right-angled wedge edges."""
        centre = np.asarray(centre, float)
        h = 0.5 * np.asarray(dims, float)
        ax = [R[:, 0], R[:, 1], R[:, 2]]
        if with_faces:
            for i in range(3):
                j, k = (i + 1) % 3, (i + 2) % 3
                for sgn in (1.0, -1.0):
                    self.face(body, mat, centre + sgn * h[i] * ax[i], sgn * ax[i], ax[j], h[j], h[k])
        if with_edges:
            for i in range(3):              # edge direction along axis i
                j, k = (i + 1) % 3, (i + 2) % 3
                for sj in (1.0, -1.0):
                    for sk in (1.0, -1.0):
                        base = centre + sj * h[j] * ax[j] + sk * h[k] * ax[k]
                        self.edge(body, mat, base - h[i] * ax[i], base + h[i] * ax[i],
                                  sj * ax[j], sk * ax[k])

    def build(self, tx, rx):
        def arr(rows, dt):
            out = np.zeros(len(rows), dt)
            for i, r in enumerate(rows):
                out[i] = r
            return out
        bodies = np.zeros(len(self.bodies), BODY)
        for i, b in enumerate(self.bodies):
            bodies[i] = (b["o"], b["v"], b["a"], b["k"], b["w0"], b["wdot"])
        t = np.zeros((), TERMINAL)
        t[()] = tx
        r = np.zeros((), TERMINAL)
        r[()] = rx
        return Scene(self.name, t, r, bodies, arr(self.materials, MATERIAL), arr(self.faces, FACE),
                     arr(self.edges, EDGE), arr(self.tiles, TILE))


def scene_tiny(seed: int = 0) -> Scene:
    """28 GHz tiny scene: fixed TX (0,0,5), RX from (50,0,1.5) at +10 m/s along x, infinite concrete
    ground (eps_r 5.3, sigma 0.1 S/m) and one 4.5 x 1.8 x 1.5 m metal box on the ground at +15 m/s
    along x, in the TX-RX lane ahead of RX (its rear face then faces both terminals).  seed 0 puts
    the rear face 21 m beyond RX, so the ground-then-box reflection point slides off the bottom of
    the face about 0.6 s in; seed 1 puts it 5.75 m beyond RX, where that point stays on the face."""
    b = _Builder(f"tiny-seed{seed}")
    concrete = b.material(5.3, 0.1)
    metal = b.material(1.0, 0.0, pec=True)
    b.face(0, concrete, [0, 0, 0], [0, 0, 1], [1, 0, 0], math.inf, math.inf)
    x0 = {0: 73.25, 1: 58.0}.get(seed, 58.0 + 15.0 * np.random.default_rng(seed).random())
    centre = np.array([x0, 0.0, 0.75])
    body = b.body(centre, [15.0, 0, 0], [0, 0, 0])
    b.box(body, metal, centre, np.eye(3), (4.5, 1.8, 1.5))
    tx = ([0.0, 0.0, 5.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    rx = ([50.0, 0.0, 1.5], [10.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    return b.build(tx, rx)


def chains_tiny(scene: Scene):
    """LoS plus every reflection chain of order <= 2 over the scene's faces (candidates)."""
    nf = len(scene.faces)
    chains = [[]]
    chains += [[(T_R, f)] for f in range(nf)]
    chains += [[(T_R, f), (T_R, g)] for f in range(nf) for g in range(nf) if f != g]
    return chains_to_pathset(chains)


def scene_canyon(seed: int = 0, n_facades: int = 40, n_vehicles: int = 8, width: float = 20.0,
                 tile_size: float = 2.0) -> Scene:
    """Urban canyon along x, `width` m wide: facades on both sides (rectangles 10-30 m long, 10-30 m
    high, random +-5 deg yaw/tilt, eps_r ~ U[3,7], sigma ~ U[0.01,0.1] S/m) with right-angled end and
    roof edges and ER scattering tiles (S ~ U[0.2,0.5], alpha_R in {2,4}); a concrete ground plane;
    metal 4.5 x 1.8 x 1.5 m vehicles in four lanes with speeds U[5,30] m/s, yaw rates
    U[-0.3,0.3] rad/s and accelerations U[-2,2] m/s^2 along the heading.  TX and RX ride 0.25 m
    above the roofs of vehicles 0 and 1 with those vehicles' velocity and acceleration."""
    rng = np.random.default_rng(1000 + seed)
    b = _Builder(f"canyon-seed{seed}")
    concrete = b.material(5.3, 0.1)
    metal = b.material(1.0, 0.0, pec=True)
    b.face(0, concrete, [0, 0, 0], [0, 0, 1], [1, 0, 0], math.inf, math.inf)
    per_side = n_facades // 2
    for side in (+1.0, -1.0):
        x = -0.5 * per_side * 21.5
        for _ in range(per_side):
            length = rng.uniform(10, 30)
            height = rng.uniform(10, 30)
            yaw = math.radians(rng.uniform(-5, 5))
            tilt = math.radians(rng.uniform(-5, 5))
            mat = b.material(rng.uniform(3, 7), rng.uniform(0.01, 0.1))
            # facade frame: u along street, n into the street, w up
            R = _rot_z(yaw)
            u = R @ np.array([1.0, 0, 0])
            n = R @ np.array([0, -side, 0])
            Rt = _rot_axis(u, tilt)
            n = Rt @ n
            up = np.cross(n, u) * side           # upward in-plane axis
            centre = np.array([x + 0.5 * length, side * 0.5 * width, 0.0]) + 0.5 * height * up
            f = b.face(0, mat, centre, n, u, 0.5 * length, 0.5 * height)
            del f
            lo, hi = centre - 0.5 * height * up, centre + 0.5 * height * up
            for s_end in (-1.0, 1.0):         # vertical building corners at the facade ends
                off = s_end * 0.5 * length * u
                b.edge(0, mat, lo + off, hi + off, n, s_end * u)
            b.edge(0, mat, hi - 0.5 * length * u, hi + 0.5 * length * u, n, up)   # roof edge
            nu = max(1, int(round(length / tile_size)))
            nw = max(1, int(round(height / tile_size)))
            for iu in range(nu):
                for iw in range(nw):
                    cu = (iu + 0.5) / nu - 0.5
                    cw = (iw + 0.5) / nw - 0.5
                    c = centre + cu * length * u + cw * height * up
                    b.tile(0, mat, c, n, (length / nu) * (height / nw), rng.uniform(0.2, 0.5),
                           float(rng.choice([2.0, 4.0])), rng.uniform(0, 2 * math.pi))
            x += length + rng.uniform(0.5, 3.0)
    lanes = [(-7.5, 1.0), (-2.5, 1.0), (2.5, -1.0), (7.5, -1.0)]
    veh = []
    order = [1, 2, 0, 3, 1, 2, 0, 3]
    for i in range(n_vehicles):
        ly, dirn = lanes[order[i % len(order)]]
        x0 = rng.uniform(-30, 30) if i < 2 else rng.uniform(-80, 80)
        speed = rng.uniform(5, 30)
        yaw_rate = rng.uniform(-0.3, 0.3)
        acc = rng.uniform(-2, 2)
        heading = np.array([dirn, 0.0, 0.0])
        centre = np.array([x0, ly, 0.3 + 0.75])
        body = b.body(centre, speed * heading, acc * heading, [0, 0, 1], yaw_rate, 0.0)
        b.box(body, metal, centre, np.eye(3), (4.5, 1.8, 1.5))
        veh.append((centre, speed * heading, acc * heading))
    (c0, v0, a0), (c1, v1, a1) = veh[0], veh[1]
    tx = (c0 + [0, 0, 1.0], v0, a0)
    rx = (c1 + [0, 0, 1.0], v1, a1)
    return b.build(tx, rx)


def scene_link(seed: int = 0, n_facades: int = 24, tile_size: float = 3.0) -> Scene:
    """A link of the batched workload: the tiny 28 GHz scene (fixed TX at (0,0,5), RX from
    (50,0,1.5) at +10 m/s, concrete ground, one metal 4.5 x 1.8 x 1.5 m box at +15 m/s ahead of RX,
    its start drawn in [58, 73] m) plus `n_facades` static building facades around the road
    (8-30 m either side of it, 10-30 m long, 5-20 m high, +-20 deg yaw, eps_r ~ U[3,7],
    sigma ~ U[0.01,0.1] S/m) with their end and roof wedge edges and ER tiles (S ~ U[0.2,0.5],
    alpha_R in {2,4}) on which the extra paths of the link are drawn."""
    rng = np.random.default_rng(5000 + seed)
    b = _Builder(f"link-seed{seed}")
    concrete = b.material(5.3, 0.1)
    metal = b.material(1.0, 0.0, pec=True)
    b.face(0, concrete, [0, 0, 0], [0, 0, 1], [1, 0, 0], math.inf, math.inf)
    x0 = rng.uniform(58.0, 73.0)
    centre = np.array([x0, 0.0, 0.75])
    body = b.body(centre, [15.0, 0, 0], [0, 0, 0])
    b.box(body, metal, centre, np.eye(3), (4.5, 1.8, 1.5))
    for i in range(n_facades):
        side = 1.0 if i % 2 == 0 else -1.0
        length, height = rng.uniform(10, 30), rng.uniform(5, 20)
        yaw = math.radians(rng.uniform(-20, 20))
        mat = b.material(rng.uniform(3, 7), rng.uniform(0.01, 0.1))
        R = _rot_z(yaw)
        u = R @ np.array([1.0, 0, 0])
        n = R @ np.array([0, -side, 0])          # facing the road
        up = np.array([0.0, 0.0, 1.0])
        centre = np.array([rng.uniform(-20, 110), side * rng.uniform(8, 30), 0.5 * height])
        b.face(0, mat, centre, n, u, 0.5 * length, 0.5 * height)
        lo, hi = centre - 0.5 * height * up, centre + 0.5 * height * up
        for s_end in (-1.0, 1.0):
            off = s_end * 0.5 * length * u
            b.edge(0, mat, lo + off, hi + off, n, s_end * u)
        b.edge(0, mat, hi - 0.5 * length * u, hi + 0.5 * length * u, n, up)
        nu = max(1, int(round(length / tile_size)))
        nw = max(1, int(round(height / tile_size)))
        for iu in range(nu):
            for iw in range(nw):
                c = centre + ((iu + 0.5) / nu - 0.5) * length * u + ((iw + 0.5) / nw - 0.5) * height * up
                b.tile(0, mat, c, n, (length / nu) * (height / nw), rng.uniform(0.2, 0.5),
                       float(rng.choice([2.0, 4.0])), rng.uniform(0, 2 * math.pi))
    tx = ([0.0, 0.0, 5.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    rx = ([50.0, 0.0, 1.5], [10.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    return b.build(tx, rx)


HIGHWAY = dict(n_links=64, n_tiles=20000, n_rd=300, carriers=(28e9, 60e9), bandwidth=400e6, n_bins=1024,
               dt=1e-4, n_steps=20000)


def _highway_base(seed: int):
    """Static part and vehicles of the highway scene (see scene_highway)."""
    rng = np.random.default_rng(3000 + seed)
    b = _Builder(f"highway-seed{seed}")
    concrete = b.material(5.3, 0.1)
    metal = b.material(1.0, 0.0, pec=True)
    b.face(0, concrete, [0, 0, 0], [0, 0, 1], [1, 0, 0], math.inf, math.inf)
    # noise barriers along both road sides, 4 m high, in 50 m panels with top wedge edges; ER tiles
    # of 0.6 m x 0.8 m (2000 x 5 per side) on their road-facing sides
    half, n_panel, panel, height = 600.0, 24, 50.0, 4.0
    n_col, n_row = HIGHWAY["n_tiles"] // 10, 5
    up = np.array([0.0, 0.0, 1.0])
    for side in (+1.0, -1.0):
        mat = b.material(rng.uniform(4, 6), rng.uniform(0.01, 0.05))
        n = np.array([0.0, -side, 0.0])                      # facing the road
        u = np.array([1.0, 0.0, 0.0])
        for k in range(n_panel):
            centre = np.array([-half + (k + 0.5) * panel, side * 13.0, 0.5 * height])
            b.face(0, mat, centre, n, u, 0.5 * panel, 0.5 * height)
            top = centre + 0.5 * height * up
            b.edge(0, mat, top - 0.5 * panel * u, top + 0.5 * panel * u, n, up)
        w, h = 2 * half / n_col, height / n_row
        for i in range(n_col):
            for j in range(n_row):
                c = np.array([-half + (i + 0.5) * w, side * 13.0, (j + 0.5) * h])
                b.tile(0, mat, c, n, w * h, rng.uniform(0.2, 0.5), float(rng.choice([2.0, 4.0])),
                       rng.uniform(0, 2 * math.pi))
    # 60 vehicles, 10 per lane (3 lanes each way, 3.5 m wide): 3 in 4 cars (4.5 x 1.8 x 1.5 m), the
    # rest trucks (12 x 2.5 x 3.8 m); speeds U[20, 36] m/s, yaw rates U[-0.02, 0.02] rad/s,
    # accelerations U[-1, 1] m/s^2 along the heading
    veh = []
    for lane in range(6):
        y = (-8.75, -5.25, -1.75, 1.75, 5.25, 8.75)[lane]
        dirn = 1.0 if y < 0 else -1.0
        for i in range(10):
            truck = rng.uniform() < 0.25
            dims = (12.0, 2.5, 3.8) if truck else (4.5, 1.8, 1.5)
            centre = np.array([-300.0 + 60.0 * i + rng.uniform(0, 30), y, 0.3 + 0.5 * dims[2]])
            heading = np.array([dirn, 0.0, 0.0])
            speed, acc = rng.uniform(20, 36), rng.uniform(-1, 1)
            body = b.body(centre, speed * heading, acc * heading, [0, 0, 1], rng.uniform(-0.02, 0.02), 0.0)
            b.box(body, metal, centre, np.eye(3), dims)
            veh.append((centre + [0, 0, 0.5 * dims[2] + 0.25], speed * heading, acc * heading))
    return b, veh


def scene_highway(seed: int = 0, link: int = 0) -> Scene:
    """Large vehicular highway: 6 lanes, 60 translating and yawing vehicles (metal boxes), a
    concrete ground plane and two 4 m noise barriers 13 m either side of the centre line carrying
    20000 ER tiles (S ~ U[0.2,0.5], alpha_R in {2,4}) that face the road.  Link `link` puts TX and
    RX 0.25 m above the roofs of two distinct vehicles drawn near the middle of the road (seeded),
    with those vehicles' velocity and acceleration.  The tiles face every terminal on the road, so
    every single-scatter chain is a ray at t0."""
    if seed not in _HIGHWAY_CACHE:
        b, veh = _highway_base(seed)
        _HIGHWAY_CACHE[seed] = (b.build(veh[0], veh[1]), veh)
    base, veh = _HIGHWAY_CACHE[seed]
    rng = np.random.default_rng(7000 + 100 * seed + link)
    mid = [i for i, (c, _, _) in enumerate(veh) if abs(c[0]) < 200.0]
    i, j = rng.choice(mid, size=2, replace=False)
    tx, rx = np.zeros((), TERMINAL), np.zeros((), TERMINAL)
    tx[()], rx[()] = veh[int(i)], veh[int(j)]
    return dataclasses.replace(base, name=f"{base.name}-link{link}", tx=tx, rx=rx)


_HIGHWAY_CACHE: dict = {}   # seed -> (scene with the static part and vehicles, vehicle terminals)


def highway_tile_chains(n_tiles: int):
    """The single-scatter chains of the highway links, one per tile."""
    ps = PathSet(np.ones(n_tiles, np.uint8), np.zeros((n_tiles, 4), np.uint8), np.full((n_tiles, 4), -1, np.int32),
                 np.zeros((n_tiles, 4)))
    ps.types[:, 0] = T_S
    ps.prims[:, 0] = np.arange(n_tiles, dtype=np.int32)
    return ps


def highway_pathset(rd: PathSet, link: int, n_tiles: int | None = None, n_rd: int | None = None) -> PathSet:
    """Path set of highway link `link`: its reflection / diffraction chains (rows
    [link n_rd, (link + 1) n_rd) of the committed set `rd`) and one single-scatter chain per tile."""
    n_tiles = HIGHWAY["n_tiles"] if n_tiles is None else n_tiles
    n_rd = HIGHWAY["n_rd"] if n_rd is None else n_rd
    return PathSet.concat([rd.subset(np.arange(link * n_rd, (link + 1) * n_rd)), highway_tile_chains(n_tiles)])


def draw_chains_batch(rng, scene: Scene, n: int, p_r: float = 0.75, lengths=(1, 2)) -> PathSet:
    """n candidate reflection / diffraction chains at once: length uniform on `lengths`, each vertex R
    with probability p_r else D, uniform faces / edges, a vertex never repeating its predecessor's
    primitive (the next index is taken instead), D edge parameters at the edge midpoint."""
    nf, ne = len(scene.faces), len(scene.edges)
    L = rng.choice(np.asarray(lengths), size=n)
    is_r = rng.uniform(size=(n, MAX_INT)) < p_r
    u = rng.uniform(size=(n, MAX_INT))
    prim = np.where(is_r, (u * nf).astype(np.int64), (u * ne).astype(np.int64))
    for j in range(1, MAX_INT):
        same = (is_r[:, j] == is_r[:, j - 1]) & (prim[:, j] == prim[:, j - 1])
        prim[same, j] = (prim[same, j] + 1) % np.where(is_r[same, j], nf, ne)
    live = np.arange(MAX_INT)[None, :] < L[:, None]
    types = np.where(live, np.where(is_r, T_R, T_D), T_NONE).astype(np.uint8)
    prims = np.where(live, prim, -1).astype(np.int32)
    half = 0.5 * np.linalg.norm(scene.edges["b"] - scene.edges["a"], axis=1) if ne else np.zeros(1)
    s0 = np.where(live & ~is_r, half[np.clip(prim, 0, max(ne - 1, 0))], 0.0)
    return PathSet(L.astype(np.uint8), types, prims, s0)


def draw_chain_types(rng, p_types=(0.6, 0.2, 0.2), lengths=(1, 2, 3)):
    """Interaction types of one chain: length uniform on `lengths`, types i.i.d. R:D:S."""
    n = int(rng.choice(lengths))
    return [int(t) for t in rng.choice([T_R, T_D, T_S], size=n, p=p_types)]


def draw_chain_prims(rng, scene: Scene, types):
    """Uniform random primitive for each interaction type (faces / edges / tiles).

    Two consecutive interactions never use the same primitive; edge parameters s0 start at the
    edge midpoint."""
    n_prim = {T_R: len(scene.faces), T_D: len(scene.edges), T_S: len(scene.tiles)}
    chain, s0 = [], []
    for t in types:
        if n_prim[t] == 0:
            return None, None
        for _ in range(8):
            p = int(rng.integers(n_prim[t]))
            if not chain or chain[-1] != (t, p):
                break
        chain.append((t, p))
        if t == T_D:
            e = scene.edges[p]
            s0.append(0.5 * float(np.linalg.norm(e["b"] - e["a"])))
        else:
            s0.append(0.0)
    return chain, s0


# ----------------------------------------------------------------------------------------------
# Workload descriptions (sizes of the paper-shaped synthetic workloads)
# ----------------------------------------------------------------------------------------------
WORKLOADS = {
    # LoS + reflections of order <= 2, 28 GHz, 1000 x 1 ms, 256 bins over 400 MHz
    "tiny": dict(scene=scene_tiny, fc=28e9, bandwidth=400e6, n_bins=256, dt=1e-3, n_steps=1000),
    # full-3D canyon, 512 chains of <= 3 interactions (R:D:S = 6:2:2), 60 GHz, 2000 x 0.5 ms,
    # 512 bins over 1 GHz
    "canyon": dict(scene=scene_canyon, fc=60e9, bandwidth=1e9, n_bins=512, dt=0.5e-3,
                   n_steps=2000, n_paths=512),
}


# the batched workload: `n_links` links of scene_link(seed % LINK_SCENES) with the first P paths of
# that scene's path set, P log-uniform in [8, 2048], horizons uniform in [100, 5000] steps of 1 ms,
# 256 bins over 400 MHz at 28 GHz
LINK_SCENES = 4
BATCH = dict(fc=28e9, bandwidth=400e6, n_bins=256, dt=1e-3, p_range=(8, 2048), t_range=(100, 5000))


def batch_links(n_links: int, seed: int = 0, p_range=None, t_range=None):
    """Per link of the batched workload: (scene index, path count P, horizon T), seeded."""
    rng = np.random.default_rng(9000 + seed)
    p_lo, p_hi = p_range or BATCH["p_range"]
    t_lo, t_hi = t_range or BATCH["t_range"]
    P = np.exp(rng.uniform(math.log(p_lo), math.log(p_hi), n_links)).astype(np.int64)
    T = rng.integers(t_lo, t_hi + 1, n_links)
    return [(i % LINK_SCENES, int(max(p_lo, min(p_hi, P[i]))), int(T[i])) for i in range(n_links)]


def grids(workload: str, n_steps: int | None = None, n_bins: int | None = None):
    w = WORKLOADS[workload]
    tg = TimeGrid(0.0, w["dt"], n_steps if n_steps is not None else w["n_steps"])
    fg = FreqGrid(w["fc"], w["bandwidth"], n_bins if n_bins is not None else w["n_bins"])
    return tg, fg
