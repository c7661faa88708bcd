"""Write the committed path sets of the synthetic workloads (the "ray-tracing run at t0").

DRT starts from the multipath geometry found by a conventional ray-tracing run at t0 (Sec. II); that
run is outside the DRT hot path.  This script stands in for it: it draws candidate interaction
chains from the seeded generators of ``paper_2205_00237_gb300.inputs`` and keeps those that the FP64
oracle finds valid at t0 (every point on its face or edge, every neighbour on the correct side).  It
calls only ``oracle/`` and the input generators, never the CUDA library.

  python tests/golden/make_pathsets.py        # rewrites tests/golden/pathset_*.npz (--all: and the
                                              # highway chains; --highway-only: those alone)

Chain draws for the canyon follow the stated recipe: LoS plus chains of length uniform on {1,2,3}
with i.i.d. types R:D:S = 0.6:0.2:0.2 and uniform primitives; a drawn type sequence gets up to
`tries` random primitive assignments and is redrawn when none of them is valid at t0.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2205_00237_gb300 import inputs as I  # noqa: E402


def keep_valid_at_t0(scene, ps, fc, n_threads=8):
    r = O.extrapolate(scene, ps, I.TimeGrid(0.0, 1.0, 1), fc, n_threads=n_threads, points=True)
    ok = np.nonzero(r["flags"][0] == 0)[0]
    out = ps.subset(ok)
    # edge parameters of the D vertices at t0 (the ray-tracing result the Newton warm start uses)
    pts = r["pts"][0, ok]
    for p in range(out.n_paths):
        for j in range(int(out.n_int[p])):
            if out.types[p, j] == I.T_D:
                e = scene.edges[out.prims[p, j]]
                ed = (e["b"] - e["a"]) / np.linalg.norm(e["b"] - e["a"])
                out.s0[p, j] = float(np.dot(pts[p, j] - e["a"], ed))
    return out


def chain_key(ps, p):
    return tuple((int(ps.types[p, j]), int(ps.prims[p, j])) for j in range(int(ps.n_int[p])))


def drawn_pathset(scene, rng, n_paths, fc, kept=None, tries=60000, batch=3000):
    """Fill up to n_paths with drawn chains valid at t0; a chain already in the set is not taken
    again (a ray-tracing run finds each ray once)."""
    kept = kept or [keep_valid_at_t0(scene, I.chains_to_pathset([[]]), fc)]       # line of sight
    seen = {chain_key(k, p) for k in kept for p in range(k.n_paths)}
    n = sum(k.n_paths for k in kept)
    exhausted = set()
    while n < n_paths:
        types = I.draw_chain_types(rng)
        if tuple(types) in exhausted:      # no fresh valid chain left for this type sequence
            continue
        found = None
        for _ in range(tries // batch):
            chains, s0s = [], []
            for _ in range(batch):
                ch, s0 = I.draw_chain_prims(rng, scene, types)
                if ch is not None:
                    chains.append(ch)
                    s0s.append(s0)
            ps = I.chains_to_pathset(chains)
            for i, s in enumerate(s0s):
                ps.s0[i, :len(s)] = s
            v = keep_valid_at_t0(scene, ps, fc)
            fresh = [p for p in range(v.n_paths) if chain_key(v, p) not in seen]
            if fresh:
                found = v.subset([fresh[0]])
                break
        if found is None:
            exhausted.add(tuple(types))
        else:
            kept.append(found)
            seen.add(chain_key(found, 0))
            n += 1
            if n % 256 == 0:
                print(f"  {n} chains", flush=True)
    return I.PathSet.concat(kept)


def canyon_pathset(seed, n_paths=512, fc=60e9):
    scene = I.scene_canyon(seed)
    return scene, drawn_pathset(scene, np.random.default_rng(77 + seed), n_paths, fc)


def link_pathset(seed, n_paths=2048, fc=28e9):
    """Links of the batched workload: LoS and the valid reflections of order <= 2 of the tiny
    geometry first, then drawn R:D:S chains on the facades.  A link of P paths takes the first P."""
    scene = I.scene_link(seed)
    base = keep_valid_at_t0(scene, I.chains_tiny(scene), fc)
    return scene, drawn_pathset(scene, np.random.default_rng(177 + seed), n_paths, fc, kept=[base])


def highway_rd_pathsets(seed=0, fc=28e9, batch=20000):
    """Reflection / diffraction chains of the highway links: LoS, then candidate chains of length
    uniform on {1, 2} with i.i.d. types R:D = 3:1 and uniform faces / edges, kept in draw order when
    valid at t0 and not yet taken, until `n_rd` chains per link.  The tile chains of a link are implicit
    (one per tile, every tile faces the road: inputs.highway_tile_chains)."""
    hw = I.HIGHWAY
    rng = np.random.default_rng(4000 + seed)
    out = []
    for link in range(hw["n_links"]):
        scene = I.scene_highway(seed, link)
        kept = [keep_valid_at_t0(scene, I.chains_to_pathset([[]]), fc)]
        seen = {()}
        n = 1
        while n < hw["n_rd"]:
            v = keep_valid_at_t0(scene, I.draw_chains_batch(rng, scene, batch), fc)
            for p in range(v.n_paths):
                k = chain_key(v, p)
                if k not in seen and n < hw["n_rd"]:
                    seen.add(k)
                    kept.append(v.subset([p]))
                    n += 1
        out.append(I.PathSet.concat(kept))
        print(f"  highway link {link}: {n} chains", flush=True)
    return I.PathSet.concat(out)


def tiny_pathset(seed, fc=28e9):
    scene = I.scene_tiny(seed)
    return scene, keep_valid_at_t0(scene, I.chains_tiny(scene), fc)


def main():
    if "--highway-only" in sys.argv or "--all" in sys.argv:
        ps = highway_rd_pathsets(0)
        ps.to_npz(os.path.join(HERE, "pathset_highway_rd_seed0.npz"))
        print(f"highway seed 0: {ps.n_paths} reflection / diffraction chains over {I.HIGHWAY['n_links']} links")
        if "--highway-only" in sys.argv:
            return
    for seed in (0, 1):
        scene, ps = tiny_pathset(seed)
        ps.to_npz(os.path.join(HERE, f"pathset_tiny_seed{seed}.npz"))
        print(f"tiny seed {seed}: {ps.n_paths} paths")
    for seed in range(I.LINK_SCENES):
        scene, ps = link_pathset(seed)
        ps.to_npz(os.path.join(HERE, f"pathset_link_seed{seed}.npz"))
        print(f"link seed {seed}: {ps.n_paths} paths")
    if "--links-only" in sys.argv:
        return

    scene, ps = canyon_pathset(0)
    ps.to_npz(os.path.join(HERE, "pathset_canyon_seed0.npz"))
    sig = {}
    for p in range(ps.n_paths):
        k = "".join("xRDS"[t] for t in ps.types[p, :ps.n_int[p]]) or "LoS"
        sig[k] = sig.get(k, 0) + 1
    print(f"canyon seed 0: {ps.n_paths} paths", sorted(sig.items(), key=lambda x: -x[1]))


if __name__ == "__main__":
    main()
