"""CPU checks of the highway workload inputs: sizes, the per-link terminal choice, and that every
single-scatter chain is a ray over the whole horizon (the tiles face the road)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_highway_scene_shape():
    hw = I.HIGHWAY
    sc = I.scene_highway(0, 0)
    assert len(sc.tiles) == hw["n_tiles"]
    assert len(sc.bodies) == 61                       # the static world + 60 vehicles
    assert set(np.unique(sc.tiles["alpha_r"])) <= {2.0, 4.0}
    assert (sc.tiles["s"] >= 0.2).all() and (sc.tiles["s"] <= 0.5).all()
    a, b = I.scene_highway(0, 1), I.scene_highway(0, 1)
    assert np.array_equal(a.tx["r"], b.tx["r"]) and not np.array_equal(a.tx["r"], sc.tx["r"])
    assert sc.bodies is a.bodies                      # links share the static part


@pytest.mark.parametrize("link", [0, 37])
def test_every_tile_chain_is_a_ray_over_the_horizon(link):
    hw = I.HIGHWAY
    sc = I.scene_highway(0, link)
    ps = I.highway_tile_chains(hw["n_tiles"])
    steps = [0, hw["n_steps"] // 2, hw["n_steps"] - 1]
    for n in steps:
        r = O.extrapolate(sc, ps, I.TimeGrid(n * hw["dt"], hw["dt"], 1), hw["carriers"][0], n_threads=8)
        assert (r["flags"] == 0).all()


def test_highway_link_pathsets():
    path = os.path.join(GOLD, "pathset_highway_rd_seed0.npz")
    if not os.path.exists(path):
        pytest.skip("highway chains not generated")
    hw = I.HIGHWAY
    rd = I.PathSet.from_npz(path)
    assert rd.n_paths == hw["n_links"] * hw["n_rd"]
    for link in (0, hw["n_links"] - 1):
        ps = I.highway_pathset(rd, link)
        assert ps.n_paths == hw["n_rd"] + hw["n_tiles"]
        assert ps.n_int[0] == 0                        # line of sight first
        assert set(np.unique(ps.types[:hw["n_rd"], 0])) <= {I.T_NONE, I.T_R, I.T_D}
        r = O.extrapolate(I.scene_highway(0, link), ps.subset(np.arange(hw["n_rd"])),
                          I.TimeGrid(0.0, 1.0, 1), hw["carriers"][0], n_threads=8)
        assert (r["flags"][0] == 0).all()              # the chains are rays at t0
