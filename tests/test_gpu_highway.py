"""The large vehicular highway at full size, through the batched FP32-bulk form, against the oracle.

64 links of the highway scene (60 translating and yawing vehicles, 20000 ER tiles on the road-side
barriers, 300 reflection / diffraction chains per link), each at 28 GHz and at 60 GHz (geometry
recomputed per carrier), 20000 steps of 0.1 ms and 1024 bins: 128 batch entries, 5.2e10 path-steps.
Rows sampled from three links per carrier are compared with the oracle's direct FP64 sum within the
FP32-bulk H bars (boundary path-steps bounded by their amplitudes).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_gpu_parity import compare_H_band

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


def test_highway_full_size_sampled(ctx):
    import torch
    hw = I.HIGHWAY
    rd = I.PathSet.from_npz(os.path.join(GOLD, "pathset_highway_rd_seed0.npz"))
    assert rd.n_paths == hw["n_links"] * hw["n_rd"]
    tg = I.TimeGrid(0.0, hw["dt"], hw["n_steps"])
    fgs = [I.FreqGrid(fc, hw["bandwidth"], hw["n_bins"]) for fc in hw["carriers"]]
    scenes, sets, links = [], [], []
    for l in range(hw["n_links"]):
        scenes.append(I.scene_highway(0, l))
        sets.append(I.highway_pathset(rd, l))
        links.append(ctx.load(scenes[-1], sets[-1]))
    entries = [(l, fg) for fg in fgs for l in range(hw["n_links"])]
    Hs = [torch.empty((tg.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda") for _, fg in entries]
    with ctx.batch([links[l] for l, _ in entries], [tg] * len(entries), [fg for _, fg in entries], Hs) as b:
        b.run(use_graph=True)
        torch.cuda.synchronize()
        redo = b.info(redo=True)["redo_steps"]
    total = len(entries) * tg.n_steps * sets[0].n_paths
    assert redo < 1e-3 * total, (redo, total)
    rng = np.random.default_rng(11)
    for k, (l, fg) in enumerate(entries):
        if l not in (0, 31, 63):
            continue
        rows = np.unique(np.concatenate([[0, tg.n_steps - 1], rng.integers(0, tg.n_steps, 2)]))
        Hg = Hs[k][torch.as_tensor(rows, device="cuda")].cpu().numpy()
        assert np.isfinite(Hg).all()
        for j, t in enumerate(rows):
            r = O.extrapolate(scenes[l], sets[l], I.TimeGrid(t * tg.dt, tg.dt, 1), fg.fc, n_threads=16)
            compare_H_band(Hg[j:j + 1], r, fg)
    del Hs
    for lk in links:
        lk.unload()
