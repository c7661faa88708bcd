"""Tracing on the GPU: the launch-group timeline against the per-kind totals of the same record."""
import os

import pytest

from paper_2205_00237_gb300 import inputs as I

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


@pytest.mark.parametrize("form", ["fp64", "fp32_bulk"])
def test_timeline_matches_profile(ctx, form):
    import torch
    from paper_2205_00237_gb300 import drt
    prec = drt.FP64 if form == "fp64" else drt.FP32_BULK
    sc, ps = I.scene_canyon(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))
    tg, fg = I.grids("canyon", n_steps=300, n_bins=64)
    link = ctx.load(sc, ps)
    H = torch.empty((tg.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda")
    link.synthesize_H(tg, fg, prec, H)   # warm-up: scratch allocations outside the record
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()
    link.synthesize_H(tg, fg, prec, H)
    tl = ctx.profile_timeline()
    prof = ctx.profile_read()   # the same record, then cleared
    ctx.profile(False)
    assert ctx.profile_timeline() == []
    # one entry per bracketed group, the kinds and summed durations of the per-kind read
    assert len(tl) == sum(n for n, _ in prof.values())
    for name, (n, ms) in prof.items():
        mine = [t1 - t0 for k, t0, t1 in tl if k == name]
        assert len(mine) == n
        # each difference of two event times may round by the events' resolution (~0.5 us)
        assert abs(sum(mine) - ms) <= 1e-3 * ms + 2e-3 * n
    assert tl[0][1] == 0.0
    # groups on other streams may start a few microseconds before the first one's opening event
    assert all(t1 >= t0 > -0.05 for _, t0, t1 in tl)
    # on the launch stream the synthesis follows the extrapolation
    ext = [t1 for k, _, t1 in tl if k == "extrapolate"]
    syn = [t0 for k, t0, _ in tl if k == "synth"]
    assert ext and syn and min(syn) >= max(ext) - 1e-6
    link.unload()
