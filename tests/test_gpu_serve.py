"""The serving loop (drt_submit / drt_poll / drt_wait): continuous batching of prediction requests.

Each served result must be the same whether the request ran alone or in a mix with others (within
1e-6 of the row RMS: the only batch-dependent step is the order of the FP64 redo additions), must
match the FP64 oracle within the FP32-bulk bars, and the loop must keep its contracts: records when
asked, admission by arena size (a request larger than the arena fails with DRT_ENOMEM, others
queue until memory frees up), bounded waits, no unloading of a link with pending requests.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2205_00237_gb300 import inputs as I

from test_gpu_parity import compare_H_band

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture()
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    c = drt.Context(0, hbm_budget=8 << 30)
    yield c
    c.close()


def canyon():
    return I.scene_canyon(0), I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))


def requests(seed, n, links):
    """n requests over the loaded links: horizons U{50..500} x 1 ms from t_start U[0, 0.5] s, 512 bins."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        li = int(rng.integers(len(links)))
        T = int(rng.integers(50, 501))
        out.append((li, I.TimeGrid(float(rng.integers(0, 500)) * 1e-3, 1e-3, T), I.FreqGrid(60e9, 1e9, 512)))
    return out


def test_alone_equals_in_mix_and_matches_oracle(ctx):
    import torch
    sc, ps = canyon()
    links = [ctx.load(sc, ps), ctx.load(sc, ps.subset(np.arange(100))), ctx.load(sc, ps.subset(np.arange(7)))]
    reqs = requests(1, 24, links)
    ctx.serve_start(pool_bytes=2 << 30, n_slots=3, max_batch=8)
    alone = []
    for li, tg, fg in reqs:
        H = torch.full((tg.n_steps, fg.n_bins), float("nan"), dtype=torch.complex64, device="cuda")
        res = ctx.wait(ctx.submit(links[li], tg, fg, H))
        assert res["status"] == 0 and res["batch_requests"] == 1
        alone.append(H.cpu().numpy())
    # the same requests submitted at once, in another order: batched and overlapped
    mix = [None] * len(reqs)
    tickets = []
    for i in np.random.default_rng(2).permutation(len(reqs)):
        li, tg, fg = reqs[i]
        mix[i] = torch.full((tg.n_steps, fg.n_bins), float("nan"), dtype=torch.complex64, device="cuda")
        tickets.append(ctx.submit(links[li], tg, fg, mix[i]))
    sizes = [ctx.wait(t)["batch_requests"] for t in tickets]
    assert max(sizes) > 1
    st = ctx.serve_stats()
    assert st["completed"] == st["submitted"] == 2 * len(reqs) and st["queued"] == 0
    for a, m in zip(alone, mix):
        m = m.cpu().numpy()
        rms = np.sqrt(np.mean(np.abs(a) ** 2, axis=1, keepdims=True)) + 1e-30
        assert (np.abs(m - a) / rms).max() < 1e-6
    # against the oracle: two requests in full
    subsets = [ps, ps.subset(np.arange(100)), ps.subset(np.arange(7))]
    for i in (0, 1):
        li, tg, fg = reqs[i]
        r = O.extrapolate(sc, subsets[li], tg, fg.fc, n_threads=8)
        compare_H_band(alone[i], r, fg)
    ctx.serve_stop()
    for lk in links:
        lk.unload()


def test_records_and_contracts(ctx):
    import torch
    from paper_2205_00237_gb300 import drt
    from test_gpu_parity import compare_records_bulk
    sc, ps = canyon()
    sub = ps.subset(np.arange(64))
    link = ctx.load(sc, sub)
    tg, fg = I.TimeGrid(0.2, 1e-3, 120), I.FreqGrid(60e9, 1e9, 512)
    T, P = tg.n_steps, sub.n_paths
    rec = dict(tau=torch.empty((T, P), dtype=torch.float64, device="cuda"),
               amp=torch.empty((T, P, 2), dtype=torch.float32, device="cuda"),
               doppler=torch.empty((T, P), dtype=torch.float32, device="cuda"),
               angles=torch.empty((T, P, 4), dtype=torch.float32, device="cuda"),
               flags=torch.empty((T, P), dtype=torch.uint8, device="cuda"))
    H = torch.empty((T, fg.n_bins), dtype=torch.complex64, device="cuda")
    t = ctx.submit(link, tg, fg, H, records=rec)
    while ctx.poll(t) is None:
        pass
    with pytest.raises(drt.DrtError) as ei:
        ctx.poll(t)                               # retired once its result was returned
    assert ei.value.code == drt.DRT_ENOTFOUND
    r = O.extrapolate(sc, sub, tg, fg.fc, n_threads=8)
    compare_records_bulk(rec, r, fg.fc)
    compare_H_band(H.cpu().numpy(), r, fg)
    # unloading a link with pending requests is refused; a bounded wait reports DRT_ETIMEOUT
    big = ctx.load(sc, ps)
    tgb = I.TimeGrid(0.0, 0.5e-3, 2000)
    Hb = [torch.empty((tgb.n_steps, 512), dtype=torch.complex64, device="cuda") for _ in range(6)]
    tk = [ctx.submit(big, tgb, fg, h) for h in Hb]
    with pytest.raises(drt.DrtError) as ei:
        big.unload()
    assert ei.value.code == drt.DRT_EBUSY
    try:
        ctx.wait(tk[-1], timeout_ms=0)
    except drt.DrtError as e:
        assert e.code == drt.DRT_ETIMEOUT
    for x in tk:
        ctx.wait(x)
    big.unload()
    link.unload()


def test_request_larger_than_the_arena_fails_cleanly():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    sc, ps = canyon()
    with drt.Context(0) as ctx:
        link = ctx.load(sc, ps)
        ctx.serve_start(pool_bytes=2 << 20, n_slots=2, max_batch=4)
        fg = I.FreqGrid(60e9, 1e9, 64)
        small, large = I.TimeGrid(0.0, 1e-3, 8), I.TimeGrid(0.0, 1e-3, 2000)
        Hs = torch.empty((8, 64), dtype=torch.complex64, device="cuda")
        Hl = torch.empty((2000, 64), dtype=torch.complex64, device="cuda")
        t1, t2 = ctx.submit(link, large, fg, Hl), ctx.submit(link, small, fg, Hs)
        assert ctx.wait(t1)["status"] == drt.DRT_ENOMEM
        assert ctx.wait(t2)["status"] == 0
        r = O.extrapolate(sc, ps, small, fg.fc, n_threads=8)
        compare_H_band(Hs.cpu().numpy(), r, fg)
        ctx.serve_stop()
        link.unload()


def test_redo_list_overflow_is_reported(monkeypatch):
    """A batch whose FP64 redo list is too small for the steps FP32 could not resolve leaves their
    contributions out of H: drt_batch_info says so (DRT_ENOMEM) and the serving loop marks every
    request of such a batch DRT_ENOMEM instead of DRT_OK.  The list is shrunk to one entry through
    DRT_BATCH_REDO_CAP (a host-side setting read when a plan is built); with the default list the
    same request is served with DRT_OK."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    sc, ps = canyon()
    tg, fg = I.TimeGrid(0.0, 1e-3, 400), I.FreqGrid(60e9, 1e9, 128)
    with drt.Context(0) as ctx:
        link = ctx.load(sc, ps)
        H = torch.empty((tg.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda")
        ctx.serve_start(pool_bytes=1 << 30, n_slots=2, max_batch=4)
        res = ctx.wait(ctx.submit(link, tg, fg, H))
        assert res["status"] == 0
        ctx.serve_stop()
        monkeypatch.setenv("DRT_BATCH_REDO_CAP", "1")
        with ctx.batch([link], [tg], [fg], [H]) as b:
            b.run(use_graph=False)
            with pytest.raises(drt.DrtError) as ei:
                b.info(redo=True)
            assert ei.value.code == drt.DRT_ENOMEM
        ctx.serve_start(pool_bytes=1 << 30, n_slots=2, max_batch=4)
        res = ctx.wait(ctx.submit(link, tg, fg, H))
        assert res["status"] == drt.DRT_ENOMEM
        ctx.serve_stop()
        link.unload()
