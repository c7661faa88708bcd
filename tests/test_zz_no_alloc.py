"""The allocation-free synthesis entry point (drt_synthesize_H_noalloc) against drt_synthesize_H.

Callers that cannot allocate device memory when they ask for a prediction (a latency-bound
prediction loop that must not stall in cudaMalloc / cudaFree, or a process whose device memory is
reserved by another allocator) use the variant whose scratch is a static 32 MiB device array.  This
file is collected last so that a run stopping at the first failure has run every other test first.
"""
import os

import numpy as np
import pytest

from paper_2205_00237_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_noalloc_matches_allocating_entry_point_twice():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt

    scene = I.scene_canyon(0)
    paths = I.PathSet.from_npz(os.path.join(GOLD, "pathset_canyon_seed0.npz"))
    tg, fg = I.grids("canyon")        # 512 paths x 2000 steps: 23 MB of the 32 MiB array
    with drt.Context(0) as ctx:
        link = ctx.load(scene, paths)
        ref = link.synthesize_H(tg, fg, drt.FP64).cpu().numpy()
        rms = np.sqrt(np.mean(np.abs(ref) ** 2, axis=1, keepdims=True))
        for call in range(2):
            H = torch.full((tg.n_steps, fg.n_bins), float("nan"), dtype=torch.complex64, device="cuda")
            link.synthesize_H_noalloc(tg, fg, H, drt.FP64)
            torch.cuda.synchronize()
            got = H.cpu().numpy()
            assert np.isfinite(got).all(), call
            err = np.abs(got.astype(np.complex128) - ref) / rms
            assert err.max() < 1e-4, (call, err.max())
        # a second link on the same array gives its own result (the array keeps no state)
        tiny = ctx.load(I.scene_tiny(1), I.PathSet.from_npz(os.path.join(GOLD, "pathset_tiny_seed1.npz")))
        tg1, fg1 = I.grids("tiny")
        ref1 = tiny.synthesize_H(tg1, fg1, drt.FP64).cpu().numpy()
        H1 = torch.empty((tg1.n_steps, fg1.n_bins), dtype=torch.complex64, device="cuda")
        tiny.synthesize_H_noalloc(tg1, fg1, H1, drt.FP64)
        torch.cuda.synchronize()
        rms1 = np.sqrt(np.mean(np.abs(ref1) ** 2, axis=1, keepdims=True))
        assert (np.abs(H1.cpu().numpy().astype(np.complex128) - ref1) / rms1).max() < 1e-4
        # beyond the static array the call is refused with a clear error, before any device work
        big = I.TimeGrid(0.0, 0.5e-3, 4000)
        Hb = torch.empty((big.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda")
        with pytest.raises(drt.DrtError) as e:
            link.synthesize_H_noalloc(big, fg, Hb, drt.FP64)
        assert e.value.code == drt.DRT_EINVAL and "static array" in str(e.value)
        tiny.unload()
        link.unload()
