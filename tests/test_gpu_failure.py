"""Failure detection on the GPU: per-result conditions are flags, never faults or call errors.

A chain through two edges that meet at a box corner has no interior stationary point (the unfolded
length is not smooth where the two diffraction points meet), so the Newton solve of its segment
cannot converge: every path-step must carry DRT_F_NOCONV, in both forms (the FP32-bulk form hands the
step to its FP64 redo, which flags it), and H must not contain the chain: H of the link with the chain
equals H of the link without it.  The inputs are host-constructed and fault nothing.
"""
import numpy as np
import pytest

from paper_2205_00237_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def corner_scene():
    b = I._Builder("corner")
    metal = b.material(1.0, 0.0, pec=True)
    b.box(0, metal, [0, 0, 0], np.eye(3), (2.0, 2.0, 2.0), with_faces=False)
    tx = [0.49753464, -2.40345731, -0.92775335]
    rx = [-5.66016395, -4.50860068, 2.04749298]
    sc = b.build((tx, [0.3, 0.2, 0.1], [0, 0, 0]), (rx, [0, 0, 0], [0, 0, 0]))
    # edges 2 and 9 of the box both end at the corner (1, -1, 1)
    assert np.allclose(sc.edges[2]["a"], [1, -1, 1]) and np.allclose(sc.edges[9]["a"], [1, -1, 1])
    with_chain = I.chains_to_pathset([[], [(I.T_D, 2), (I.T_D, 9)]])
    with_chain.s0[1, :2] = 1.0
    return sc, with_chain


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_unconverged_newton_is_flagged_and_left_out_of_H(form):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt
    prec = drt.FP64 if form == "fp64" else drt.FP32_BULK
    sc, ps = corner_scene()
    tg, fg = I.TimeGrid(0.0, 0.01, 50), I.FreqGrid(3e9, 1e8, 64)
    with drt.Context(0) as ctx:
        both = ctx.load(sc, ps)
        los = ctx.load(sc, ps.subset([0]))
        rec = both.extrapolate(tg, fg, prec)
        torch.cuda.synchronize()
        flags = rec["flags"].cpu().numpy()
        assert (flags[:, 1] & drt.F_NOCONV).all()
        assert (flags[:, 0] == 0).all()
        H1 = both.synthesize_H(tg, fg, prec).cpu().numpy()
        H0 = los.synthesize_H(tg, fg, prec).cpu().numpy()
        assert np.array_equal(H1, H0)
        both.unload()
        los.unload()
