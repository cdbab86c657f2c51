"""The allocation-free pivot selection (turboreg_select_pivots_noalloc).

It serves callers that cannot call cudaMalloc (a plugin inside a framework
that owns all device memory, a real-time loop that forbids allocation after
start-up).  Its results must equal the pivots the regular registration path
computes from the same weight matrix, on consecutive calls that share the
entry point's one fixed scratch array: a large problem first, then a smaller
one, so stale scratch contents from the first call would show in the second.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import paper_2507_01439_gb300 as trg
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_01439_gb300 import build
    build.build()
    c = trg.TurboReg(max_n=5000)
    yield c
    c.close()


def test_noalloc_pivots_equal_register_path(ctx):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    cases = [("indoor", 5000, 0.05, 71, 2000), ("cube", 1500, 0.10, 72, 700), ("cube", 1500, 0.10, 72, 700)]
    for shape, n, ratio, seed, k1 in cases:
        p = synth.make_problem(shape, n, ratio, seed)
        res = ctx.register(p.x, p.y, trg.default_params(p.tau, k1, p.theta))
        assert res.status == 0
        W = ctx.buffer(trg.BUF_SC2)                 # uint16 [n_pad, n_pad], weights above the diagonal
        want = ctx.buffer(trg.BUF_PIVOTS)           # int32 [|P|, 4] from the regular path
        w_dev = torch.from_numpy(W.view(np.int16)).to(dev)
        piv = torch.full((k1, 4), -7, dtype=torch.int32, device=dev)
        npiv = torch.full((1,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        rc = trg.turboreg_select_pivots_noalloc(w_dev, n, W.shape[1], k1, piv, npiv, stream.cuda_stream)
        assert rc == trg.OK
        torch.cuda.synchronize()
        m = int(npiv.item())
        assert m == res.n_pivots == want.shape[0]
        got = piv[:m].cpu().numpy()
        assert np.array_equal(got, want), np.argwhere(got != want)[:5]
        assert (piv[m:].cpu().numpy() == -7).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2507_01439_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    big = trg.TURBOREG_NOALLOC_MAX_N + 8
    w = torch.zeros((8, big), dtype=torch.int16, device=dev)
    piv = torch.zeros((16, 4), dtype=torch.int32, device=dev)
    npiv = torch.zeros(1, dtype=torch.int32, device=dev)
    assert trg.turboreg_select_pivots_noalloc(w, big, big, 16, piv, npiv) == trg.ERR_INVALID_ARG
    assert trg.turboreg_select_pivots_noalloc(w, 8, big, trg.TURBOREG_K1_MAX + 1, piv, npiv) == trg.ERR_INVALID_ARG
    assert trg.turboreg_select_pivots_noalloc(w, 8, 7, 4, piv, npiv) == trg.ERR_INVALID_ARG
