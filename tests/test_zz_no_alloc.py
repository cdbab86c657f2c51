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


def _packed_w(n, ldw, wmax, seed, density=0.6):
    """uint16 [n, ldw]: upper-triangle weights in 0..wmax (a few values, so
    that many edges tie at the threshold across rows), nonzero junk in the
    lower triangle, on the diagonal and past column n (ignored by contract)."""
    rng = np.random.default_rng(seed)
    W = rng.integers(1, 65536, size=(n, ldw), dtype=np.int64).astype(np.uint16)   # junk everywhere
    up = np.triu(np.ones((n, n), dtype=bool), 1)
    vals = rng.integers(0, wmax + 1, size=(n, n)) * (rng.random((n, n)) < density)
    W[:, :n][up] = vals[up].astype(np.uint16)
    S = np.zeros((n, n), dtype=np.int32)                      # what the oracle sees: the O2Graph
    S[up] = vals[up]
    return W, S


def _noalloc(W, n, k1):
    import torch
    dev = torch.device("cuda:0")
    w_dev = torch.from_numpy(W.view(np.int16).copy()).to(dev)
    piv = torch.full((k1, 4), -7, dtype=torch.int32, device=dev)
    npiv = torch.full((1,), -9, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    rc = trg.turboreg_select_pivots_noalloc(w_dev, n, W.shape[1], k1, piv, npiv,
                                            torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    return rc, int(npiv.item()), piv.cpu().numpy()


@pytest.mark.parametrize("n,k1,wmax,seed", [
    (1, 4, 0, 1), (2, 4, 0, 2), (9, 5, 7, 3), (9, 100, 7, 4),          # tiny n; k1 above the edge count
    (100, 300, 3, 5), (1003, 2000, 2, 6), (4097, 6000, 5, 7),          # heavy ties at the threshold
    (2500, 40000 // 8, 2498, 8),                                       # the full weight range 0..n-2
])
def test_noalloc_tightly_packed_junk_outside_triangle(n, k1, wmax, seed):
    import oracle
    ldw = (n + 7) // 8 * 8                                   # the tightest leading dimension allowed
    W, S = _packed_w(n, ldw, max(0, min(wmax, n - 2)), seed)
    opi, opj, opw = oracle.pivots(S, k1)
    rc, m, got = _noalloc(W, n, k1)
    assert rc == trg.OK
    assert m == len(opi)
    assert np.array_equal(got[:m, 0], opi) and np.array_equal(got[:m, 1], opj)
    assert np.array_equal(got[:m, 2], opw) and (got[:m, 3] == 0).all()
    assert (got[m:] == -7).all()


def test_noalloc_rejects_weight_above_n_minus_2_then_recovers():
    import oracle
    n, k1 = 600, 500
    ldw = (n + 7) // 8 * 8
    W, S = _packed_w(n, ldw, 20, 11)
    bad = W.copy()
    bad[3, 400] = 65535                                      # far beyond the n + 1 histogram bins
    rc, m, got = _noalloc(bad, n, k1)
    assert rc == trg.OK                                      # the values are only seen on the GPU
    assert m == -trg.ERR_INVALID_ARG
    assert (got == -7).all()                                 # nothing written
    bad = W.copy()
    bad[0, n - 1] = n - 1                                    # one above the largest SC^2 count
    rc, m, got = _noalloc(bad, n, k1)
    assert rc == trg.OK and m == -trg.ERR_INVALID_ARG and (got == -7).all()
    rc, m, got = _noalloc(W, n, k1)                          # the next valid call is unaffected
    opi, opj, opw = oracle.pivots(S, k1)
    assert rc == trg.OK and m == len(opi)
    assert np.array_equal(got[:m, :3], np.stack([opi, opj, opw], 1))
