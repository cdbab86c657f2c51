"""Runtime behaviour of the C ABI around the kernels: page-locked host inputs
read in place by the first kernel, the per-slot control block that the
finalize kernel leaves cleared for the next registration (and that the host
clears after entry points running only part of the path), and a single
problem at the largest size whose edge-weight histogram the GEMM still keeps
in shared memory (the count pass then stages that histogram too)."""
import numpy as np
import pytest

import paper_2507_01439_gb300 as trg
import synth
from test_gpu_maxsize import _check_large

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_01439_gb300 import build
    build.build()
    c = trg.TurboReg(max_n=5000, max_batch=4)
    yield c
    c.close()


def _same(a, b):
    assert a.status == b.status
    assert a.hypothesis == b.hypothesis and a.inlier_count == b.inlier_count
    assert np.array_equal(a.R, b.R) and np.array_equal(a.t, b.t)


def test_page_locked_inputs_equal_pageable_and_device(ctx):
    import torch
    p = synth.make_problem("indoor", 4000, 0.05, 901)
    prm = trg.default_params(p.tau, 1500, p.theta)
    r_pageable = ctx.register(p.x, p.y, prm)
    xp = torch.from_numpy(p.x).pin_memory()
    yp = torch.from_numpy(p.y).pin_memory()
    r_pinned = ctx.register(xp, yp, prm)
    xd, yd = xp.cuda(), yp.cuda()
    torch.cuda.synchronize()
    r_device = ctx.register(xd, yd, prm)
    assert r_pageable.status == 0
    _same(r_pinned, r_pageable)
    _same(r_device, r_pageable)
    # one page-locked side, one device side
    _same(ctx.register(xp, yd, prm), r_pageable)
    # a non-finite page-locked coordinate is rejected before any launch
    xbad = xp.clone().pin_memory()
    xbad[11, 0] = float("nan")
    assert ctx.register(xbad, yp, prm).status == trg.ERR_NONFINITE
    _same(ctx.register(xp, yp, prm), r_pageable)


def test_registrations_clean_after_partial_entry_points(ctx):
    import torch
    p = synth.make_problem("indoor", 3000, 0.05, 902)
    prm = trg.default_params(p.tau, 1000, p.theta)
    ref = ctx.register(p.x, p.y, prm)
    assert ref.status == 0
    # the feature entry point runs the first stages only; a non-finite device
    # coordinate sets the error bits of the control block it shares
    xd = torch.from_numpy(p.x).cuda()
    yd = torch.from_numpy(p.y).cuda()
    yd[5, 1] = float("nan")
    torch.cuda.synchronize()
    with pytest.raises(RuntimeError):
        ctx.features(xd, yd, prm)
    _same(ctx.register(p.x, p.y, prm), ref)
    # clique Kabsch and transform scoring entry points in between
    idx = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    ctx.kabsch_cliques(p.x, p.y, idx)
    rt = np.zeros((2, 12), dtype=np.float32)
    rt[:, [0, 4, 8]] = 1.0
    ctx.score_transforms(p.x, p.y, prm, rt)
    _same(ctx.register(p.x, p.y, prm), ref)
    # a registration whose input is non-finite on the device, then a clean one
    bad = ctx.register(xd, yd, prm)
    assert bad.status == trg.ERR_NONFINITE
    _same(ctx.register(p.x, p.y, prm), ref)
    # batched calls share the slots' control blocks too
    out = ctx.register_batched(np.concatenate([p.x, p.x]), np.concatenate([p.y, p.y]),
                               np.array([0, p.n, 2 * p.n]), prm)
    for r in out:
        _same(r, ref)
    _same(ctx.register(p.x, p.y, prm), ref)


def test_histogram_at_shared_memory_limit():
    # 8500 matches: 8501 bins still fit beside the GEMM's pipeline (the limit is
    # 8576), so the GEMM keeps them in shared memory and the count blocks stage
    # all of them to choose the threshold
    _check_large(8500, 703, k1=1500, samples=300)


def test_batched_many_small_problems_equal_plain():
    # 64 problems of 50..400 matches: one or a few GEMM blocks each, so the
    # GEMM's CTAs move between problems at almost every block and flush their
    # shared-memory histograms each time
    probs = synth.make_batch(64, seed=905, n_lo=50, n_hi=400)
    c = trg.TurboReg(max_n=400, max_batch=64)
    try:
        params = [trg.default_params(p.tau, min(p.k1, 300), p.theta) for p in probs]
        offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
        out = c.register_batched(np.concatenate([p.x for p in probs]), np.concatenate([p.y for p in probs]),
                                 offs, params)
        for p, prm, rb in zip(probs, params, out):
            rp = c.register(p.x, p.y, prm)
            assert rb.n_pivots == rp.n_pivots, (p.n, p.shape)
            _same(rb, rp)
    finally:
        c.close()
