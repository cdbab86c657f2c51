"""The stream form of the registration call (turboreg_register_async): the
same results as the synchronous call, enqueued back to back."""
import re

import numpy as np
import pytest

import paper_2507_01439_gb300 as trg
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_01439_gb300 import build
    build.build()
    c = trg.TurboReg(max_n=5000, max_batch=1)
    yield c
    c.close()


def _same(a, b):
    assert a.status == b.status and a.hypothesis == b.hypothesis and a.clique == b.clique
    assert np.array_equal(a.R, b.R) and np.array_equal(a.t, b.t)
    assert a.inlier_count == b.inlier_count and a.n_pivots == b.n_pivots and a.n_valid == b.n_valid


def test_async_device_inputs_match_sync(ctx):
    import torch
    probs = [synth.make_problem(s, n, r, 300 + k) for k, (s, n, r) in
             enumerate([("indoor", 5000, 0.05), ("indoor", 5000, 0.05), ("outdoor", 2500, 0.2),
                        ("cube", 777, 0.1), ("indoor", 5000, 0.05)])]
    prm = [trg.default_params(p.tau, min(2000, 2 * p.n), p.theta) for p in probs]
    dev = [(torch.from_numpy(p.x).cuda(), torch.from_numpy(p.y).cuda()) for p in probs]
    torch.cuda.synchronize()
    slots = trg.ResultSlots(len(probs))
    for k, (dx, dy) in enumerate(dev):      # mixed shapes: graphs captured between queued launches
        ctx.register_async(dx, dy, prm[k], slots, k)
    ctx.synchronize()
    for k, p in enumerate(probs):
        _same(slots.result(k), ctx.register(p.x, p.y, prm[k]))


def test_async_pinned_host_inputs_match_sync(ctx):
    import torch
    probs = [synth.make_problem("indoor", 4000, 0.05, 310 + k) for k in range(3)]
    prm = trg.default_params(probs[0].tau, 1500, probs[0].theta)
    pinned = [(torch.from_numpy(p.x).pin_memory(), torch.from_numpy(p.y).pin_memory()) for p in probs]
    slots = trg.ResultSlots(3)
    for k, (hx, hy) in enumerate(pinned):
        ctx.register_async(hx, hy, prm, slots, k)
    ctx.synchronize()
    for k, p in enumerate(probs):
        _same(slots.result(k), ctx.register(p.x, p.y, prm))


def test_reused_buffers_and_result_slots(ctx):
    """The replayed graph keeps the input and result pointers of its last call
    and patches them only when they change: the same buffers refilled, and
    buffers and result slots alternating, give what a fresh context gives."""
    import torch
    probs = [synth.make_problem("indoor", 4000, 0.05, 320 + k) for k in range(3)]
    prm = trg.default_params(probs[0].tau, 1500, probs[0].theta)
    ref = []
    for p in probs:
        with trg.TurboReg(max_n=5000, max_batch=1) as fresh:
            ref.append(fresh.register(p.x, p.y, prm))
    bx = [torch.empty((4000, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    by = [torch.empty((4000, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    slots = trg.ResultSlots(2)
    # one buffer pair and one result slot, refilled for every problem
    for k, p in enumerate(probs):
        bx[0].copy_(torch.from_numpy(p.x)); by[0].copy_(torch.from_numpy(p.y))
        torch.cuda.synchronize()
        ctx.register_async(bx[0], by[0], prm, slots, 0)
        ctx.synchronize()
        _same(slots.result(0), ref[k])
        _same(ctx.register(bx[0], by[0], prm), ref[k])        # the synchronous call on the same buffers
    # buffers and slots alternating: A, B, A
    order = [0, 1, 2]
    for k in order:
        b = k % 2
        bx[b].copy_(torch.from_numpy(probs[k].x)); by[b].copy_(torch.from_numpy(probs[k].y))
        torch.cuda.synchronize()
        ctx.register_async(bx[b], by[b], prm, slots, b)
        ctx.synchronize()
        _same(slots.result(b), ref[k])
    # host inputs staged through the workspace (the same staging pointer every call)
    for k, p in enumerate(probs):
        _same(ctx.register(p.x, p.y, prm), ref[k])


def test_async_rejections(ctx):
    import torch
    p = synth.make_problem("cube", 300, 0.2, 320)
    prm = trg.default_params(p.tau, 100, p.theta)
    slots = trg.ResultSlots(1)
    with pytest.raises(RuntimeError, match=re.escape(trg.status_string(trg.ERR_INVALID_ARG))):          # pageable host inputs
        ctx.register_async(p.x, p.y, prm, slots, 0)
    hx, hy = torch.from_numpy(p.x).pin_memory(), torch.from_numpy(p.y).pin_memory()
    with pytest.raises(RuntimeError, match=re.escape(trg.status_string(trg.ERR_TOO_FEW))):
        ctx.register_async(hx[:2].contiguous().pin_memory(), hy[:2].contiguous().pin_memory(), prm, slots, 0)
    learned = trg.default_params(p.tau, 100, p.theta)
    learned.proposal = trg.PROPOSAL_LEARNED
    with pytest.raises(RuntimeError, match=re.escape(trg.status_string(trg.ERR_INVALID_ARG))):
        ctx.register_async(hx, hy, learned, slots, 0)
    bad = p.x.copy(); bad[3, 0] = np.inf
    with pytest.raises(RuntimeError, match=re.escape(trg.status_string(trg.ERR_NONFINITE))):
        ctx.register_async(torch.from_numpy(bad).pin_memory(), hy, prm, slots, 0)
    # the context still works
    ctx.register_async(hx, hy, prm, slots, 0)
    ctx.synchronize()
    _same(slots.result(0), ctx.register(p.x, p.y, prm))


def test_async_nonfinite_device_input_reported_in_result(ctx):
    import torch
    p = synth.make_problem("cube", 500, 0.2, 321)
    x = p.x.copy(); x[7, 2] = np.nan
    slots = trg.ResultSlots(1)
    ctx.register_async(torch.from_numpy(x).cuda(), torch.from_numpy(p.y).cuda(),
                       trg.default_params(p.tau, 100, p.theta), slots, 0)
    ctx.synchronize()
    assert slots.result(0).status == trg.ERR_NONFINITE
