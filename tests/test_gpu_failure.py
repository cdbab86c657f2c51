"""Failure paths of the runtime, exercised without faulting the GPU.

  bounded wait   TURBOREG_FLAG_DEBUG_STALL_COMPAT makes every compatibility
                 block skip the copy of its row points, so its mbarrier wait
                 (bounded at 20 ms under the hook) can only expire: the
                 registration must report TURBOREG_ERR_TIMEOUT, and the
                 context must stay usable (the next registration equals a
                 fresh context's).
  allocation     TURBOREG_DEBUG_FAIL_ALLOC=k fails the k-th allocation of
                 turboreg_create: every k must give TURBOREG_ERR_OOM and
                 leave no device memory behind.
"""
import ctypes
import os

import numpy as np
import pytest

import paper_2507_01439_gb300 as trg
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_01439_gb300 import build
    build.build()


def _same(a, b):
    return (a.status == b.status and a.hypothesis == b.hypothesis and a.inlier_count == b.inlier_count
            and np.array_equal(a.R, b.R) and np.array_equal(a.t, b.t) and a.n_pivots == b.n_pivots)


@pytest.mark.parametrize("no_graph", [False, True])
def test_expired_wait_reports_timeout_and_context_recovers(no_graph):
    p = synth.make_problem("indoor", 3000, 0.05, 5)
    flags = trg.FLAG_NO_GRAPH if no_graph else 0
    prm = trg.default_params(p.tau, 1000, p.theta, flags=flags)
    stall = trg.default_params(p.tau, 1000, p.theta, flags=flags | trg.FLAG_DEBUG_STALL_COMPAT)
    with trg.TurboReg(max_n=3000) as fresh:
        ref = fresh.register(p.x, p.y, prm)
    assert ref.status == trg.OK
    with trg.TurboReg(max_n=3000) as ctx:
        before = ctx.register(p.x, p.y, prm)
        bad = ctx.register(p.x, p.y, stall)
        assert bad.status == trg.ERR_TIMEOUT
        assert bad.hypothesis == -1 and bad.inlier_count == 0
        # the adjacency of the timed-out call is empty (its tiles were left clear)
        assert not ctx.buffer(trg.BUF_ADJ_BITS).any()
        after = ctx.register(p.x, p.y, prm)
        again = ctx.register(p.x, p.y, stall)            # a second expiry after a good call
        last = ctx.register(p.x, p.y, prm)
    assert again.status == trg.ERR_TIMEOUT
    assert _same(before, ref) and _same(after, ref) and _same(last, ref)


def test_expired_wait_in_a_batch():
    probs = [synth.make_problem("indoor", 1500, 0.05, 40 + b) for b in range(3)]
    offs = np.cumsum([0] + [q.n for q in probs]).astype(np.int64)
    xs = np.concatenate([q.x for q in probs])
    ys = np.concatenate([q.y for q in probs])
    prm = [trg.default_params(q.tau, 500, q.theta) for q in probs]
    stall = [trg.default_params(q.tau, 500, q.theta, flags=trg.FLAG_DEBUG_STALL_COMPAT) for q in probs]
    with trg.TurboReg(max_n=1500, max_batch=3) as ctx:
        ref = ctx.register_batched(xs, ys, offs, prm)
        bad = ctx.register_batched(xs, ys, offs, stall)
        after = ctx.register_batched(xs, ys, offs, prm)
    assert all(r.status == trg.OK for r in ref)
    assert all(r.status == trg.ERR_TIMEOUT for r in bad)
    assert all(_same(a, b) for a, b in zip(ref, after))


def test_every_failed_allocation_returns_oom_without_leak():
    import torch
    torch.cuda.init()
    max_n = 5000
    with trg.TurboReg(max_n=max_n):                      # warm the runtime (module load, attributes)
        pass
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    lib = trg.load_library()
    fails = 0
    try:
        for k in range(1, 64):
            os.environ["TURBOREG_DEBUG_FAIL_ALLOC"] = str(k)
            h = ctypes.c_void_p()
            rc = lib.turboreg_create(0, max_n, 1, None, ctypes.byref(h))
            if rc != trg.OK:
                assert rc == trg.ERR_OOM, f"allocation {k}: status {rc}"
                assert not h.value, "no context is returned on failure"
                fails += 1
                free, _ = torch.cuda.mem_get_info()
                assert free >= free0 - (4 << 20), f"allocation {k}: {(free0 - free) >> 20} MB not freed"
                continue
            lib.turboreg_destroy(h)                      # k beyond the number of allocations
            break
        else:
            pytest.fail("turboreg_create never completed")
    finally:
        os.environ.pop("TURBOREG_DEBUG_FAIL_ALLOC", None)
    assert fails >= 20                                   # every workspace buffer was tried
    with trg.TurboReg(max_n=max_n) as ctx:               # and creation works again
        p = synth.make_problem("cube", 1000, 0.1, 3)
        assert ctx.register(p.x, p.y, trg.default_params(p.tau, 300, p.theta)).status == trg.OK
    del lib
