"""GPU checks of the batched-form autotuner: every tile shape gives the same
results, and a tuned schedule reaches the best success rate of its
candidates with batched results equal to single calls."""
import numpy as np
import pytest

import paper_2507_01439_gb300 as trg
import synth
from paper_2507_01439_gb300 import autotune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_01439_gb300 import build
    build.build()
    c = trg.TurboReg(max_n=3000, max_batch=32)
    yield c
    c.close()


def _calib(probs):
    return [autotune.Calib(p.x, p.y, p.R_gt, p.t_gt, p.tau, p.theta, p.re_deg, p.te_m) for p in probs]


def test_tile_shapes_give_identical_results(ctx):
    probs = synth.make_batch(12, seed=31, n_lo=300, n_hi=2500, ratio_lo=0.03, ratio_hi=0.2)
    offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
    xs = np.concatenate([p.x for p in probs])
    ys = np.concatenate([p.y for p in probs])
    ref = None
    for name, fl in autotune.TILE_CANDIDATES.items():
        prm = [trg.default_params(p.tau, 500, p.theta, flags=fl, scoring=trg.SCORE_MSE if b % 3 == 0 else 0)
               for b, p in enumerate(probs)]
        out = ctx.register_batched(xs, ys, offs, prm)
        got = [(r.status, r.hypothesis, r.clique, r.inlier_count, r.score, r.R.tobytes(), r.t.tobytes())
               for r in out]
        if ref is None:
            ref = got
        assert got == ref, name


def test_tuned_schedule(ctx):
    calib = _calib(synth.make_batch(24, seed=32, n_lo=500, n_hi=2500, ratio_lo=0.02, ratio_hi=0.2))
    tiles = {k: autotune.TILE_CANDIDATES[k] for k in ("sc2_pair+verify256", "sc2_single+verify512")}
    sched = autotune.tune(ctx, calib, k1_candidates=(20, 100, 500), bucket_edges=(1500, 2500), tiles=tiles,
                          reps=2, log=print)
    assert sched.tile in tiles and sched.flags == tiles[sched.tile]
    assert all(k in (20, 100, 500) for _, _, k in sched.k1_rules)
    # on the calibration set the schedule reaches each class's best success count
    offs = np.cumsum([0] + [c.x.shape[0] for c in calib]).astype(np.int64)
    xs = np.concatenate([c.x for c in calib])
    ys = np.concatenate([c.y for c in calib])
    prm = [sched.params(c.x.shape[0], c.tau, c.theta) for c in calib]
    out = ctx.register_batched(xs, ys, offs, prm)
    ok = sum(autotune._success(r, c) for r, c in zip(out, calib))
    best = sum(max(v.values()) for v in sched.success.values())
    assert ok == best
    # batched with the schedule's parameters = single calls
    for c, p, rb in zip(calib[:6], prm[:6], out[:6]):
        rs = ctx.register(c.x, c.y, p)
        assert rb.hypothesis == rs.hypothesis and rb.inlier_count == rs.inlier_count
        assert np.array_equal(rb.R, rs.R) and np.array_equal(rb.t, rs.t)
    # JSON round trip keeps the decisions
    again = autotune.Schedule.from_json(sched.to_json())
    assert [again.k1_for(c.x.shape[0], c.tau) for c in calib] == [sched.k1_for(c.x.shape[0], c.tau) for c in calib]
