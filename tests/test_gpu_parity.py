"""GPU parity of the CUDA registration path with the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle
import paper_2507_01439_gb300 as trg
import synth
from parity_util import (check_final, check_graph_stages, check_hypotheses, check_pivots_cliques,
                         oracle_stages)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2507_01439_gb300 import build
    build.build()
    c = trg.TurboReg(max_n=5000, max_batch=8)
    yield c
    c.close()


def _full_parity(ctx, p, k1, k2=2, flags=0, tau=None, theta=None):
    tau = p.tau if tau is None else tau
    theta = p.theta if theta is None else theta
    prm = trg.default_params(tau, k1, theta, k2=k2, flags=flags)
    res = ctx.register(p.x, p.y, prm)
    A, S, piv, cliq = oracle_stages(p.x, p.y, tau, k1, k2)
    n = p.n
    assert ctx.shape()[0] == n
    check_graph_stages(ctx, A, S, n)
    check_pivots_cliques(ctx, piv, cliq, k2)
    orc = oracle.register(p.x, p.y, tau, k1, theta, k2=k2)
    assert res.n_pivots == orc.n_pivots
    stats = check_hypotheses(ctx, p.x, p.y, theta, orc)
    if p.shape in ("cube", "indoor"):
        # room-scale coordinates: FP32 resolves the contract's 1e-5 m band, so no
        # inlier decision may differ outside it
        assert stats["outside_1e-5"] == 0, stats["mismatches"]
    assert res.n_valid == orc.n_valid
    kind = check_final(res, ctx, orc, p.x, p.y, theta)
    return res, orc, stats, kind


@pytest.mark.parametrize("flags", [0, trg.FLAG_SC2_GEMM, trg.FLAG_SC2_BITSET])
@pytest.mark.parametrize("n,seed", [(3, 1), (7, 2), (33, 3), (63, 11), (64, 12), (65, 13), (127, 4), (128, 5),
                                    (129, 6), (255, 7), (256, 8), (257, 9), (600, 10)])
def test_small_ragged_sizes(ctx, n, seed, flags):
    # dense enough to have edges at tiny N: generous tau on a small cube; the
    # default (the CUDA-core path at these sizes), the tensor-core GEMM
    # (128/256 tiles) and the bitset path forced
    p = synth.make_problem("cube", n, 0.5, seed, tau=0.3, theta=0.1)
    _full_parity(ctx, p, k1=min(200, 4 * n), k2=2, flags=flags)


def test_config_cube_1000(ctx):
    p = synth.make_problem("cube", 1000, 0.10, 0)
    res, orc, stats, kind = _full_parity(ctx, p, k1=1000)
    assert res.status == 0
    assert synth.rotation_error_deg(p.R_gt, res.R) < 15 and synth.translation_error(p.t_gt, res.t) < 0.3


def test_config_indoor_5000(ctx):
    p = synth.make_problem("indoor", 5000, 0.05, 0)
    res, orc, stats, kind = _full_parity(ctx, p, k1=2000)
    print("indoor-5000", stats, kind)
    assert res.status == 0
    assert synth.rotation_error_deg(p.R_gt, res.R) < 15 and synth.translation_error(p.t_gt, res.t) < 0.3


def test_config_outdoor_2500(ctx):
    p = synth.make_problem("outdoor", 2500, 0.20, 0)
    res, orc, stats, kind = _full_parity(ctx, p, k1=1000)
    print("outdoor-2500", stats, kind)
    assert res.status == 0
    assert synth.rotation_error_deg(p.R_gt, res.R) < 5 and synth.translation_error(p.t_gt, res.t) < 0.6


@pytest.mark.parametrize("k2", [1, 3, 5])
def test_k2_variants(ctx, k2):
    p = synth.make_problem("cube", 800, 0.2, 40 + k2)
    _full_parity(ctx, p, k1=300, k2=k2)


def test_k1_max(ctx):
    # K1 = K1_MAX: the clique search stages 8192 selected keys (64 KB of shared memory)
    p = synth.make_problem("indoor", 3000, 0.1, 45)
    _full_parity(ctx, p, k1=trg.TURBOREG_K1_MAX)


def test_k2_max(ctx):
    # K2 = K2_MAX: the generic clique-search variant (16 cliques per pivot)
    p = synth.make_problem("cube", 1200, 0.2, 46)
    _full_parity(ctx, p, k1=400, k2=trg.TURBOREG_K2_MAX)


@pytest.mark.parametrize("flags", [trg.FLAG_SC2_BITSET, trg.FLAG_SC2_GEMM])
@pytest.mark.parametrize("shape,n,k1", [("indoor", 3000, 1500), ("indoor", 5000, 2000), ("outdoor", 2500, 1000),
                                        ("cube", 1000, 1000)])
def test_forced_sc2_path_matches(ctx, shape, n, k1, flags):
    # each SC^2 path forced: AND + popcount over the bitset, and the pair-MMA
    # GEMM with the FP8 matrix from the compatibility kernel (same integers)
    p = synth.make_problem(shape, n, 0.05 if shape == "indoor" else 0.2, 11)
    _full_parity(ctx, p, k1=k1, flags=flags)


@pytest.mark.parametrize("shape,n", [("cube", 300), ("cube", 777), ("indoor", 3000), ("indoor", 5000)])
def test_single_cta_sc2_matches(ctx, shape, n):
    # the GEMM on independent CTAs (no 2-CTA pair MMAs) gives the same integers
    p = synth.make_problem(shape, n, 0.05, 17)
    _full_parity(ctx, p, k1=min(1500, 2 * n), flags=trg.FLAG_SC2_SINGLE_CTA)


@pytest.mark.parametrize("flags", [trg.FLAG_SC2_SINGLE_CTA, trg.FLAG_SC2_BITSET])
def test_sc2_forms_batched(ctx, flags):
    # batched form (global histogram): the other GEMM form equals the default (pair MMA) batched call
    probs = [synth.make_problem(s, n, r, 90 + b) for b, (s, n, r) in
             enumerate([("indoor", 1200, 0.1), ("outdoor", 900, 0.2), ("indoor", 3000, 0.05), ("cube", 257, 0.1)])]
    offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
    xs = np.concatenate([p.x for p in probs])
    ys = np.concatenate([p.y for p in probs])
    ref = ctx.register_batched(xs, ys, offs, [trg.default_params(p.tau, p.k1, p.theta) for p in probs])
    out = ctx.register_batched(xs, ys, offs, [trg.default_params(p.tau, p.k1, p.theta, flags=flags)
                                              for p in probs])
    for a, b in zip(ref, out):
        assert a.status == b.status and a.hypothesis == b.hypothesis and a.n_pivots == b.n_pivots
        assert np.array_equal(a.R, b.R) and np.array_equal(a.t, b.t) and a.inlier_count == b.inlier_count


@pytest.mark.parametrize("flags", [0, trg.FLAG_SC2_GEMM, trg.FLAG_SC2_SINGLE_CTA, trg.FLAG_SC2_BITSET])
def test_complete_graph_exactness(ctx, flags):
    # (the default chooses the GEMM here, on the FP8 operand expanded from the bitset)
    # tau huge: G is complete, every SC^2 entry is N-2 (largest integer the FP8 GEMM accumulates)
    p = synth.make_problem("cube", 5000, 0.1, 12)
    prm = trg.default_params(1e6, 50, 0.1, flags=flags)
    res = ctx.register(p.x, p.y, prm)
    n = p.n
    W = ctx.buffer(trg.BUF_SC2)[:n, :n]
    assert (W[np.triu_indices(n, 1)] == n - 2).all()
    P = ctx.buffer(trg.BUF_PIVOTS)
    # all edges tie: the first 50 in (i, j) order
    assert P[:, 0].tolist() == [0] * 50 and P[:, 1].tolist() == list(range(1, 51))
    assert (ctx.buffer(trg.BUF_ROWSCORE) == (n - 1) * (n - 2)).all()
    assert res.status == 0


def test_no_edges_gives_no_hypothesis(ctx):
    p = synth.make_problem("cube", 500, 0.1, 13)
    res = ctx.register(p.x, p.y, trg.default_params(0.0, 100, 0.1))
    assert res.status == trg.ERR_NO_HYPOTHESIS and res.n_pivots == 0
    assert np.array_equal(res.R, np.eye(3, dtype=np.float32)) and not res.t.any()


def test_fewer_edges_than_k1(ctx):
    p = synth.make_problem("cube", 400, 0.1, 14, tau=0.02)
    _full_parity(ctx, p, k1=8000)


def test_duplicate_and_collinear_points(ctx):
    p = synth.make_problem("cube", 300, 0.5, 15, sigma=0.0, tau=0.05)
    x, y = p.x.copy(), p.y.copy()
    inl = np.flatnonzero(p.inlier)
    x[inl[1]] = x[inl[0]]; y[inl[1]] = y[inl[0]]                 # duplicate match
    for k in range(2, 6):                                         # collinear inlier run
        x[inl[k]] = x[inl[0]] + k * (x[inl[20]] - x[inl[0]]) / 10
        y[inl[k]] = y[inl[0]] + k * (y[inl[20]] - y[inl[0]]) / 10
    q = synth.Problem(x, y, p.R_gt, p.t_gt, p.inlier, 0.05, 0.05, 300, 15, 0.3, "cube", 15)
    _full_parity(ctx, q, k1=300)


def test_invalid_inputs(ctx):
    p = synth.make_problem("cube", 100, 0.1, 16)
    prm = trg.default_params(0.1, 10, 0.1)
    assert ctx.register(p.x[:2], p.y[:2], prm).status == trg.ERR_TOO_FEW
    bad = p.x.copy(); bad[5, 1] = np.nan
    assert ctx.register(bad, p.y, prm).status == trg.ERR_NONFINITE
    assert ctx.register(p.x, p.y, trg.default_params(-1.0, 10, 0.1)).status == trg.ERR_INVALID_ARG
    assert ctx.register(p.x, p.y, trg.default_params(0.1, 0, 0.1)).status == trg.ERR_INVALID_ARG
    assert ctx.register(p.x, p.y, trg.default_params(0.1, 10, 0.0)).status == trg.ERR_INVALID_ARG
    big = synth.make_problem("cube", 5001, 0.1, 16)
    assert ctx.register(big.x, big.y, prm).status == trg.ERR_INVALID_ARG
    # the context still works afterwards
    assert ctx.register(p.x, p.y, trg.default_params(0.3, 50, 0.1)).status in (0, trg.ERR_NO_HYPOTHESIS)


def test_device_inputs_and_nonfinite_on_device(ctx):
    import torch
    p = synth.make_problem("indoor", 2000, 0.1, 17)
    prm = trg.default_params(p.tau, 500, p.theta)
    r_host = ctx.register(p.x, p.y, prm)
    xd = torch.from_numpy(p.x).cuda()
    yd = torch.from_numpy(p.y).cuda()
    torch.cuda.synchronize()
    r_dev = ctx.register(xd, yd, prm)
    assert r_dev.status == r_host.status == 0
    assert r_dev.hypothesis == r_host.hypothesis and np.array_equal(r_dev.R, r_host.R)
    yd[7, 2] = float("inf")
    torch.cuda.synchronize()
    assert ctx.register(xd, yd, prm).status == trg.ERR_NONFINITE


def test_deterministic_repeats(ctx):
    p = synth.make_problem("indoor", 5000, 0.05, 18)
    prm = trg.default_params(p.tau, 2000, p.theta)
    first = ctx.register(p.x, p.y, prm)
    IN0 = ctx.buffer(trg.BUF_INLIERS).copy()
    W0 = ctx.buffer(trg.BUF_SC2).copy()
    for _ in range(5):
        r = ctx.register(p.x, p.y, prm)
        assert r.hypothesis == first.hypothesis and np.array_equal(r.R, first.R)
        assert np.array_equal(ctx.buffer(trg.BUF_INLIERS), IN0)
    n = p.n
    iu = np.triu_indices(n, 1)
    assert np.array_equal(ctx.buffer(trg.BUF_SC2)[:n, :n][iu], W0[:n, :n][iu])


@pytest.mark.parametrize("n,tau,want", [(5000, 0.1, 1), (5000, 0.4, 2), (3000, 0.3, 2), (1500, 0.4, 1)])
def test_sc2_path_chosen_on_the_device(ctx, n, tau, want):
    # one problem without an SC^2 flag: the path is chosen on the device from N
    # and the edge count (CUDA-core on sparse graphs, the GEMM on dense ones, the
    # FP8 operand then expanded from the bitset); results and W equal both forced paths
    p = synth.make_problem("indoor", n, 0.05, 23)
    r = ctx.register(p.x, p.y, trg.default_params(tau, 1000, p.theta))
    assert ctx.sc2_path() == want
    W = ctx.buffer(trg.BUF_SC2)[:n, :n].copy()
    if want == 2 and n <= 3000:   # the expanded FP8 operand and every graph stage against the oracle
        A, S, _, _ = oracle_stages(p.x, p.y, tau, 1000, 2)
        check_graph_stages(ctx, A, S, n)
    iu = np.triu_indices(n, 1)
    for fl, path in ((trg.FLAG_SC2_GEMM, 2), (trg.FLAG_SC2_BITSET, 1)):
        rf = ctx.register(p.x, p.y, trg.default_params(tau, 1000, p.theta, flags=fl))
        assert ctx.sc2_path() == path
        assert rf.status == r.status and rf.hypothesis == r.hypothesis and rf.n_pivots == r.n_pivots
        assert np.array_equal(rf.R, r.R) and np.array_equal(rf.t, r.t) and rf.inlier_count == r.inlier_count
        assert np.array_equal(ctx.buffer(trg.BUF_SC2)[:n, :n][iu], W[iu])


def test_bitset_sc2_many_small_problems():
    # the CUDA-core SC^2 over a batch of small problems: a CTA's run of work
    # units crosses many problems (one to four tiles each), so problem changes,
    # histogram flushes and the per-problem descriptors are exercised; the
    # results equal the tensor-core GEMM's batch, and single calls on the same
    # path give the oracle's stage buffers
    sizes = [3, 17, 64, 65, 128, 200, 256, 257, 300, 511, 512, 640] * 4
    probs = [synth.make_problem(("indoor", "outdoor", "cube")[b % 3], n, 0.2, 300 + b)
             for b, n in enumerate(sizes)]
    offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
    xs = np.concatenate([p.x for p in probs])
    ys = np.concatenate([p.y for p in probs])
    with trg.TurboReg(max_n=640, max_batch=len(probs)) as c:
        ref = c.register_batched(xs, ys, offs, [trg.default_params(p.tau, min(p.k1, 100), p.theta) for p in probs])
        out = c.register_batched(xs, ys, offs, [trg.default_params(p.tau, min(p.k1, 100), p.theta,
                                                                    flags=trg.FLAG_SC2_BITSET) for p in probs])
        for a, b in zip(ref, out):
            assert a.status == b.status and a.hypothesis == b.hypothesis and a.n_pivots == b.n_pivots
            assert np.array_equal(a.R, b.R) and np.array_equal(a.t, b.t) and a.inlier_count == b.inlier_count
        for k in (0, 1, 7, 10, 11):   # single calls on the same path: the stage buffers against the oracle
            p = probs[k]
            c.register(p.x, p.y, trg.default_params(p.tau, min(p.k1, 100), p.theta, flags=trg.FLAG_SC2_BITSET))
            A, S, _, _ = oracle_stages(p.x, p.y, p.tau, 100, 2)
            check_graph_stages(c, A, S, p.n)


def test_batched_equals_plain(ctx):
    probs = [synth.make_problem(s, n, r, 50 + b) for b, (s, n, r) in
             enumerate([("indoor", 1200, 0.1), ("outdoor", 900, 0.2), ("indoor", 3000, 0.05),
                        ("cube", 1000, 0.1), ("outdoor", 2500, 0.15)])]
    params = [trg.default_params(p.tau, p.k1, p.theta) for p in probs]
    offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
    xs = np.concatenate([p.x for p in probs])
    ys = np.concatenate([p.y for p in probs])
    out = ctx.register_batched(xs, ys, offs, params)
    for p, prm, rb in zip(probs, params, out):
        rp = ctx.register(p.x, p.y, prm)
        assert rb.status == rp.status and rb.hypothesis == rp.hypothesis
        assert np.array_equal(rb.R, rp.R) and np.array_equal(rb.t, rp.t)
        assert rb.inlier_count == rp.inlier_count


def test_stage_times_reported(ctx):
    p = synth.make_problem("indoor", 5000, 0.05, 19)
    prm = trg.default_params(p.tau, 2000, p.theta, flags=trg.FLAG_STAGE_TIMES)
    ctx.register(p.x, p.y, prm)
    st = ctx.stage_times()
    assert list(st) == ["pack", "compat", "sc2", "proposal", "topk", "pgs", "verify", "finalize"]
    assert all(v >= 0 for v in st.values())
    print(st)


def test_graph_replay_equals_direct_launches(ctx):
    # same shape, different inputs: the captured graph is replayed with patched input pointers
    for seed in (60, 61, 62):
        p = synth.make_problem("indoor", 4000, 0.05, seed)
        direct = ctx.register(p.x, p.y, trg.default_params(p.tau, 1500, p.theta, flags=trg.FLAG_NO_GRAPH))
        IN_d = ctx.buffer(trg.BUF_INLIERS).copy()
        graph = ctx.register(p.x, p.y, trg.default_params(p.tau, 1500, p.theta))
        assert graph.status == direct.status and graph.hypothesis == direct.hypothesis
        assert np.array_equal(graph.R, direct.R) and np.array_equal(graph.t, direct.t)
        assert np.array_equal(ctx.buffer(trg.BUF_INLIERS), IN_d)


def test_kappa_distribution_report(ctx):
    p = synth.make_problem("indoor", 5000, 0.05, 0)
    res = ctx.register(p.x, p.y, trg.default_params(p.tau, 2000, p.theta))
    RT = ctx.buffer(trg.BUF_RT)
    flags = RT[:, 13].view(np.int32)
    kap = RT[(flags & 1) != 0, 12]
    print("kappa quantiles", np.quantile(kap, [0.5, 0.9, 0.99]).round(2), "fp64", int(((flags & 2) != 0).sum()),
          ">1e3", int((kap > 1e3).sum()), "winner kappa", RT[res.hypothesis, 12])


def test_batched_uneven_sizes_equal_plain():
    # a batch of mixed indoor/outdoor problems of uneven N, one launch per stage for all of them
    probs = synth.make_batch(12, seed=7, n_lo=300, n_hi=3000)
    c = trg.TurboReg(max_n=3000, max_batch=12)
    try:
        params = [trg.default_params(p.tau, p.k1, p.theta) for p in probs]
        offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
        xs = np.concatenate([p.x for p in probs])
        ys = np.concatenate([p.y for p in probs])
        out = c.register_batched(xs, ys, offs, params)
        out2 = c.register_batched(xs, ys, offs, params)          # replay of the captured batch graph
        for p, prm, rb, rb2 in zip(probs, params, out, out2):
            rp = c.register(p.x, p.y, prm)
            assert rb.status == rp.status and rb.hypothesis == rp.hypothesis, (p.n, p.shape)
            assert np.array_equal(rb.R, rp.R) and np.array_equal(rb.t, rp.t)
            assert rb.inlier_count == rp.inlier_count and rb.n_pivots == rp.n_pivots
            assert rb2.hypothesis == rb.hypothesis and np.array_equal(rb2.R, rb.R)
        # the first problem's stage buffers match the oracle after a batched call
        c.register_batched(xs, ys, offs, params)
        p = probs[0]
        A, S, piv, cl = oracle_stages(p.x, p.y, p.tau, p.k1, 2)
        check_graph_stages(c, A, S, p.n)
        check_pivots_cliques(c, piv, cl, 2)
    finally:
        c.close()


def test_batched_direct_launch_mode(ctx):
    probs = [synth.make_problem("cube", n, 0.1, 80 + n) for n in (700, 1500, 400)]
    params = [trg.default_params(p.tau, 500, p.theta, flags=trg.FLAG_NO_GRAPH) for p in probs]
    offs = np.cumsum([0] + [p.n for p in probs]).astype(np.int64)
    out = ctx.register_batched(np.concatenate([p.x for p in probs]), np.concatenate([p.y for p in probs]),
                               offs, params)
    for p, rb in zip(probs, out):
        rp = ctx.register(p.x, p.y, trg.default_params(p.tau, 500, p.theta))
        assert rb.hypothesis == rp.hypothesis and np.array_equal(rb.R, rp.R)
