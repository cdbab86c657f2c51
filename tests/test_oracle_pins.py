"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, exact-arithmetic geometry, brute force on tiny inputs, an independent
library routine, invariants, or the hand-worked graph of App. E.1.  They are
chosen so that a dropped term, a wrong sign or index, a flipped comparison or
a transposed operand in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _random_graph(n, p, seed):
    rng = _rng(seed)
    U = np.triu((rng.random((n, n)) < p).astype(np.uint8), 1)
    return U | U.T


def _load_golden(golden_dir):
    g = {"edge": [], "pivot": [], "clique": [], "uclique": []}
    with open(os.path.join(golden_dir, "appE1_graph.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            key, vals = line[0], [int(v) for v in line[1:]]
            if key in g:
                g[key].append(vals)
            else:
                g[key] = vals[0]
    return g


# --------------------------------------------------------------------------
# Eq. 1: compatibility graph
# --------------------------------------------------------------------------

def test_compat_symmetric_zero_diagonal():
    p = synth.make_problem("cube", 300, 0.2, 3)
    A = oracle.compat(p.x, p.y, p.tau)
    assert np.array_equal(A, A.T)
    assert not A.diagonal().any()
    assert set(np.unique(A)) <= {0, 1}


def test_compat_pure_translation_is_complete_even_at_tau_zero():
    # integer coordinates and an integer shift: every distance is preserved
    # exactly in floating point, so |dX - dY| = 0 <= tau for tau = 0 (Eq. 1 uses <=)
    rng = _rng(1)
    x = rng.integers(-20, 20, size=(40, 3)).astype(np.float32)
    y = x + np.float32([3, -7, 11])
    A = oracle.compat(x, y, 0.0)
    assert np.array_equal(A, 1 - np.eye(40, dtype=np.uint8))


def test_compat_scaled_line_gives_band_matrix():
    # points on a line at integer positions, target scaled by 2:
    # dX = |i-j|, dY = 2|i-j|, so |dX - dY| = |i-j| and the graph is the band |i-j| <= tau.
    n = 12
    x = np.zeros((n, 3), dtype=np.float32)
    x[:, 0] = np.arange(n)
    y = 2 * x
    for tau, width in [(2.0, 2), (2.5, 2), (0.5, 0), (1.0, 1)]:
        A = oracle.compat(x, y, tau)
        band = np.zeros((n, n), dtype=np.uint8)
        for i in range(n):
            for j in range(n):
                if i != j and abs(i - j) <= width:
                    band[i, j] = 1
        assert np.array_equal(A, band), tau


def test_compat_pythagorean_distances():
    # dX = 5 (3-4-5 triangle), dY = 13 (5-12-13): |dX - dY| = 8 exactly
    x = np.float32([[0, 0, 0], [3, 4, 0]])
    y = np.float32([[1, 1, 1], [6, 13, 1]])
    assert oracle.compat(x, y, 8.0)[0, 1] == 1
    assert oracle.compat(x, y, np.nextafter(np.float32(8.0), np.float32(0)))[0, 1] == 0


def test_compat_threshold_extremes():
    p = synth.make_problem("cube", 200, 0.1, 5)
    assert not oracle.compat(p.x, p.y, -1.0).any()
    A = oracle.compat(p.x, p.y, 1e30)
    assert np.array_equal(A, 1 - np.eye(200, dtype=np.uint8))


def test_compat_noiseless_inliers_form_a_clique():
    # App. A.3: with sigma = 0 the inlier triangles are congruent, so the inlier
    # block is complete for any tau covering float32 rounding of y.
    p = synth.make_problem("cube", 300, 0.3, 7, sigma=0.0)
    A = oracle.compat(p.x, p.y, 1e-5)
    idx = np.flatnonzero(p.inlier)
    blk = A[np.ix_(idx, idx)]
    assert np.array_equal(blk, 1 - np.eye(len(idx), dtype=np.uint8))


# --------------------------------------------------------------------------
# Eq. 2: SC^2
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 0), (2, 1.0, 0), (7, 0.6, 1), (63, 0.3, 2),
                                      (64, 0.5, 3), (65, 0.1, 4), (130, 0.2, 5)])
def test_sc2_matches_integer_matmul(n, p, seed):
    A = _random_graph(n, p, seed)
    S = oracle.sc2(A)
    A64 = A.astype(np.int64)
    assert np.array_equal(S, (A64 @ A64) * A64)


def test_sc2_counts_triangles():
    # App. B: G^_ij is the number of 3-cliques containing edge (i,j), so the
    # sum over edges equals 3 x (number of triangles), counted here by brute force.
    for seed in range(4):
        A = _random_graph(25, 0.35, seed)
        S = oracle.sc2(A)
        tri = sum(1 for a, b, c in itertools.combinations(range(25), 3)
                  if A[a, b] and A[a, c] and A[b, c])
        assert int(np.triu(S, 1).sum()) == 3 * tri
        for a, b in itertools.combinations(range(25), 2):
            if A[a, b]:
                assert S[a, b] == sum(1 for c in range(25) if A[a, c] and A[b, c])


def test_sc2_complete_graph():
    for n in (3, 10, 77):
        A = 1 - np.eye(n, dtype=np.uint8)
        S = oracle.sc2(A)
        assert np.array_equal(S, (n - 2) * (1 - np.eye(n, dtype=np.int32)))


def test_sc2_appendix_graph(golden_dir):
    g = _load_golden(golden_dir)
    n = g["n"]
    A = np.zeros((n, n), dtype=np.uint8)
    for u, v, _ in g["edge"]:
        A[u - 1, v - 1] = A[v - 1, u - 1] = 1
    S = oracle.sc2(A)
    expect = np.zeros((n, n), dtype=np.int32)
    for u, v, w in g["edge"]:
        expect[u - 1, v - 1] = expect[v - 1, u - 1] = w
    assert np.array_equal(S, expect)
    assert int(np.triu(S, 1).sum()) == 3 * g["triangles"]


# --------------------------------------------------------------------------
# Eq. 4 on the O2Graph: pivots
# --------------------------------------------------------------------------

def test_pivots_brute_force_sort():
    for seed, (n, p, k1) in enumerate([(30, 0.4, 10), (60, 0.2, 100), (50, 0.5, 1000), (40, 0.05, 7)]):
        A = _random_graph(n, p, seed)
        S = oracle.sc2(A)
        pi, pj, pw = oracle.pivots(S, k1)
        edges = [(-int(S[i, j]), i, j) for i in range(n) for j in range(i + 1, n) if S[i, j] > 0]
        edges.sort()
        want = edges[:k1]
        assert len(pi) == len(want) == min(k1, len(edges))
        assert [(-w, i, j) for w, i, j in want] == list(zip(pw.tolist(), pi.tolist(), pj.tolist()))
        # selection invariant: no unselected edge outranks a selected one
        if len(edges) > k1:
            assert pw.min() >= -edges[k1][0]


def test_pivots_ignore_zero_weight_edges():
    # an isolated edge has no common neighbour: SC^2 = 0, not an O2Graph edge
    A = np.zeros((5, 5), dtype=np.uint8)
    A[0, 1] = A[1, 0] = 1
    S = oracle.sc2(A)
    pi, pj, pw = oracle.pivots(S, 10)
    assert len(pi) == 0


def test_pivots_appendix_graph(golden_dir):
    g = _load_golden(golden_dir)
    n = g["n"]
    A = np.zeros((n, n), dtype=np.uint8)
    for u, v, _ in g["edge"]:
        A[u - 1, v - 1] = A[v - 1, u - 1] = 1
    pi, pj, pw = oracle.pivots(oracle.sc2(A), g["k1"])
    assert [[a + 1, b + 1, w] for a, b, w in zip(pi, pj, pw)] == g["pivot"]


# --------------------------------------------------------------------------
# Eq. 5-7, Alg. 1, App. C: TurboCliques
# --------------------------------------------------------------------------

def _exhaustive_cliques(A, S, pi, pj, k2):
    """All 3-cliques grouped by their lowest pair (App. C), ranked by Eq. 6."""
    n = A.shape[0]
    by_pair = {}
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[a, c] and A[b, c]:
            by_pair.setdefault((a, b), []).append((-(S[a, b] + S[a, c] + S[b, c]), c))
    out = []
    for i, j in zip(pi.tolist(), pj.tolist()):
        lst = sorted(by_pair.get((i, j), []))[:k2]
        out.append([z for _, z in lst])
    return out


@pytest.mark.parametrize("n,p,k1,k2,seed", [(20, 0.5, 15, 2, 0), (40, 0.3, 60, 3, 1),
                                            (60, 0.25, 200, 2, 2), (60, 0.6, 50, 1, 3),
                                            (33, 0.9, 500, 5, 4), (12, 0.2, 20, 2, 5)])
def test_cliques_exhaustive_small(n, p, k1, k2, seed):
    A = _random_graph(n, p, seed)
    S = oracle.sc2(A)
    pi, pj, pw = oracle.pivots(S, k1)
    cl, va = oracle.cliques(S, pi, pj, k2)
    want = _exhaustive_cliques(A, S, pi, pj, k2)
    np_ = len(pi)
    seen = set()
    for p_ in range(np_):
        got = [int(cl[r * np_ + p_, 2]) for r in range(k2) if va[r * np_ + p_]]
        assert got == want[p_]
        for r in range(k2):
            h = r * np_ + p_
            if not va[h]:
                continue
            i, j, z = cl[h]
            assert (i, j) == (pi[p_], pj[p_])
            assert i < j < z                                   # O2Graph orientation
            assert A[i, j] * A[i, z] * A[j, z] > 0             # Eq. 8
            assert (i, j, z) not in seen                       # Unique Assignment (App. C)
            seen.add((i, j, z))


def test_neighbour_test_equals_adjacency():
    # Eq. 5 tests G~_iz > 0 and G~_jz > 0; on a pivot edge this is the same set as
    # z > j with A_iz = A_jz = 1, because j is then a common neighbour of (i, z).
    A = _random_graph(50, 0.3, 9)
    S = oracle.sc2(A)
    for i in range(50):
        for j in range(i + 1, 50):
            if S[i, j] <= 0:
                continue
            via_s = {z for z in range(50) if z not in (i, j)
                     and (i < z and S[i, z] > 0) and (j < z and S[j, z] > 0)}
            via_a = {z for z in range(j + 1, 50) if A[i, z] and A[j, z]}
            assert via_s == via_a


def test_cliques_appendix_graph(golden_dir):
    g = _load_golden(golden_dir)
    n = g["n"]
    A = np.zeros((n, n), dtype=np.uint8)
    for u, v, _ in g["edge"]:
        A[u - 1, v - 1] = A[v - 1, u - 1] = 1
    S = oracle.sc2(A)
    pi, pj, _ = oracle.pivots(S, g["k1"])
    cl, va = oracle.cliques(S, pi, pj, g["k2"])
    assert va.all()
    assert [[h] + (cl[h] + 1).tolist() for h in range(len(cl))] == g["clique"]


def test_cliques_appendix_graph_undirected(golden_dir):
    g = _load_golden(golden_dir)
    n = g["n"]
    A = np.zeros((n, n), dtype=np.uint8)
    for u, v, _ in g["edge"]:
        A[u - 1, v - 1] = A[v - 1, u - 1] = 1
    S = oracle.sc2(A)
    pi, pj, _ = oracle.pivots(S, g["k1"])
    cl, va = oracle.cliques(S, pi, pj, g["k2"], graph_mode=oracle.GRAPH_SC2)
    assert va.all()
    assert [[h] + (cl[h] + 1).tolist() for h in range(len(cl))] == g["uclique"]


def _exhaustive_cliques_undirected(A, S, pi, pj, k2):
    """Every 3-clique containing the pivot edge, ranked by Eq. 6 on the
    symmetric SC^2 graph (ties: lower z)."""
    n = A.shape[0]
    tri = [(a, b, c) for a, b, c in itertools.combinations(range(n), 3)
           if A[a, b] and A[a, c] and A[b, c]]
    out = []
    for i, j in zip(pi.tolist(), pj.tolist()):
        lst = []
        for t in tri:
            if i in t and j in t:
                z = [v for v in t if v not in (i, j)][0]
                lst.append((-(S[i, j] + S[i, z] + S[j, z]), z))
        out.append([z for _, z in sorted(lst)[:k2]])
    return out


@pytest.mark.parametrize("n,p,k1,k2,seed", [(20, 0.5, 15, 2, 0), (40, 0.3, 60, 3, 1),
                                            (60, 0.25, 200, 2, 2), (33, 0.9, 500, 5, 4)])
def test_cliques_undirected_exhaustive_small(n, p, k1, k2, seed):
    A = _random_graph(n, p, seed)
    S = oracle.sc2(A)
    pi, pj, pw = oracle.pivots(S, k1)
    cl, va = oracle.cliques(S, pi, pj, k2, graph_mode=oracle.GRAPH_SC2)
    want = _exhaustive_cliques_undirected(A, S, pi, pj, k2)
    np_ = len(pi)
    for p_ in range(np_):
        got = [int(cl[r * np_ + p_, 2]) for r in range(k2) if va[r * np_ + p_]]
        assert got == want[p_]
        for r in range(k2):
            h = r * np_ + p_
            if va[h]:
                i, j, z = cl[h]
                assert A[i, j] * A[i, z] * A[j, z] > 0             # Eq. 8
                assert z not in (i, j)


def test_undirected_search_finds_at_least_the_o2_cliques():
    # with K2 at least the largest common-neighbour count, every O2Graph clique
    # of a pivot is also one of its undirected cliques (z > j is a subset)
    A = _random_graph(45, 0.35, 11)
    S = oracle.sc2(A)
    pi, pj, _ = oracle.pivots(S, 80)
    k2 = 45
    co, vo = oracle.cliques(S, pi, pj, k2)
    cu, vu = oracle.cliques(S, pi, pj, k2, graph_mode=oracle.GRAPH_SC2)
    so = {tuple(sorted(c)) for c, v in zip(co.tolist(), vo) if v}
    su = {tuple(sorted(c)) for c, v in zip(cu.tolist(), vu) if v}
    assert so <= su
    # every triangle through a pivot edge appears, and the O2Graph finds each once
    assert sum(vo) == len(so)


def test_cliques_missing_slots_are_invalid():
    # a pivot with one common neighbour cannot fill K2 = 3 slots
    A = np.zeros((4, 4), dtype=np.uint8)
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        A[a, b] = A[b, a] = 1
    S = oracle.sc2(A)
    pi, pj, _ = oracle.pivots(S, 5)
    cl, va = oracle.cliques(S, pi, pj, 3)
    # pivots: (0,1),(0,2),(1,2) all weight 1; only (0,1) has z=2 > j
    assert len(pi) == 3
    assert va.tolist() == [True, False, False] + [False] * 6
    assert cl[0].tolist() == [0, 1, 2]


# --------------------------------------------------------------------------
# Sec. 3.5: Kabsch
# --------------------------------------------------------------------------

def _rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _horn(xs, ys):
    """Horn's closed-form quaternion solution (max eigenvector of the 4x4 matrix)."""
    cx, cy = xs.mean(0), ys.mean(0)
    M = (xs - cx).T @ (ys - cy)
    Sxx, Sxy, Sxz = M[0]; Syx, Syy, Syz = M[1]; Szx, Szy, Szz = M[2]
    N = np.array([
        [Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
        [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
        [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
        [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    wv, vv = np.linalg.eigh(N)
    q0, qx, qy, qz = vv[:, np.argmax(wv)]
    R = np.array([
        [q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy)],
        [2 * (qy * qx + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx)],
        [2 * (qz * qx - q0 * qy), 2 * (qz * qy + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz]])
    return R, cy - R @ cx


def test_svd3_reconstructs_and_matches_numpy():
    rng = _rng(11)
    for _ in range(200):
        H = rng.normal(size=(3, 3)) * 10 ** rng.uniform(-3, 3)
        U, s, V = oracle.svd3(H)
        assert np.allclose(U @ np.diag(s) @ V.T, H, atol=1e-12 * np.abs(H).max())
        assert np.allclose(U.T @ U, np.eye(3), atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)
        assert np.allclose(s, np.linalg.svd(H, compute_uv=False), rtol=1e-12, atol=1e-14 * s[0])


def test_kabsch_noiseless_recovery():
    # App. A.3: three noiseless matches fix the rigid transform exactly
    rng = _rng(12)
    for _ in range(300):
        R = _rand_rot(rng)
        t = rng.uniform(-10, 10, 3)
        xs = rng.uniform(-5, 5, (3, 3))
        ys = xs @ R.T + t
        ok, Re, te, kappa = oracle.kabsch(xs, ys)
        assert ok
        assert np.abs(Re - R).max() < 1e-9
        assert np.abs(te - t).max() < 1e-9


def test_kabsch_agrees_with_horn_on_noisy_triangles():
    rng = _rng(13)
    for _ in range(300):
        xs = rng.uniform(-5, 5, (3, 3))
        ys = xs @ _rand_rot(rng).T + rng.normal(scale=0.5, size=(3, 3)) + rng.uniform(-3, 3, 3)
        ok, Re, te, kappa = oracle.kabsch(xs, ys)
        assert ok
        Rh, th = _horn(xs, ys)
        assert np.abs(Re - Rh).max() < 1e-9 * max(1.0, kappa)
        assert np.abs(te - th).max() < 1e-8 * max(1.0, kappa)
        assert np.allclose(Re.T @ Re, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(Re) - 1) < 1e-12


def test_kabsch_mirrored_triangle_gives_proper_rotation():
    # target is a reflection of the source: the best proper rotation flips the plane normal
    rng = _rng(14)
    for _ in range(100):
        xs = rng.uniform(-5, 5, (3, 3))
        ys = xs.copy()
        ys[:, 2] *= -1
        ok, Re, te, _ = oracle.kabsch(xs, ys)
        assert ok
        assert abs(np.linalg.det(Re) - 1) < 1e-12
        # three points are coplanar: a proper rotation can still map them exactly
        assert np.abs(xs @ Re.T + te - ys).max() < 1e-9
        Rh, th = _horn(xs, ys)
        assert np.abs(Re - Rh).max() < 1e-8


def test_kabsch_degenerate_triangles_invalid():
    xs = np.array([[0, 0, 0], [1, 1, 1], [2, 2, 2.0]])      # collinear
    ok, *_ = oracle.kabsch(xs, xs + 1)
    assert not ok
    xs = np.array([[1, 2, 3], [1, 2, 3], [4, 5, 6.0]])      # duplicate point
    ok, *_ = oracle.kabsch(xs, xs)
    assert not ok
    ok, *_ = oracle.kabsch(np.ones((3, 3)), np.ones((3, 3)))
    assert not ok


def test_kabsch_n_recovers_noiseless_and_agrees_with_horn():
    rng = _rng(19)
    for m in (4, 10, 25):
        for _ in range(40):
            R = _rand_rot(rng)
            t = rng.uniform(-3, 3, 3)
            xs = rng.uniform(-5, 5, (m, 3))
            ok, Re, te, _ = oracle.kabsch_n(xs, xs @ R.T + t)
            assert ok and np.abs(Re - R).max() < 1e-9 and np.abs(te - t).max() < 1e-9
            ys = xs @ R.T + t + rng.normal(scale=0.3, size=(m, 3))
            ok, Re, te, kappa = oracle.kabsch_n(xs, ys)
            Rh, th = _horn(xs, ys)
            assert ok and np.abs(Re - Rh).max() < 1e-9 * max(1.0, kappa)
            assert np.abs(te - th).max() < 1e-8 * max(1.0, kappa)
            assert abs(np.linalg.det(Re) - 1) < 1e-12
            # the matches' order does not matter
            perm = rng.permutation(m)
            ok2, Rp, tp, _ = oracle.kabsch_n(xs[perm], ys[perm])
            assert ok2 and np.abs(Rp - Re).max() < 1e-9 * max(1.0, kappa)


def test_kabsch_n_mirrored_cloud_and_degenerate():
    rng = _rng(20)
    xs = rng.uniform(-5, 5, (10, 3))
    ys = xs.copy()
    ys[:, 2] *= -1                         # a reflection: no proper rotation fits 10 generic points
    ok, Re, te, _ = oracle.kabsch_n(xs, ys)
    Rh, th = _horn(xs, ys)
    assert ok and abs(np.linalg.det(Re) - 1) < 1e-12 and np.abs(Re - Rh).max() < 1e-8
    line = np.outer(np.arange(10.0), [1.0, 2.0, -1.0])
    assert not oracle.kabsch_n(line, line + 1)[0]
    # three points: identical to the 3-point routine
    tri = rng.uniform(-5, 5, (3, 3))
    tri_y = tri @ _rand_rot(rng).T + rng.normal(scale=0.1, size=(3, 3))
    a, b = oracle.kabsch(tri, tri_y), oracle.kabsch_n(tri, tri_y)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


# --------------------------------------------------------------------------
# Sec. 3.5: inlier number
# --------------------------------------------------------------------------

def test_inliers_exact_residuals():
    # R = I, t = 0, residuals exactly 0.25, 0.5, 0.75 m along x; theta = 0.5 counts
    # the 0.5 m one (<=) and rejects 0.75.
    x = np.zeros((6, 3), dtype=np.float32)
    x[:, 1] = np.arange(6)
    y = x.copy()
    y[:, 0] += np.float32([0.0, 0.25, 0.5, 0.75, 1.0, 0.5])
    c, near = oracle.inliers(x, y, np.eye(3), np.zeros(3), 0.5, band=1e-6)
    assert c == 4 and near == 2
    # a rotation by 90 degrees about z with the matching translation
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    y2 = (x.astype(np.float64) @ Rz.T + [1, 2, 3]).astype(np.float32)
    assert oracle.inliers(x, y2, Rz, np.array([1.0, 2, 3]), 1e-3)[0] == 6
    assert oracle.inliers(x, y2, Rz.T, np.array([1.0, 2, 3]), 1e-3)[0] <= 1


def test_inliers_ground_truth_counts_noiseless_inliers():
    p = synth.make_problem("cube", 500, 0.2, 15, sigma=0.0)
    c, _ = oracle.inliers(p.x, p.y, p.R_gt, p.t_gt, 1e-4)
    assert c >= p.inlier.sum()


# --------------------------------------------------------------------------
# Hypothesis scores of the ranking study (Table 6): IN, MAE, MSE
# --------------------------------------------------------------------------

def test_score_hand_example():
    # y = Rz x + t + offsets with residuals 0.5, 0.25, 2 and 0 m (all exact in
    # binary); theta = 1:  IN = 3, MAE = (0.5 + 0.25 + 1 + 0) / 4 = 0.4375,
    # MSE = (0.25 + 0.0625 + 1 + 0) / 4 = 0.328125  (the 2 m residual is capped at theta)
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    t = np.array([1.0, -2.0, 4.0])
    x = np.array([[1, 2, 3], [-4, 0, 1], [2, 2, -2], [0, 5, 1]], dtype=np.float32)
    y = (x.astype(np.float64) @ Rz.T + t).astype(np.float32)
    y[0, 0] += 0.5
    y[1, 1] -= 0.25
    y[2, 2] += 2.0
    assert oracle.score(x, y, Rz, t, 1.0, oracle.SCORE_IN) == 3.0
    assert oracle.score(x, y, Rz, t, 1.0, oracle.SCORE_MAE) == 0.4375
    assert oracle.score(x, y, Rz, t, 1.0, oracle.SCORE_MSE) == 0.328125
    # theta = 0.5: the 0.5 m residual sits exactly on the threshold
    assert oracle.score(x, y, Rz, t, 0.5, oracle.SCORE_IN) == 3.0
    assert oracle.score(x, y, Rz, t, 0.5, oracle.SCORE_MAE) == (0.5 + 0.25 + 0.5) / 4
    assert oracle.score(x, y, Rz, t, 0.5, oracle.SCORE_MSE) == (0.25 + 0.0625 + 0.25) / 4


def test_score_bounds_and_extremes():
    rng = _rng(17)
    p = synth.make_problem("cube", 400, 0.3, 17)
    th = p.theta
    for _ in range(30):
        R = _rand_rot(rng) if rng.random() < 0.5 else p.R_gt
        t = p.t_gt + rng.normal(scale=0.05, size=3)
        inn = oracle.score(p.x, p.y, R, t, th, oracle.SCORE_IN)
        mae = oracle.score(p.x, p.y, R, t, th, oracle.SCORE_MAE)
        mse = oracle.score(p.x, p.y, R, t, th, oracle.SCORE_MSE)
        n = p.n
        # every residual is capped at theta; an outlier of (R,t) costs exactly theta
        th64 = float(np.float32(th))
        assert 0 <= mse <= th64 * mae + 1e-15 and mae <= th64 + 1e-15
        assert mae >= th64 * (n - inn) / n - 1e-15
        assert mse >= th64 * th64 * (n - inn) / n - 1e-15
        assert inn == oracle.inliers(p.x, p.y, R, t, th)[0]
    # exact fit: zero error; everything far away: theta and theta^2
    x = p.x[:50]
    y = (x.astype(np.float64) @ p.R_gt.T + p.t_gt).astype(np.float32)
    assert oracle.score(x, x, np.eye(3), np.zeros(3), 0.1, oracle.SCORE_MAE) == 0.0
    assert oracle.score(x, x, np.eye(3), np.zeros(3), 0.1, oracle.SCORE_MSE) == 0.0
    far = np.array([1e3, 0, 0])
    assert oracle.score(x, y, p.R_gt, p.t_gt + far, 0.1, oracle.SCORE_MAE) == float(np.float32(0.1))
    assert oracle.score(x, y, p.R_gt, p.t_gt + far, 0.1, oracle.SCORE_MSE) == float(np.float32(0.1)) ** 2


@pytest.mark.parametrize("scoring", [1, 2])
def test_register_scoring_selects_smallest_error(scoring):
    p = synth.make_problem("indoor", 600, 0.08, 23)
    r = oracle.register(p.x, p.y, p.tau, 120, p.theta, scoring=scoring)
    r0 = oracle.register(p.x, p.y, p.tau, 120, p.theta)
    assert r.status == 0
    # the same hypotheses as the inlier-number run; the winner minimises the score
    assert np.array_equal(r.hyp_valid, r0.hyp_valid)
    assert np.array_equal(r.in_counts, r0.in_counts)
    sc = np.where(r.hyp_valid, r.scores, np.inf)
    assert r.hypothesis == int(np.argmin(sc))           # argmin returns the lowest h on ties
    h = r.hypothesis
    assert r.score == sc[h]
    assert r.score == oracle.score(p.x, p.y, r.rt[h, :9].reshape(3, 3), r.rt[h, 9:], p.theta, scoring)
    assert r.inlier_count == r.in_counts[h]
    # IN-mode scores are the inlier numbers
    assert np.array_equal(np.where(r0.hyp_valid, r0.scores, -1).astype(np.int64), r0.in_counts.astype(np.int64))
    assert synth.rotation_error_deg(p.R_gt, r.R) < p.re_deg
    assert synth.translation_error(p.t_gt, r.t) < p.te_m


def test_register_scoring_noiseless_reaches_ground_truth_error():
    # sigma = 0: a clique of three inliers reproduces (R_gt, t_gt), whose capped
    # error is the smallest any hypothesis can reach on these matches up to rounding
    p = synth.make_problem("cube", 300, 0.3, 29, sigma=0.0)
    for scoring in (1, 2):
        r = oracle.register(p.x, p.y, 1e-4, 150, 1e-3, scoring=scoring)
        gt = oracle.score(p.x, p.y, p.R_gt, p.t_gt, 1e-3, scoring)
        assert r.status == 0
        assert r.score <= gt + 1e-9
        assert np.abs(r.R - p.R_gt).max() < 1e-5


def test_register_undirected_graph_mode():
    # same pivots as the O2Graph run; every clique is a 3-clique of G
    p = synth.make_problem("cube", 200, 0.3, 37)
    ro = oracle.register(p.x, p.y, p.tau, 60, p.theta)
    ru = oracle.register(p.x, p.y, p.tau, 60, p.theta, graph_mode=oracle.GRAPH_SC2)
    assert ru.status == 0 and ru.n_pivots == ro.n_pivots
    assert ru.n_valid >= ro.n_valid
    assert synth.rotation_error_deg(p.R_gt, ru.R) < p.re_deg
    A = oracle.compat(p.x, p.y, p.tau)
    i, j, z = ru.clique
    assert A[i, j] and A[i, z] and A[j, z]


# --------------------------------------------------------------------------
# Whole path
# --------------------------------------------------------------------------

def test_register_composes_the_stages():
    p = synth.make_problem("cube", 150, 0.3, 21)
    r = oracle.register(p.x, p.y, p.tau, 40, p.theta, k2=2)
    A = oracle.compat(p.x, p.y, p.tau)
    S = oracle.sc2(A)
    pi, pj, pw = oracle.pivots(S, 40)
    cl, va = oracle.cliques(S, pi, pj, 2)
    assert r.n_pivots == len(pi)
    best, best_in = -1, -1
    for h in range(len(cl)):
        if not va[h]:
            continue
        ok, R, t, _ = oracle.kabsch(p.x[cl[h]].astype(np.float64), p.y[cl[h]].astype(np.float64))
        if not ok:
            continue
        c, _ = oracle.inliers(p.x, p.y, R, t, p.theta)
        assert r.in_counts[h] == c
        if c > best_in:
            best, best_in = h, c
    assert r.hypothesis == best and r.inlier_count == best_in
    assert tuple(cl[best].tolist()) == r.clique


@pytest.mark.parametrize("shape,n,ratio", [("cube", 1000, 0.1), ("outdoor", 1500, 0.2)])
def test_register_recovers_ground_truth(shape, n, ratio):
    p = synth.make_problem(shape, n, ratio, 31)
    r = oracle.register(p.x, p.y, p.tau, p.k1, p.theta)
    assert r.status == 0
    assert synth.rotation_error_deg(p.R_gt, r.R) < p.re_deg
    assert synth.translation_error(p.t_gt, r.t) < p.te_m


def test_register_noiseless_is_exact():
    p = synth.make_problem("cube", 400, 0.25, 41, sigma=0.0)
    r = oracle.register(p.x, p.y, 1e-4, 200, 1e-3)
    assert r.status == 0
    assert np.abs(r.R - p.R_gt).max() < 1e-5
    assert r.inlier_count >= p.inlier.sum()


def test_register_no_hypothesis_and_bad_args():
    p = synth.make_problem("cube", 50, 0.1, 1)
    r = oracle.register(p.x, p.y, -1.0, 10, 0.1)
    assert r.status == 1
    r = oracle.register(p.x, p.y, 0.0, 10, 0.1)          # no compatible pair
    assert r.status == 7 and r.n_pivots == 0
    assert np.array_equal(r.R, np.eye(3))
    r = oracle.register(p.x[:2], p.y[:2], 0.1, 10, 0.1)
    assert r.status == 2
