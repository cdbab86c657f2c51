"""The compatibility kernel's FP32 decision (Eq. 1 without square roots),
emulated in NumPy operation by operation, against the FP64 definition.

With s_X, s_Y the squared distances, D = s_X - s_Y, Q = s_X + s_Y and
delta = |d_X - d_Y|, the parallelogram law gives (d_X + d_Y)^2 = 2Q - delta^2,
so D^2 = delta^2 (2Q - delta^2), increasing in delta^2 on [0, Q].  Hence
delta <= tau iff Phi = D^2 - 2 tau^2 max(Q, tau^2) + tau^4 <= 0 (for
Q < tau^2 the pair is compatible and Phi <= Q^2 - tau^4 < 0).  The kernel
evaluates Phi in FP32 and sends a pair to the FP64 evaluation when |Phi|
lies within the band g = Qc (16u |D| + 32u^2 Qc + 24u tau^2).

Checked here: the identity itself in exact rational arithmetic; every pair
the FP32 test decides (outside the band) agrees with the FP64 definition, on
pairs built to sit on the threshold and on random pairs over six orders of
magnitude of scale; the band catches the pairs where a plain FP32 evaluation
of |d_X - d_Y| is wrong; and few pairs of a random problem fall in the band.
"""
from fractions import Fraction

import numpy as np
import pytest

from test_compat_ties import dist64, tie_problem

F32, F64 = np.float32, np.float64
U = 2.0 ** -24


def _r32(x):
    return np.asarray(x, F64).astype(F32)


def _fma32(a, b, c):
    # a * b of two FP32 values is exact in FP64; one rounding of the sum to
    # FP64 then FP32 (double rounding moves a result by at most one ulp in
    # rare cases, far inside the band's margin)
    return _r32(np.asarray(a, F64) * np.asarray(b, F64) + np.asarray(c, F64))


def _sq32(a, b):
    d = (a - b).astype(F32)
    s = _r32(d[..., 0].astype(F64) * d[..., 0])
    s = _fma32(d[..., 1], d[..., 1], s)
    return _fma32(d[..., 2], d[..., 2], s)


def fp32_decision(xi, xj, yi, yj, tau):
    """(compatible, inside the band) of each pair, in the kernel's operation order."""
    tau = F32(tau)
    t2 = F32(tau * tau)
    e = _fma32(tau, tau, -t2)
    c1 = F32(-2.0) * t2
    c0 = _fma32(t2, t2, _r32(F64(F32(2.0) * t2) * F64(e)))
    sX, sY = _sq32(xi, xj), _sq32(yi, yj)
    D = _r32(sX.astype(F64) - sY)
    Q = _r32(sX.astype(F64) + sY)
    Qc = np.maximum(Q, t2)
    phi = _fma32(D, D, _fma32(Qc, c1, c0))
    w = _fma32(Qc, F32(32 * U * U), _r32(F64(F32(24 * U)) * F64(t2)))
    w = _fma32(np.abs(D), F32(16 * U), w)
    g = _r32(Qc.astype(F64) * w)
    return phi <= 0, ~(np.abs(phi) > g)


def fp64_decision(xi, xj, yi, yj, tau):
    return np.abs(dist64(xi, xj) - dist64(yi, yj)) <= F64(F32(tau))


def test_identity_exact():
    rng = np.random.default_rng(0)
    for _ in range(300):
        a, b = (Fraction(int(v), 64) for v in rng.integers(0, 640, 2))
        tau = Fraction(int(rng.integers(1, 200)), 64)
        sx, sy = a * a, b * b
        D, Q = sx - sy, sx + sy
        phi = D * D - 2 * tau * tau * max(Q, tau * tau) + tau ** 4
        assert (phi <= 0) == (abs(a - b) <= tau)


@pytest.mark.parametrize("kind,tau,seed", [("exact", 0.09375, 1), ("exact", 0.59375, 2),
                                           ("searched", 0.1, 3), ("searched", 0.6, 4)])
def test_band_holds_at_the_threshold(kind, tau, seed):
    X, Y, _ = tie_problem(kind, tau, seed)
    xi, xj, yi, yj = X[0::2], X[1::2], Y[0::2], Y[1::2]
    a, near = fp32_decision(xi, xj, yi, yj, tau)
    d64 = fp64_decision(xi, xj, yi, yj, tau)
    assert ((a != d64) & ~near).sum() == 0
    # the plain FP32 |dX - dY| gets some of these pairs wrong: all of them are in the band
    d32 = np.abs(np.sqrt(_sq32(xi, xj)) - np.sqrt(_sq32(yi, yj))) <= F32(tau)
    wrong32 = d32 != d64
    assert wrong32.sum() >= 1
    assert near[wrong32].all()


@pytest.mark.parametrize("scale,tau", [(0.05, 0.1), (1e-3, 1e-3), (1.0, 0.1), (35.0, 0.1), (1e4, 3.0),
                                       (1e6, 1048576.0)])
def test_band_holds_on_random_pairs(scale, tau):
    rng = np.random.default_rng(11)
    m = 100_000
    xi = (rng.normal(size=(m, 3)) * scale).astype(F32)
    xj = (xi + rng.normal(size=(m, 3)) * scale * rng.choice([0.01, 1.0], (m, 1))).astype(F32)
    yi = (rng.normal(size=(m, 3)) * scale).astype(F32)
    dirn = rng.normal(size=(m, 3))
    dirn /= np.linalg.norm(dirn, axis=1, keepdims=True)
    yj = (yi + dirn * (dist64(xi, xj) + rng.uniform(-2, 2, m) * tau)[:, None]).astype(F32)
    a, near = fp32_decision(xi, xj, yi, yj, tau)
    d64 = fp64_decision(xi, xj, yi, yj, tau)
    assert ((a != d64) & ~near).sum() == 0
    assert near.mean() < 0.01


def test_few_pairs_in_the_band_on_a_problem():
    import synth
    p = synth.make_problem("indoor", 1500, 0.05, 0)
    i, j = np.triu_indices(p.x.shape[0], 1)
    a, near = fp32_decision(p.x[i], p.x[j], p.y[i], p.y[j], 0.1)
    d64 = fp64_decision(p.x[i], p.x[j], p.y[i], p.y[j], 0.1)
    assert ((a != d64) & ~near).sum() == 0
    assert near.sum() <= 20
    assert 0.01 < d64.mean() < 0.2
