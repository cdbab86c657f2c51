"""Pins of the FP64 proposal-MLP oracle (the learned proposal is a project
extension; these pin the oracle against finite differences, an independent
bfloat16 conversion and hand-computed features)."""
import numpy as np
import pytest

from oracle import mlp


def _rand_theta(seed, scale=0.5):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(scale=scale, size=mlp.N_PARAMS)


def test_parameter_count():
    assert mlp.N_PARAMS == 17217
    th = _rand_theta(0)
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)


def test_gradient_matches_finite_differences():
    rng = np.random.Generator(np.random.PCG64(1))
    th = _rand_theta(2)
    feat = rng.normal(size=(16, 8))
    lab = (rng.random(16) < 0.5).astype(np.float64)
    g, L = mlp.grad(th, feat, lab, bf16_round=False)
    assert abs(L - mlp.loss(th, feat, lab, bf16_round=False)) < 1e-12
    idx = rng.choice(mlp.N_PARAMS, size=300, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss(th + e, feat, lab, False) - mlp.loss(th - e, feat, lab, False)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, g[k])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.Generator(np.random.PCG64(3))
    a = np.concatenate([rng.normal(size=5000) * 10 ** rng.uniform(-20, 20, 5000),
                        [0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3e38]]).astype(np.float32)
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(a), want)
    assert mlp.bf16(np.float32(1.0 + 2 ** -8)) == 1.0          # tie to even
    assert mlp.bf16(np.float32(1.0 + 3 * 2 ** -9)) == 1.0 + 2 ** -7


def test_features_by_hand():
    # four points on a square around (1, 1, 0): centred coordinates +-1, rms = sqrt(2)
    x = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0], [2, 2, 0]], dtype=np.float32)
    y = 3 * x
    A = np.array([[0, 1, 1, 0], [1, 0, 0, 0], [1, 0, 0, 1], [0, 0, 1, 0]], dtype=np.uint8)
    S = np.array([[0, 2, 1, 0], [2, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 0]])
    f = mlp.features(x, y, A, S)
    r2 = 1 / np.sqrt(2)
    assert np.allclose(f[:, :3], [[-r2, -r2, 0], [r2, -r2, 0], [-r2, r2, 0], [r2, r2, 0]])
    assert np.allclose(f[:, 3:6], f[:, :3])                   # scale-free
    assert np.allclose(f[:, 6], [0.5, 0.25, 0.5, 0.25])
    assert np.allclose(f[:, 7], [1.0, 2 / 3, 1 / 3, 0.0])


def test_bce_gradient_closed_form_single_unit():
    # with every weight zero but b4, p = sigmoid(b4) and dL/db4 = mean(p - y)
    th = np.zeros(mlp.N_PARAMS)
    th[-1] = 0.7
    feat = np.ones((5, 8))
    lab = np.array([1, 0, 1, 1, 0.0])
    g, L = mlp.grad(th, feat, lab, bf16_round=False)
    p = 1 / (1 + np.exp(-0.7))
    assert abs(g[-1] - np.mean(p - lab)) < 1e-15
    assert abs(L - np.mean(-(lab * np.log(p) + (1 - lab) * np.log(1 - p)))) < 1e-12
