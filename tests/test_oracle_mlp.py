"""Pins for the predictor's oracle (oracle/mlp.py): finite differences of its own loss,
closed-form GELU values, and a sketch identity that reduces to a LAPACK SVD of Omega."""
import math

import numpy as np

from oracle import mlp


def _params(seed=0, scale=0.1):
    g = np.random.default_rng(seed)
    p = g.standard_normal(mlp.N_PARAMS) * scale
    p[mlp.N_TRAINABLE + 35:mlp.N_TRAINABLE + 70] = 1.0 + 0.1 * np.abs(g.standard_normal(35))  # input std
    p[mlp.N_TRAINABLE + 72:] = 1.0 + 0.1 * np.abs(g.standard_normal(2))  # target std
    return p


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu_grad(np.array([0.0])), [0.5], rtol=0, atol=1e-15)
    # GELU(x) = x Phi(x): Phi(1) = 0.841344746068543, Phi(-2) = 0.022750131948179
    np.testing.assert_allclose(mlp.gelu(np.array([1.0, -2.0])), [0.841344746068543, -2 * 0.022750131948179],
                               rtol=1e-13)
    z = np.linspace(-4, 4, 81)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-8,
                               atol=1e-10)


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    p = _params(1)
    X = g.standard_normal((7, 35))
    Y = g.standard_normal((7, 2))
    loss, grad = mlp.loss_and_grad(p, X, Y)
    idx = np.concatenate([g.choice(mlp.N_TRAINABLE, 60, replace=False),
                          np.arange(mlp.N_TRAINABLE - 2, mlp.N_TRAINABLE)])
    h = 1e-6
    for i in idx:
        q = p.copy(); q[i] += h
        lp, _ = mlp.loss_and_grad(q, X, Y)
        q[i] -= 2 * h
        lm, _ = mlp.loss_and_grad(q, X, Y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_forward_destandardizes():
    p = _params(2)
    X = np.random.default_rng(5).standard_normal((4, 35))
    out, cache = mlp.forward(p, X)
    O = cache[-1]
    W1, b1, W2, b2, W3, b3, xmu, xsd, ymu, ysd = mlp.unpack(p)
    np.testing.assert_allclose(out, O * ysd + ymu, rtol=1e-15)


def test_sketch_of_orthonormal_columns_is_svd_of_omega():
    """A = Q (m x n, orthonormal columns, n <= 32): Y = Q Omega has the singular values of
    Omega (n x 32), so the features are the logs of svd(Omega) / (sqrt(32) sqrt(n))."""
    g = np.random.default_rng(7)
    m, n = 90, 20
    Q, _ = np.linalg.qr(g.standard_normal((m, n)))
    f = mlp.sketch_features(Q, seed=11)
    s = np.linalg.svd(mlp.omega(11, n), compute_uv=False)
    ref = math.sqrt(32) * math.sqrt(n)
    np.testing.assert_allclose(f[:n], np.log(s / ref), rtol=0, atol=1e-12)
    assert np.all(f[n:32] < math.log(1e-12))  # the rank-deficient tail is at the rounding level
    np.testing.assert_allclose(f[32:], [0.5 * math.log(n), math.log(m), math.log(n)], atol=1e-12)


def test_sketch_scale_invariance():
    g = np.random.default_rng(8)
    A = g.standard_normal((50, 40))
    f1 = mlp.sketch_features(A, 3)
    f2 = mlp.sketch_features(7.5 * A, 3)
    np.testing.assert_allclose(f2[:32], f1[:32], atol=1e-12)
    np.testing.assert_allclose(f2[32], f1[32] + math.log(7.5), atol=1e-12)


def test_adam_constant_gradient_closed_form():
    """From zero moments with a constant gradient g, the bias corrections make m^ = g and
    v^ = g^2 at every step t, so each update is exactly lr g / (|g| + eps).  A wrong power
    of beta, a missing correction or eps inside the root fails this (g spans 1e-6..10)."""
    g = np.array([0.5, -2.0, 1e-4, -1e-6, 10.0])
    p = np.array([1.0, -1.0, 0.25, 3.0, 0.0])
    m = np.zeros_like(g)
    v = np.zeros_like(g)
    lr = 1e-3
    for t in range(1, 6):
        p_new, m, v = mlp.adam_step(p, m, v, g, t, lr)
        np.testing.assert_allclose(p - p_new, lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        p = p_new


def test_adam_hand_worked_step():
    """One step with nonzero moments, worked by hand: p = 1, m = 0.1, v = 0.01, g = 0.5,
    t = 2, lr = 0.1 gives m = 0.14, v = 0.01024, m^ = 0.14 / 0.19 = 14/19,
    v^ = 0.01024 / 0.001999, update = 0.1 (14/19) / (sqrt(v^) + 1e-8) = 0.0325559858872132."""
    p, m, v = mlp.adam_step(np.array([1.0]), np.array([0.1]), np.array([0.01]), np.array([0.5]), 2, 0.1)
    np.testing.assert_allclose(m, [0.14], rtol=1e-15)
    np.testing.assert_allclose(v, [0.01024], rtol=1e-15)
    np.testing.assert_allclose(p, [1.0 - 0.0325559858872132], rtol=1e-14)


def test_round_bf16_matches_torch_conversion():
    """The oracle's bf16 rounding (used for the sketch's Omega of bf16 operators) against torch's
    round-to-nearest-even conversion, including ties and values near the f32 limits."""
    import torch

    from oracle import mlp

    g = np.random.default_rng(8)
    x = np.concatenate([g.standard_normal(20000).astype(np.float32),
                        np.array([1 + 2**-8, 1 + 3 * 2**-8, -1 - 2**-8, 3e38, -3e38, 1e-38, 0.0], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.round_bf16(x), ref)
