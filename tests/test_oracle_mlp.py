"""Pins of the FP64 network reference: finite differences and invariants."""
import numpy as np

from oracle import mlp


def test_backward_matches_finite_differences():
    rng = np.random.Generator(np.random.PCG64(7))
    p = mlp.init_params(1) + 0.01 * rng.normal(size=mlp.NPARAMS)
    X = rng.normal(size=(9, 14))
    T = rng.normal(size=(9, 3))
    loss, g = mlp.loss_grad(p, X, T)
    idx = rng.choice(mlp.NPARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 256 * 14, mlp.NPARAMS - 1, mlp.NPARAMS - 4]])
    for i in idx:
        e = np.zeros(mlp.NPARAMS)
        e[i] = 1e-6
        fd = (mlp.loss_grad(p + e, X, T)[0] - mlp.loss_grad(p - e, X, T)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_residual_has_zero_gradient_and_bf16_rounding():
    p = mlp.init_params(2)
    X = np.random.Generator(np.random.PCG64(3)).normal(size=(5, 14))
    pred, _ = mlp.forward(p, X)
    loss, g = mlp.loss_grad(p, X, pred)
    assert loss == 0.0 and np.all(g == 0.0)
    # bfloat16 keeps 7 mantissa bits: spacing 2^-7 just above 1
    v = np.array([1.0, 1.00390625, 1.01171875, 1.005859375, -3.14159, 0.0])
    r = mlp.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0            # halfway between 1 and 1 + 2^-7: ties go to the even mantissa
    assert r[2] == 1.015625       # halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert r[3] == 1.0078125      # nearest
    assert abs(r[4] - v[4]) <= 2 ** -8 * abs(v[4]) and r[5] == 0.0


def test_bf16_stored_intermediates_change_only_values():
    # with weights, biases and inputs such that every activation and every
    # back-propagated dL/dZ is a small dyadic number (exact in bfloat16),
    # storing the intermediates in BF16 changes nothing; on random data it
    # moves the gradient by about the BF16 spacing
    rng = np.random.Generator(np.random.PCG64(4))
    layers = []
    for n, k in mlp.SIZES:
        W = np.zeros((n, k))
        W[rng.random((n, k)) < 0.02] = 0.5
        layers.append((W, np.where(rng.random(n) < 0.5, 0.5, 0.0)))
    p = mlp.pack(layers)
    X = rng.integers(0, 3, size=(6, 14)).astype(float)
    pred, _ = mlp.forward(p, X)
    T = pred - 1.125                  # dL/dpred = 2 * 1.125 / (3 * 6) = 1/8 in every entry
    l0, g0 = mlp.loss_grad(p, X, T)
    l1, g1 = mlp.loss_grad(p, X, T, store=mlp.bf16_round)
    assert l0 == l1 and np.array_equal(g0, g1) and np.abs(g0).max() > 0
    p = mlp.init_params(6)
    X = rng.normal(size=(40, 14))
    T = rng.normal(size=(40, 3))
    _, g0 = mlp.loss_grad(p, X, T)
    _, g1 = mlp.loss_grad(p, X, T, store=mlp.bf16_round)
    assert 0 < np.linalg.norm(g1 - g0) <= 2e-2 * np.linalg.norm(g0)
