"""Pins of the FP64 surrogate-network oracle (no GPU)."""
import math

import numpy as np

from oracle import mlp as M
from paper_1912_05494_gb300 import scenes as S


def small_problem(seed=0, nb=16):
    rng = np.random.default_rng(seed)
    B, params = S.surrogate_init(seed)
    x = rng.uniform(0, 1, (nb, 7))
    y = rng.uniform(0, 1, (nb, 6))
    return B, params, M.features(x, B), y


def test_backprop_matches_central_differences():
    B, params, f, y = small_problem()
    # give the biases non-zero values so their gradients are exercised away from the start
    params = [(W, np.random.default_rng(1 + i).normal(0, 0.1, b.shape)) for i, (W, b) in enumerate(params)]
    _, grads = M.loss_and_grads(params, f, y)
    rng = np.random.default_rng(3)
    h = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = M.loss_and_grads(params, f, y)
                arr[idx] = old - h
                lm, _ = M.loss_and_grads(params, f, y)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][which][idx]
                assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (li, which, idx, fd, an)


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-13)      # Phi(x) + Phi(-x) = 1
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    assert np.allclose(M.gelu(np.array([8.0])), 8.0, rtol=1e-12)
    g = (M.gelu(x + 1e-6) - M.gelu(x - 1e-6)) / 2e-6
    assert np.allclose(g, M.gelu_grad(x), atol=1e-8)


def test_features_are_unit_fourier_pairs_plus_inputs():
    rng = np.random.default_rng(2)
    B, _ = S.surrogate_init(2)
    x = rng.uniform(0, 1, (50, 7))
    f = M.features(x, B)
    assert f.shape == (50, 48)
    assert np.allclose(f[:, :16] ** 2 + f[:, 16:32] ** 2, 1.0)
    assert np.array_equal(f[:, 32:39], x) and np.all(f[:, 39:] == 0)


def test_first_adam_step_moves_each_weight_by_lr():
    B, params, f, y = small_problem(nb=64)
    _, grads = M.loss_and_grads(params, f, y)
    opt = M.Adam(params, lr=1e-3)
    new = opt.step(params, grads)
    for (W0, b0), (W1, b1), (gW, gb) in zip(params, new, grads):
        big = np.abs(gW) > 1e-6  # then |m_hat / sqrt(v_hat)| = 1 up to eps
        assert np.allclose((W0 - W1)[big], 1e-3 * np.sign(gW[big]), rtol=1e-2, atol=0)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(5)
    B, params = S.surrogate_init(5)
    x = rng.uniform(0, 1, (512, 7))
    y = np.stack([0.2 + 0.6 * x[:, 0], 0.1 * x[:, 5], x[:, 3], np.full(512, 0.9), 0.5 * x[:, 1], x[:, 2]], axis=1)
    f = M.features(x, B)
    opt = M.Adam(params, lr=3e-3)
    first, _ = M.loss_and_grads(params, f, y)
    for _ in range(150):
        loss, g = M.loss_and_grads(params, f, y)
        params = opt.step(params, g)
    assert loss < 0.2 * first
