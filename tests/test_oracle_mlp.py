"""Pins of the FP64 surrogate-network oracle (no GPU)."""
import math

import numpy as np
import pytest

from oracle import mlp as M
from paper_1912_05494_gb300 import scenes as S


def targets(rng, nb):
    y = np.zeros((nb, M.N_TARGET))
    y[:, 0] = rng.uniform(0.2, 0.9, nb)
    y[:, 1] = rng.uniform(0.0, 0.5, nb)
    y[:, 2:10] = rng.dirichlet(np.full(8, 0.5), nb)
    y[:, 10:18] = rng.dirichlet(np.full(8, 0.5), nb)
    return y


def small_problem(seed=0, nb=16):
    rng = np.random.default_rng(seed)
    B, params = S.surrogate_init(seed)
    x = rng.uniform(0, 1, (nb, 7))
    return B, params, M.features(x, B), targets(rng, nb)


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
    """Targets a network of this shape can reach: T, R and histograms of a two-lobe mixture
    whose parameters vary smoothly with the inputs."""
    rng = np.random.default_rng(5)
    B, params = S.surrogate_init(5)
    x = rng.uniform(0, 1, (512, 7))
    y = np.zeros((512, M.N_TARGET))
    y[:, 0] = 0.2 + 0.6 * x[:, 0]
    y[:, 1] = 0.1 * x[:, 5]
    y[:, 2:10] = M.lobe_mass(0.3 + 0.4 * x[:, 3], np.exp(8 + 2 * x[:, 2]), np.exp(1 + x[:, 1]))[0]
    y[:, 10:18] = M.lobe_mass(0.8 - 0.3 * x[:, 4], np.exp(10 - x[:, 6]), np.exp(2 * x[:, 0]))[0]
    f = M.features(x, B)
    opt = M.Adam(params, lr=3e-3)
    first, _ = M.loss_and_grads(params, f, y)
    for _ in range(150):
        loss, g = M.loss_and_grads(params, f, y)
        params = opt.step(params, g)
    assert loss < 0.2 * first


# ----------------------------------------------------------------------------- lobe head
def test_vmf_mass_closed_forms():
    a = M.BIN_A
    F, _ = M.vmf_cdf(a, 3.0)
    assert F[0] == 0.0 and abs(F[-1] - 1.0) < 1e-15 and np.all(np.diff(F) > 0)
    # kappa -> 0: the uniform distribution on the sphere, whose cap within angle alpha has
    # area fraction (1 - cos alpha) / 2
    F, _ = M.vmf_cdf(a, 1e-7)
    assert np.allclose(F, a / 2.0, atol=1e-6)
    # large kappa: 1 - exp(-kappa a) (the normaliser's exp(-2 kappa) is below double precision)
    F, _ = M.vmf_cdf(a, 400.0)
    assert np.allclose(F, 1.0 - np.exp(-400.0 * a), atol=1e-15)
    # derivative in kappa against central differences
    for k in (0.3, 5.0, 2000.0):
        _, dF = M.vmf_cdf(a[1:-1], k)
        h = 1e-6 * k
        fd = (M.vmf_cdf(a[1:-1], k + h)[0] - M.vmf_cdf(a[1:-1], k - h)[0]) / (2 * h)
        assert np.allclose(dF, fd, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("kappa", [2.0, 60.0])
def test_vmf_mass_against_rejection_sampling(kappa):
    """Directions uniform on the sphere accepted with probability exp(kappa (cos - 1)) follow
    vMF(kappa); their deflection histogram must match the bin masses within 4 sigma."""
    rng = np.random.default_rng(int(kappa))
    want = 200_000
    cos_acc = []
    got = 0
    while got < want:
        v = rng.normal(size=(2_000_000, 3))
        c = v[:, 2] / np.linalg.norm(v, axis=1)
        keep = rng.uniform(size=c.size) < np.exp(kappa * (c - 1.0))
        cos_acc.append(c[keep])
        got += int(keep.sum())
    c = np.concatenate(cos_acc)[:want]
    edges_cos = np.cos(np.radians(M.BIN_EDGES_DEG))
    frac = np.array([np.mean((c <= edges_cos[b]) & (c > edges_cos[b + 1]) | ((b == 0) & (c == 1.0)))
                     for b in range(M.N_BINS)])
    m = M.lobe_mass(np.array([1.0]), np.array([kappa]), np.array([1.0]))[0][0]
    sig = np.sqrt(m * (1 - m) / want)
    assert np.all(np.abs(frac - m) <= 4 * sig + 1e-12), (frac, m)


def test_lobe_mass_is_a_partition_and_mixes_linearly():
    w = np.array([0.0, 0.3, 1.0])
    k1, k2 = np.full(3, 5000.0), np.full(3, 3.0)
    m, dm_w, _, _ = M.lobe_mass(w, k1, k2)
    assert np.allclose(m.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(m[1], 0.3 * m[2] + 0.7 * m[0], atol=1e-15)
    assert np.allclose(dm_w[0], m[2] - m[0], atol=1e-15)


def test_head_maps_outputs():
    z = np.zeros((1, 16))
    z[0, 3], z[0, 7] = 100.0, -100.0
    p = M.head(z)
    assert np.allclose(p[0, [0, 1, 2, 5]], 0.5)
    assert p[0, 3] == M.LK_MAX and p[0, 7] == M.LK_MIN
    assert p[0, 4] == M.LK_OFFSET[1] and p[0, 6] == M.LK_OFFSET[0]
