"""The tile-BTDF surrogate on BF16 tensor cores against the FP64 oracle network.

Tolerances (BF16 weights and activations carry 8 significant bits, ~0.4 % per value):
forward predictions within 2e-2 absolute for the probabilities (T, R, lobe weights) and 6e-2
for the log concentrations (values up to ~14); loss within 2 % relative; gradients within 5 %
relative L2 per tensor (the oracle runs on the same BF16-rounded weights in FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp as M  # noqa: E402
from paper_1912_05494_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd as m
    return m


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def raw_inputs(seed, n):
    rng = np.random.default_rng(seed)
    return np.column_stack([rng.uniform(0.01, 1, n) * rng.choice([-1.0, 1.0], n), rng.uniform(0, 2 * np.pi, n), rng.uniform(380, 780, n),
                            rng.uniform(2.5e-3, 4.5e-3, n), rng.uniform(5e9, 1.5e10, n), rng.uniform(1.5, 1.6, n),
                            np.exp(rng.uniform(np.log(1e-7), np.log(1e-5), n))]).astype(np.float32)


def targets(rng, n):
    """T, R and two histograms (Dirichlet rows) per side."""
    y = np.zeros((n, M.N_TARGET), np.float32)
    y[:, 0] = rng.uniform(0.2, 0.9, n)
    y[:, 1] = rng.uniform(0.0, 0.5, n)
    y[:, 2:10] = rng.dirichlet(np.full(8, 0.5), n)
    y[:, 10:18] = rng.dirichlet(np.full(8, 0.5), n)
    return y


def close_predictions(a, b):
    prob = [0, 1, 2, 5]
    logk = [3, 4, 6, 7]
    return np.max(np.abs(a[:, prob] - b[:, prob])) < 2e-2 and np.max(np.abs(a[:, logk] - b[:, logk])) < 6e-2


def oracle_params(params):
    return [(bf16(W), np.asarray(b, np.float64)) for W, b in params]


def oracle_features(raw, B):
    x = M.normalise_inputs(*[raw[:, i].astype(np.float64) for i in range(7)])
    return M.features(x, B)


@pytest.mark.parametrize("n", [1000, 4096 + 37])
def test_gradients_match_the_oracle(sdd, n):
    B, params = S.surrogate_init(4)
    rng = np.random.default_rng(1)
    params = [(W, rng.normal(0, 0.05, b.shape)) for W, b in params]
    raw = raw_inputs(2, n)
    y = targets(rng, n)
    net = sdd.Surrogate(B, params, max_batch=8192)
    loss, g = net.gradients(torch.from_numpy(raw).cuda(), torch.from_numpy(y).cuda())
    lo, go = M.loss_and_grads(oracle_params(params), oracle_features(raw, B), y.astype(np.float64))
    assert abs(loss / lo - 1) < 2e-2, (loss, lo)
    gg = sdd.unflatten_params(g)
    for li, ((gW, gb), (oW, ob)) in enumerate(zip(gg, go)):
        for a, b in ((gW, oW), (gb, ob)):
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel < 5e-2, (li, rel)


def test_inference_matches_the_oracle(sdd):
    B, params = S.surrogate_init(7)
    raw = raw_inputs(3, 3000)
    net = sdd.Surrogate(B, params, max_batch=1024)  # several internal batches
    out = torch.empty((3000, 8), device="cuda")
    net.infer(torch.from_numpy(raw).cuda(), out)
    _, _, p = M.forward(oracle_params(params), oracle_features(raw, B))
    assert close_predictions(out.cpu().numpy(), p)


def test_adam_steps_match_the_oracle(sdd):
    B, params = S.surrogate_init(9)
    raw = raw_inputs(4, 2048)
    y = targets(np.random.default_rng(5), 2048)
    net = sdd.Surrogate(B, params, max_batch=2048)
    r, t = torch.from_numpy(raw).cuda(), torch.from_numpy(y).cuda()
    for _ in range(3):
        net.train_step(r, t, lr=1e-3)
    p_gpu = sdd.unflatten_params(net.params())
    opt = M.Adam(params, lr=1e-3)
    p_ora = [(np.asarray(W, np.float64), np.asarray(b, np.float64)) for W, b in params]
    f = oracle_features(raw, B)
    g_first = None
    for _ in range(3):
        _, g = M.loss_and_grads([(bf16(W), b) for W, b in p_ora], f, y.astype(np.float64))
        g_first = g if g_first is None else g_first
        p_ora = opt.step(p_ora, g)
    for (gW, gb), (oW, ob), (W0, b0), (g0, _) in zip(p_gpu, p_ora, params, g_first):
        dg, do = gW - W0, oW - W0  # three Adam updates: every coordinate moves by ~lr
        assert np.abs(dg).max() < 4e-3 and np.abs(do).max() < 4e-3
        # Adam normalises each coordinate, so its sign is meaningful only where the gradient
        # stands out of the BF16 noise
        sig = np.abs(g0) > 0.2 * np.sqrt(np.mean(g0 ** 2))
        assert np.mean(np.sign(dg[sig]) == np.sign(do[sig])) > 0.97


def test_training_on_tile_data_reduces_the_loss(sdd):
    from paper_1912_05494_gb300 import surrogate as SG
    tiles, tn, tk = S.tile_set(3, 64)
    ts = sdd.TileSetHandle(tiles)
    raw, y = SG.generate(ts.h, tiles, tn, tk, 65536, seed=6, rays=64)
    B, params = S.surrogate_init(4)
    net = sdd.Surrogate(B, params, max_batch=65536)
    first = net.train_step(raw, y, lr=1e-3)
    for _ in range(300):
        last = net.train_step(raw, y, lr=1e-3)
    assert last < 0.3 * first, (first, last)


def test_native_training_run_matches_single_steps_and_learns(sdd):
    """sdd_surrogate_train with one full-batch minibatch per step is the same Adam update as
    sdd_surrogate_train_step (row order inside the batch only changes FP32 summation order),
    and a longer run on tile data reduces the loss."""
    from paper_1912_05494_gb300 import surrogate as SG
    tiles, tn, tk = S.tile_set(3, 16)
    ts = sdd.TileSetHandle(tiles)
    raw, y = SG.generate(ts.h, tiles, tn, tk, 4096, seed=8, rays=64)
    B, params = S.surrogate_init(4)
    a = sdd.Surrogate(B, params, max_batch=4096)
    b = sdd.Surrogate(B, params, max_batch=4096)
    for _ in range(3):
        a.train_step(raw, y, lr=1e-3)
    losses = b.train(raw, y, steps=3, batch=4096, lr=1e-3, seed=1)
    assert losses.shape == (3,) and np.all(np.isfinite(losses))
    pa, pb = a.params(), b.params()
    assert np.max(np.abs(pa - pb)) < 2e-4  # three Adam steps of ~1e-3; summation order only
    w = b.weights()
    assert len(w) == 4 * b.n_params and np.array_equal(np.frombuffer(w, np.float32), pb)
    a.set_weights(w)
    assert np.array_equal(a.params(), pb)
    hist = b.train(raw, y, steps=200, batch=1024, lr=1e-3, seed=2)
    assert np.mean(hist[-20:]) < 0.5 * hist[0], (hist[0], hist[-20:])


def test_training_is_deterministic(sdd):
    """Gradients are reduced over blocks in a fixed order: two runs from the same weights on
    the same data give the same weights bit for bit."""
    raw = torch.from_numpy(raw_inputs(5, 3000)).cuda()
    y = torch.from_numpy(targets(np.random.default_rng(5), 3000)).cuda()
    B, params = S.surrogate_init(4)
    a = sdd.Surrogate(B, params, max_batch=2048)
    b = sdd.Surrogate(B, params, max_batch=2048)
    la = a.train(raw, y, steps=20, batch=2048, lr=1e-3, seed=3)
    lb = b.train(raw, y, steps=20, batch=2048, lr=1e-3, seed=3)
    assert np.array_equal(a.params(), b.params())
    assert np.allclose(la, lb, rtol=1e-5)
