"""Training the tile-BTDF network on the GPU.

Data come from the brute-force tile tracer (``sdd_tile_generate``): each query
(cos theta_in, phi_in, lambda, tile) is traced with ``rays`` rays through the tile's height
field and bubbles, and the per-query statistics (T, R, and the deflection-angle histograms of
the transmitted and reflected weight) are the training targets.  Training is one
``sdd_surrogate_train`` call: Adam on minibatches drawn by a seeded permutation of the
rows; everything stays on the device.
"""
from __future__ import annotations

import numpy as np

from . import scenes as S
from . import sdd

# Columns of the tracer's per-query statistics that the network is trained on: T, R and the
# deflection-angle bin fractions of the transmitted and reflected weight (8 each).
TARGET_COLUMNS = [0, 1] + list(range(4, 20))


def raw_inputs(q, tiles):
    """The network's seven raw inputs per query: signed cos theta_in (< 0 through the rough back face),
    phi_in, lambda (nm), mean thickness (m), bubble density (1/m^3), n, k."""
    d_mean = np.array([t["d_mean"] for t in tiles], np.float32)[q["tile"]]
    rho = np.array([t["rho"] for t in tiles], np.float32)[q["tile"]]
    return np.column_stack([q["cos_in"], q["phi_in"], q["lambda_nm"], d_mean, rho, q["n"], q["k"]]).astype(np.float32)


def generate(tileset_h, tiles, tile_n, tile_k, n_samples, seed=3, rays=256, max_events=64, device="cuda"):
    """Trace ``n_samples`` seeded queries over the tile set; returns (raw [n, 7], targets [n, 18])
    as device tensors."""
    import torch
    q = S.tile_queries(seed, n_samples, len(tiles), tile_n, tile_k)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device)
    stats = torch.empty((n_samples, 20), device=device)
    sdd.sdd_tile_generate(tileset_h, dev(q["cos_in"]), dev(q["phi_in"]), dev(q["lambda_nm"]), dev(q["n"]),
                          dev(q["k"]), dev(q["tile"]), rays, seed, max_events, stats)
    return dev(raw_inputs(q, tiles)), stats[:, TARGET_COLUMNS].contiguous()


def train(net, raw, y, steps, batch=65536, lr=1e-3, seed=4):
    """Adam steps on minibatches of the device-resident samples (sdd_surrogate_train: the
    whole loop, minibatch gathering included, runs in the library); returns the loss history
    (one value per step)."""
    return [float(v) for v in net.train(raw, y, steps, batch=batch, lr=lr, seed=seed)]


def train_for_tileset(tileset_h, tiles, tile_n, tile_k, n_samples=1 << 20, steps=2000, rays=256, batch=65536,
                      lr=1e-3, data_seed=3, init_seed=4):
    """Generate data for a tile set and train a freshly initialised network on it; returns
    (network, loss history, held-out (raw, targets))."""
    B, params = S.surrogate_init(init_seed)
    raw, y = generate(tileset_h, tiles, tile_n, tile_k, n_samples, seed=data_seed, rays=rays)
    net = sdd.Surrogate(B, params, max_batch=max(batch, 8192))
    hist = train(net, raw, y, steps, batch=batch, lr=lr, seed=init_seed)
    held = generate(tileset_h, tiles, tile_n, tile_k, 1 << 14, seed=data_seed + 1000, rays=rays)
    return net, hist, held
