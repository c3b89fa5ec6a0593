"""Pins of the oracle's heterogeneous-tile tracer (no GPU): closed forms and invariants."""
import math

import numpy as np
import pytest


def flat(G=64, d=0.0035):
    return np.full((G + 1, G + 1), d)


def rays_at(n, cos_in, phi=0.3, seed=0, L=0.1, margin=0.0):
    rng = np.random.default_rng(seed)
    xy = rng.uniform(margin, L - margin, (n, 2))
    st = math.sqrt(1 - cos_in**2)
    d = np.tile([st * math.cos(phi), st * math.sin(phi), -cos_in], (n, 1))
    return xy, d


def slab_closed_form(cos_i, n, k, d, lam):
    th = math.acos(cos_i)
    s, c = math.sin(th), cos_i
    A = n * n - k * k - s * s
    B = math.sqrt(A * A + 4 * n * n * k * k)
    a = math.sqrt(0.5 * (B + A)); b2 = 0.5 * (B - A)
    Rs = (a * a + b2 - 2 * a * c + c * c) / (a * a + b2 + 2 * a * c + c * c)
    st = s * math.tan(th) if c > 0 else 0.0
    Rp = Rs * (a * a + b2 - 2 * a * st + st * st) / (a * a + b2 + 2 * a * st + st * st) if c < 1 else Rs
    R = 0.5 * (Rs + Rp)
    ct = math.sqrt(1 - (s / n) ** 2)
    tau = math.exp(-4 * math.pi * k * d / ct / (lam * 1e-9))
    den = 1 - R * R * tau * tau
    return R + (1 - R) ** 2 * R * tau * tau / den, (1 - R) ** 2 * tau / den


TILE0 = {"d_mean": 0.0035, "amp": 0.0, "rho": 0.0, "seed": 1}


@pytest.mark.parametrize("cos_in", [1.0, 0.7071, 0.3])
def test_flat_bubble_free_tile_is_the_thin_slab(orc, cos_in):
    n, k, d, lam = 1.53, 2e-6, 0.0035, 550.0
    N = 200000
    xy, dirs = rays_at(N, cos_in)
    r = orc.tile_trace(TILE0, flat(d=d), xy, dirs, n, k, lam, px=np.arange(N), sample=0, seed=3)
    T = r["w"][r["side"] == 1].sum() / N
    R = r["w"][r["side"] == 0].sum() / N
    Rs, Ts = slab_closed_form(cos_in, n, k, d, lam)
    se = 0.5 / math.sqrt(N)
    assert abs(T - Ts) < 5 * se and abs(R - Rs) < 5 * se, (T, Ts, R, Rs)
    # straight through and mirror directions exactly
    assert np.allclose(r["dir"][r["side"] == 1], dirs[r["side"] == 1], atol=1e-12)


def test_lossless_tile_conserves_every_ray(orc):
    tile = {"d_mean": 0.0035, "amp": 0.003, "rho": 1e10, "seed": 7}
    h = orc.tile_heights(tile)
    N = 20000
    xy, dirs = rays_at(N, 0.8, seed=1)
    r = orc.tile_trace(tile, h, xy, dirs, 1.52, 0.0, 500.0, px=np.arange(N), sample=0, seed=5)
    ok = r["side"] != 2  # side 2: still inside after 64 interactions (trapped by total reflection)
    assert np.allclose(r["w"][ok], 1.0, atol=1e-12)
    assert ok.mean() > 0.97
    assert np.allclose(np.linalg.norm(r["dir"], axis=1), 1.0, atol=1e-9)
    assert r["bubbles"].mean() > 0.1


def test_bubble_encounters_follow_the_poisson_law(orc):
    """Index-matched glass (n = 1 + 1e-9) leaves rays undeflected, so each crosses the d-thick
    tile once: bubble encounters ~ Poisson(rho * pi E[r^2] * d), P(>= 1) = 1 - exp(-rho sigma d)."""
    rho, d = 1e10, 0.0035  # 1e4 per cm^3
    lo, hi = 10e-6, 100e-6
    sigma = math.pi * (hi**2 - lo**2) / (2 * math.log(hi / lo))
    mean = rho * sigma * d
    assert abs(mean - 0.236) < 0.01  # the worked size: ~0.24 bubble hits per normal pass
    tile = {"d_mean": d, "amp": 0.0, "rho": rho, "seed": 2}
    N = 100000
    xy, dirs = rays_at(N, 1.0, seed=4)
    r = orc.tile_trace(tile, flat(d=d), xy, dirs, 1.0 + 1e-9, 0.0, 550.0, px=np.arange(N), sample=0, seed=9)
    b = r["bubbles"]
    assert abs(b.mean() - mean) < 5 * math.sqrt(mean / N)
    assert abs((b > 0).mean() - (1 - math.exp(-mean))) < 5 * math.sqrt(0.2 / N)
    assert np.all(r["side"] == 1)


@pytest.mark.parametrize("beta_deg", [2.0, 8.0])
def test_wedge_back_face_deviation_is_snell(orc, beta_deg):
    """Planar back face tilted by beta: a ray entering the flat front at normal incidence
    leaves the back face deviated by asin(n sin beta) - beta (thin prism: ~ (n-1) beta)."""
    G, L, n = 64, 0.1, 1.5
    beta = math.radians(beta_deg)
    x = np.arange(G + 1) * L / G
    h = 0.0035 + (x - L / 2)[None, :] * math.tan(beta) * np.ones((G + 1, 1))
    N = 2000
    rng = np.random.default_rng(0)
    xy = np.column_stack([rng.uniform(0.04, 0.06, N), rng.uniform(0.01, 0.09, N)])
    dirs = np.tile([0.0, 0.0, -1.0], (N, 1))
    r = orc.tile_trace(TILE0, h, xy, dirs, n, 0.0, 550.0, px=np.arange(N), sample=0, seed=1)
    direct = (r["side"] == 1) & (r["events"] == 3)  # entry, one glass segment, exit: three draws
    assert direct.mean() > 0.8
    dev = np.arccos(np.clip(-r["dir"][direct, 2], -1, 1))
    want = math.asin(n * math.sin(beta)) - beta
    assert np.allclose(dev, want, atol=1e-9)
    assert abs(want - (n - 1) * beta) < 0.02 * (n - 1) * beta + 1e-4


def test_height_field_is_periodic_and_in_range(orc):
    tile = {"d_mean": 0.0035, "amp": 0.004, "rho": 0.0, "seed": 11}
    h = orc.tile_heights(tile)
    assert np.allclose(h[:, 0], h[:, -1]) and np.allclose(h[0, :], h[-1, :])
    assert h.min() >= 0.002 - 1e-15 and h.max() <= 0.005 + 1e-15
    assert h.std() > 1e-4  # not flat
    flat_tile = orc.tile_heights({"d_mean": 0.0031, "amp": 0.0, "rho": 0.0, "seed": 3})
    assert np.allclose(flat_tile, 0.0031)


def test_tile_samples_statistics(orc):
    tiles = [{"d_mean": 0.0035, "amp": 0.0, "rho": 0.0, "seed": 1}, {"d_mean": 0.003, "amp": 0.003, "rho": 1e10, "seed": 5}]
    hs = np.stack([orc.tile_heights(t) for t in tiles])
    out = orc.tile_samples(tiles, hs, [1.0, 0.9], [0.0, 1.0], [550.0, 600.0], [1.53, 1.52], [2e-6, 5e-6], [0, 1],
                           rays=4000, seed=2)
    Rs, Ts = slab_closed_form(1.0, 1.53, 2e-6, 0.0035, 550.0)
    assert abs(out[0, 0] - Ts) < 0.02 and abs(out[0, 1] - Rs) < 0.02
    assert out[0, 4] == 1.0 and np.all(out[0, 5:12] == 0.0)   # flat: all transmission within 1 degree
    assert out[0, 12] == 1.0                                   # and all reflection specular
    assert out[1, 4] < 0.99 and out[1, 3] > 0.05               # rough, bubbly tile scatters
    for r in range(2):                                         # each side's bins partition its weight
        assert abs(out[r, 4:12].sum() - 1.0) < 1e-12 and abs(out[r, 12:20].sum() - 1.0) < 1e-12


def test_tile_sample_faces(orc):
    """A bubble-free tile entered through either face: a flat one is the thin slab both ways
    (closed form, within Monte Carlo error of 3000 rays), and reflection off the flat front
    face of a rough tile stays specular while its rough back face spreads it."""
    tiles = [{"d_mean": 0.0035, "amp": 0.0, "rho": 0.0, "seed": 1}, {"d_mean": 0.0035, "amp": 0.003, "rho": 0.0, "seed": 9}]
    hs = np.stack([orc.tile_heights(t) for t in tiles])
    out = orc.tile_samples(tiles, hs, [0.8, -0.8, 0.8, -0.8], [0.4] * 4, [550.0] * 4, [1.53] * 4, [2e-6] * 4,
                           [0, 0, 1, 1], rays=3000, seed=4)
    Rs, Ts = slab_closed_form(0.8, 1.53, 2e-6, 0.0035, 550.0)
    for r in (0, 1):
        assert abs(out[r, 0] - Ts) < 0.03 and abs(out[r, 1] - Rs) < 0.03 and out[r, 4] == 1.0
    assert out[2, 12] > out[3, 12] + 0.2   # the flat front face reflects specularly first
