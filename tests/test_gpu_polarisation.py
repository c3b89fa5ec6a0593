"""Polarisation-resolved thin-slab series and finely tabulated optical constants, GPU (through
the C ABI) against the FP64 oracle.

Sec. 2 / Eq. 1 give the glass by its complex index n(lambda) + i k(lambda), measured as
spectra.  With the scene flag slab_polarisation = 1 the thin-slab series runs for s and p
light separately and the two results are averaged.  The tables here are sampled every 1 nm
and carry structure narrower than the 5-nm render grid (a 3-nm ripple of n, 1.5-nm wide
absorption lines in k), rendered at the 81 grid wavelengths and at 16 off-grid ones (four beside the lines): both
sides interpolate the same tables.  Bars as in the other parity tests: per-pixel relative
error 1e-4 (deterministic), relative image error 1e-3 and 0.1 % branch flips (Monte Carlo),
2e-6 absolute for the optics module.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1912_05494_gb300 import scenes as S  # noqa: E402
from test_gpu_parity import mc_compare, render_gpu  # noqa: E402


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd as m
    assert torch.cuda.is_available()
    return m


def test_optics_module_per_polarisation(sdd, orc):
    rng = np.random.default_rng(12)
    n = 20000
    cos_i = np.concatenate([rng.uniform(0, 1, n - 6), [1.0, 1e-3, 1e-4, 0.05, 0.0625, 0.07]]).astype(np.float32)
    nre = rng.uniform(1.45, 1.65, n).astype(np.float32)
    k = np.exp(rng.uniform(np.log(1e-8), np.log(1e-4), n)).astype(np.float32)
    d = rng.uniform(2e-3, 5e-3, n).astype(np.float32)
    lam = rng.uniform(380, 780, n).astype(np.float32)
    t = [torch.from_numpy(x).cuda() for x in (cos_i, nre, k, d, lam)]
    out = {}
    for pol in (0, 1):
        R, Rs, Ts = (torch.empty(n, device="cuda") for _ in range(3))
        sdd.sdd_eval_optics(*t, R, Rs, Ts, slab_polarisation=pol)
        Rs_ref, Ts_ref = orc.slab(cos_i, nre, k, d, lam, pol=pol)
        assert np.max(np.abs(Rs.cpu().numpy() - Rs_ref)) < 2e-6, pol
        assert np.max(np.abs(Ts.cpu().numpy() - Ts_ref)) < 2e-6, pol
        out[pol] = Ts.cpu().numpy()
    assert np.max(np.abs(out[1] - out[0])) > 1e-2  # the two series do differ at oblique incidence


def fine_tables(seed=0):
    """1-nm tables 370-790 nm: n with a 3-nm ripple, k with four 1.5-nm absorption lines."""
    lam = np.arange(370.0, 791.0, 1.0)
    rng = np.random.default_rng(seed)
    n = 1.52 + 0.0042 / (lam * 1e-3) ** 2 + 0.002 * np.sin(2 * math.pi * lam / 3.0 + rng.uniform(0, 6))
    k = np.full_like(lam, 1e-6)
    for c in (431.3, 522.7, 589.1, 655.9):
        k += 4e-5 * np.exp(-0.5 * ((lam - c) / 0.75) ** 2)
    sky = 0.6 + 0.4 * np.cos(lam / 37.0) ** 2
    return lam, n, k, sky


def slab_over_floor(pol, seed=0):
    """A horizontal 20 x 20 m thin slab at z = 0 over a Lambertian floor at z = -1, lit by an
    upper-hemisphere sky and a sun at 35 degrees, all tables on the 1-nm grid."""
    lam, n, k, sky = fine_tables(seed)
    v = np.array([[-10, -10, 0], [10, -10, 0], [10, 10, 0], [-10, 10, 0],
                  [-30, -30, -1], [30, -30, -1], [30, 30, -1], [-30, 30, -1]], np.float32)
    idx = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.uint32)
    elev = math.radians(35.0)
    return S.SceneData(
        vertices=v, indices=idx, tri_material=np.array([0, 0, 1, 1], np.uint16),
        mat_kind=np.array([S.MAT_SLAB, S.MAT_DIFFUSE], np.int32),
        mat_thickness=np.array([4e-3, 0.0], np.float32),
        table_nm=lam.astype(np.float32),
        mat_n=np.stack([n, np.ones_like(n)]).astype(np.float32),
        mat_k=np.stack([k, np.zeros_like(k)]).astype(np.float32),
        mat_albedo=np.stack([np.zeros_like(n), np.full_like(n, 0.5)]).astype(np.float32),
        sky=sky.astype(np.float32), sky_mode=1,
        sun_dir=np.array([0.0, -math.cos(elev), math.sin(elev)], np.float32), sun_half_angle=math.radians(0.2665),
        sun=(2000.0 * sky).astype(np.float32), ray_eps=1e-5, slab_polarisation=pol)


def render_lambdas():
    off = np.random.default_rng(4).uniform(381.0, 779.0, 12)
    lines = np.array([431.0, 522.9, 589.4, 655.5])  # within 0.4 nm of the absorption lines
    return np.concatenate([S.SPECTRAL_GRID_81, off, lines]).astype(np.float32)


@pytest.mark.parametrize("pol", [0, 1])
def test_oblique_slab_fine_tables_deterministic(sdd, orc, pol):
    """Pinhole view of the slab from 1.5 m at 50 degrees (incidence ~25-75 degrees across the
    frame): the reflected sky and the sunlit floor seen through the slab, split to depth 6,
    97 wavelengths; per-pixel relative error <= 1e-4 against the oracle."""
    sc = slab_over_floor(pol)
    th = math.radians(50.0)
    cam = S.CameraData(pos=(0.0, -1.5 * math.sin(th), 1.5 * math.cos(th)), look_at=(0.0, 0.0, 0.0),
                       up=(0.0, 0.0, 1.0), vfov_deg=50.0, width=32, height=24)
    spec = S.RenderSpec(lambda_nm=render_lambdas(), spp=1, seed=0, max_depth=6, mode=0)
    h = sdd.SceneHandle(sc)
    gpu, _ = render_gpu(sdd, h, cam, spec)
    ref, _, _ = orc.OracleScene(sc).render(cam, spec)
    assert np.all(ref > 0)
    rel = np.abs(gpu - ref) / np.abs(ref)
    assert rel.max() <= 1e-4, rel.max()
    if pol:
        ref0, _, _ = orc.OracleScene(slab_over_floor(0)).render(cam, spec)
        assert np.max(np.abs(ref / ref0 - 1.0)) > 1e-2  # the flag changes the image
    # the absorption lines, finer than the render grid, show where off-grid wavelengths hit them
    lam = spec.lambda_nm
    near = np.min(np.abs(lam[:, None] - np.array([431.3, 522.7, 589.1, 655.9])[None, :]), axis=1) < 0.8
    assert near.any()


@pytest.mark.parametrize("batched,bundle", [(0, 1), (2, 14)])
def test_nave_per_polarisation_matches_oracle(sdd, orc, batched, bundle):
    """The nave (thin-slab tiles, sun NEE through them) with the per-polarisation series, Monte
    Carlo on the same Philox streams: host-driven one wavelength per path, and the benchmarked
    form (graph form, bundles of 14)."""
    sc, cam, spec = S.nave_scene(seed=1)
    sc.slab_polarisation = 1
    cam = S.CameraData(**{**cam.__dict__, "width": 48, "height": 32})
    spec = S.RenderSpec(**{**spec.__dict__, "spp": 2, "bundle": bundle})
    flips, err, path_rel, gpu, ref = mc_compare(sdd, orc, sc, cam, spec, None, batched=batched)
    assert flips <= 1e-3, flips
    assert err <= 1e-3, err
