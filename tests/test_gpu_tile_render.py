"""Heterogeneous tiles inside the renderer (GPU, through the C ABI).

* Brute-force form: every tile hit traces one ray through the tile's height field and
  bubbles on the tile stream; compared path by path with the FP64 oracle on the same Philox
  streams (Monte Carlo bars: relative image error <= 1e-3, branch flips <= 0.1 %).
* Network form: tile hits are queued and shaded from the BTDF network's prediction.  It
  draws different random numbers, so it is compared with brute-force images on 8 x 8 block
  averages (relative error sum|a - b| / sum|b|), against the noise floor of two brute-force
  renders with different seeds, and against the thin-slab stand-in that ignores the tiles'
  heterogeneity (the gain the network brings).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1912_05494_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd as m
    return m


def rel_err(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def blocks(a, cam, b=8):
    img = a.reshape(cam.height, cam.width, -1).sum(-1)
    H, W = cam.height // b, cam.width // b
    return img[:H * b, :W * b].reshape(H, b, W, b).mean((1, 3))


def render(sdd, h, cam, spec, paths=False, **kw):
    n = cam.width * cam.height
    out = torch.empty((n, spec.n_lambda), device="cuda")
    pr = ph = None
    if paths:
        pr = torch.empty((n, spec.spp, spec.n_lambda), device="cuda")
        ph = torch.empty((n, spec.spp, spec.n_lambda), device="cuda", dtype=torch.int32)
    sdd.sdd_render(h.h, cam, spec, out, None, path_radiance_out=pr, path_hash_out=ph, **kw)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.float64)
    if paths:
        return res, pr.cpu().numpy().astype(np.float64), ph.cpu().numpy().view(np.uint32)
    return res


def slab_stand_in(sc):
    """The same scene with every heterogeneous tile replaced by a uniform thin slab of its
    mean thickness and optical constants."""
    sc2 = S.SceneData(**sc.__dict__)
    sc2.mat_kind = np.where(sc.mat_kind == S.MAT_TILE, S.MAT_SLAB, sc.mat_kind).astype(np.int32)
    sc2.tiles, sc2.mat_tile = None, None
    return sc2


@pytest.mark.parametrize("n_sub", [1, 2])
def test_brute_force_tiles_match_the_oracle(sdd, orc, n_sub):
    sc, cam, spec = S.tile_room_scene(width=48, height=32, spp=4)
    h = sdd.SceneHandle(sc, n_subdomains=n_sub)
    gpu, gp, gh = render(sdd, h, cam, spec, paths=True)
    ref, rp, rh = orc.OracleScene(sc).render(cam, spec, want_paths=True)
    flips = float(np.mean(gh != rh))
    assert flips <= 1e-3, flips
    assert rel_err(gpu, ref) <= 1e-3
    same = gh == rh
    path_rel = np.abs(gp[same] - rp[same]) / (np.abs(rp[same]) + 1e-6 * np.abs(rp).mean() + 1e-30)
    assert np.quantile(path_rel, 0.999) < 1e-3
    # the tiles matter: the thin-slab stand-in gives a visibly different image
    slab = orc.OracleScene(slab_stand_in(sc)).render(cam, spec)[0]
    assert rel_err(slab, ref) > 0.05


def test_network_form_requires_a_network(sdd):
    sc, cam, spec = S.tile_room_scene(width=8, height=8, spp=1)
    h = sdd.SceneHandle(sc)
    out = torch.empty((64, spec.n_lambda), device="cuda")
    with pytest.raises(RuntimeError):
        sdd.sdd_render(h.h, cam, spec, out, None, use_surrogate=1)


@pytest.fixture(scope="module")
def trained(sdd):
    from paper_1912_05494_gb300 import surrogate as SG
    tiles, tn, tk = S.tile_set(2, 16)  # the room's tile set
    ts = sdd.TileSetHandle(tiles)
    net, hist, held = SG.train_for_tileset(ts.h, tiles, tn, tk, n_samples=1 << 20, steps=8000, rays=256)
    return net, hist, held


def test_network_gain_over_the_thin_slab(sdd, trained):
    """Sky-lit room, 96 x 64: at 1024 spp (brute-force noise floor ~0.2 % on 8 x 8 block
    averages) the network form stays within 1 % of brute force, where the thin-slab stand-in
    is off by more than twenty times as much."""
    net, hist, _ = trained
    assert np.mean(hist[-50:]) < 0.2 * hist[0]
    sc, cam, spec = S.tile_room_scene(width=96, height=64, spp=1024)
    sc.sun = np.zeros_like(sc.sun)
    h = sdd.SceneHandle(sc)
    bf = render(sdd, h, cam, spec)
    bf2 = render(sdd, h, cam, S.RenderSpec(**{**spec.__dict__, "seed": spec.seed + 97}))
    net_img = render(sdd, h, cam, spec, use_surrogate=1, surrogate=net)
    slab = render(sdd, sdd.SceneHandle(slab_stand_in(sc)), cam, spec)
    noise = rel_err(blocks(bf2, cam), blocks(bf, cam))
    e_net = rel_err(blocks(net_img, cam), blocks(bf, cam))
    e_slab = rel_err(blocks(slab, cam), blocks(bf, cam))
    print(f"room, sky only, 1024 spp: network {e_net:.4f}, thin slab {e_slab:.4f}, noise floor {noise:.4f}")
    assert noise < 0.004, noise
    assert e_net < 0.01, (e_net, noise)
    assert e_net < 0.05 * e_slab, (e_net, e_slab)


def test_network_form_with_the_sun_is_within_the_noise_floor(sdd, trained):
    """Sun and sky: the sun seen through rough tiles is a caustic found only by paths that
    happen to leave a tile toward the disc, so brute-force images carry heavy-tailed noise.
    Against a 512-spp brute-force reference, the network form at 64 spp must stay within
    twice the error of a brute-force render at 64 spp (another seed) plus 1 %, and keep the
    image's mean within 15 %."""
    net, _, _ = trained
    sc, cam, spec = S.tile_room_scene(width=96, height=64, spp=64)
    h = sdd.SceneHandle(sc)
    ref = render(sdd, h, cam, S.RenderSpec(**{**spec.__dict__, "spp": 512}))
    bf = render(sdd, h, cam, S.RenderSpec(**{**spec.__dict__, "seed": spec.seed + 97}))
    net_img = render(sdd, h, cam, spec, use_surrogate=1, surrogate=net)
    noise = rel_err(blocks(bf, cam), blocks(ref, cam))
    e_net = rel_err(blocks(net_img, cam), blocks(ref, cam))
    assert e_net <= 2.0 * noise + 0.01, (e_net, noise)
    assert abs(net_img.mean() / ref.mean() - 1.0) < 0.15


def test_network_form_is_deterministic_and_counts_launches(sdd, trained):
    net, _, _ = trained
    sc, cam, spec = S.tile_room_scene(width=32, height=24, spp=4)
    h = sdd.SceneHandle(sc)
    a = render(sdd, h, cam, spec, use_surrogate=1, surrogate=net)
    b = render(sdd, h, cam, spec, use_surrogate=1, surrogate=net)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("use_net", [False, True])
def test_batched_form_is_bit_identical_with_tiles(sdd, trained, use_net):
    """The persistent form (one launch per wave for brute-force tiles; two per generation
    around the fused tile shading for the network) runs the same per-ray code: images and
    path hashes equal the host-driven form's bit for bit, frame after frame."""
    net = trained[0] if use_net else None
    sc, cam, spec = S.tile_room_scene(width=40, height=24, spp=4)
    h = sdd.SceneHandle(sc)
    kw = {"use_surrogate": 1, "surrogate": net} if use_net else {}
    a, _, ha = render(sdd, h, cam, spec, paths=True, **kw)
    b, _, hb = render(sdd, h, cam, spec, paths=True, batched=1, wave_paths=40 * 24 * 81, **kw)
    c, _, hc = render(sdd, h, cam, spec, paths=True, batched=1, wave_paths=40 * 24 * 81, **kw)
    assert np.array_equal(a, b) and np.array_equal(ha, hb)
    assert np.array_equal(b, c) and np.array_equal(hb, hc)
    st = sdd.sdd_get_stats(h.h)
    assert st["launches_persistent"] >= 1
    if use_net:
        assert st["launches_tile"] > 0


@pytest.mark.parametrize("use_net", [False, True])
def test_bundled_batched_form_is_bit_identical_with_tiles(sdd, trained, use_net):
    """Spectral bundles of 8 through heterogeneous tiles: every member leaves a tile on its own
    ray (its own brute-force trace, or its own network prediction).  With the network the
    batched form equals the host-driven one bit for bit (the tile shading is one kernel for
    both).  The brute-force tile tracer is inlined into differently register-bounded kernels
    in the two forms, and the compiler may then contract its arithmetic differently, so there
    the paths agree up to float rounding: at most 0.1 % of branch decisions flip."""
    net = trained[0] if use_net else None
    sc, cam, spec = S.tile_room_scene(width=40, height=24, spp=4)
    spec = S.RenderSpec(**{**spec.__dict__, "bundle": 8})
    h = sdd.SceneHandle(sc)
    kw = {"use_surrogate": 1, "surrogate": net} if use_net else {}
    a, pa, ha = render(sdd, h, cam, spec, paths=True, **kw)
    b, pb, hb = render(sdd, h, cam, spec, paths=True, batched=1, **kw)
    if use_net:
        assert np.array_equal(a, b) and np.array_equal(ha, hb)
    else:
        flips = float(np.mean(ha != hb))
        assert flips <= 1e-3, flips
        assert rel_err(a, b) <= 1e-3, rel_err(a, b)


def test_bundled_network_form_matches_brute_force(sdd, trained):
    """Sky-lit room as in the gain test, with bundles of 9 in the network form against the
    unbundled brute-force image: block averages within 1 %, like the unbundled network form.
    The wavelengths of a bundle share their draws, so its noise is correlated across the
    spectrum and the wavelength-summed blocks are noisier at equal spp: the bundled render
    takes 2048 spp to the reference's 1024."""
    net, _, _ = trained
    sc, cam, spec = S.tile_room_scene(width=96, height=64, spp=1024)
    sc.sun = np.zeros_like(sc.sun)
    h = sdd.SceneHandle(sc)
    bf = render(sdd, h, cam, spec)
    net_img = render(sdd, h, cam, S.RenderSpec(**{**spec.__dict__, "bundle": 9, "spp": 2048}), use_surrogate=1,
                     surrogate=net, batched=1)
    e_net = rel_err(blocks(net_img, cam), blocks(bf, cam))
    print(f"room, sky only, bundles of 9: network {e_net:.4f}")
    assert e_net < 0.01, e_net
