"""Photon maps (Sec. 3.2, Jensen's photon mapping) on the GPU, through the C ABI, against
the FP64 oracle.

Both sides trace the same photons on the same Philox streams (photon i of wavelength l:
counter (i, 0, bounce | photon stream, l)), so the stored photons are compared one by one,
keyed by (wavelength, photon index, diffuse surfaces met before): positions to 1e-4 m (1e-3 m
in the nave, whose coordinates reach ~100 m) and powers to 1e-4 relative for 99.9 % of them
(FP32 against FP64 geometry), with at most
0.2 % of either set unmatched or moved to another surface (decisions that FP32 rounding
flips, and the later stores of those photons).  The hashed grid's
density estimates are checked against the definition (brute force over the same photons)
and against the oracle's estimates over its own photons; renders that take the sun's
caustic and indirect light from the maps are compared path by path as the other Monte Carlo
parity tests are (0.1 % event-hash flips; image error 2e-3, the maps differing by the
photons FP32 decisions moved), one wavelength per path and in spectral bundles; the graph
form equals the host-driven form bit for bit.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1912_05494_gb300 import scenes as S  # noqa: E402
from test_gpu_parity import mean_rel_image_error, render_gpu  # noqa: E402
from test_oracle_pins import box_tris, quad  # noqa: E402

LAMS = np.array([450.0, 550.0, 650.0], np.float32)
CAUSTIC, GLOBAL = 0, 1


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd as m
    assert torch.cuda.is_available()
    return m


def scene_from(tris, kinds, n, k, d, albedo, sun_dir, n_sub=4, sky=0.3):
    v = np.array([p for t in tris for p in t[:3]], np.float32)
    return S.SceneData(
        vertices=v, indices=np.arange(v.shape[0], dtype=np.uint32).reshape(-1, 3),
        tri_material=np.array([t[3] for t in tris], np.uint16), mat_kind=np.array(kinds, np.int32),
        mat_thickness=np.array(d, np.float32), table_nm=LAMS, mat_n=np.array(n, np.float32),
        mat_k=np.array(k, np.float32), mat_albedo=np.array(albedo, np.float32),
        sky=np.full(LAMS.size, sky, np.float32), sky_mode=1, sun_dir=np.asarray(sun_dir, np.float32),
        sun_half_angle=math.radians(0.2665), sun=np.array([1.0e4, 1.1e4, 0.9e4], np.float32), ray_eps=1e-5,
        n_subdomains=n_sub, split_axis=0)


def court():
    """A 6 x 6 m court: Lambertian floor (albedo 0.6) and back wall (0.5); a solid glass
    block 1 cm thick and a 4-mm thin slab 5 cm over the floor, side by side; the sun at an
    oblique azimuth.  Four subdomains along x."""
    tris = quad((-3, -3, 0), (3, -3, 0), (3, 3, 0), (-3, 3, 0), 0)
    tris += quad((-3, 3, 0), (3, 3, 0), (3, 3, 3), (-3, 3, 3), 1)
    tris += box_tris((-2.5, -2.5, 0.05), (-0.2, 2.5, 0.06), 2)
    tris += quad((0.2, -2.5, 0.05), (2.5, -2.5, 0.05), (2.5, 2.5, 0.05), (0.2, 2.5, 0.05), 3)
    glass = S.cauchy_n(LAMS, 1.52, 0.0045)
    ones = np.ones(LAMS.size)
    s = np.array([0.25, -0.55, 0.80])
    return scene_from(tris, [S.MAT_DIFFUSE, S.MAT_DIFFUSE, S.MAT_SOLID, S.MAT_SLAB],
                      [ones, ones, glass, glass], [0 * ones, 0 * ones, [2e-7, 1e-7, 3e-7], [1e-6, 2e-6, 1e-6]],
                      [0, 0, 0, 4e-3], [0.6 * ones, 0.5 * ones, 0 * ones, 0 * ones], s / np.linalg.norm(s))


def keyed(ph, seq=None):
    """{(lam, id, seq): (pos, nrm, power)}; the oracle lists a photon's stores in path order."""
    lam, pid = ph["lam"].astype(np.int64), ph["id"].astype(np.int64)
    if seq is None:
        seq = np.zeros(lam.size, np.int64)
        for i in range(1, lam.size):
            if lam[i] == lam[i - 1] and pid[i] == pid[i - 1]:
                seq[i] = seq[i - 1] + 1
    return {(int(a), int(b), int(c)): i for i, (a, b, c) in enumerate(zip(lam, pid, seq))}


def compare_sets(gph, oph, global_offset=0, moved_at=1e-3):
    """Match GPU and oracle photons by key.  A matched pair whose normals differ or whose
    positions are more than 1 mm apart belongs to a photon path that an FP32 decision moved
    (another facet, an edge, a Fresnel or survival draw at its threshold) and counts with the
    unmatched (moved_at: 1 mm in scenes of a few metres).  Returns (that fraction, position and
    power errors of the other pairs)."""
    g = keyed(gph, gph["seq"].astype(np.int64) - global_offset)
    o = keyed(oph)
    common = sorted(set(g) & set(o))
    n = max(len(g), len(o), 1)
    gi = np.array([g[c] for c in common], np.int64)
    oi = np.array([o[c] for c in common], np.int64)
    if gi.size == 0:
        return (len(g) + len(o)) / n, np.zeros(1), np.zeros(1)
    dpos = np.linalg.norm(gph["pos"][gi].astype(np.float64) - oph["pos"][oi], axis=1)
    same = (np.sum(gph["nrm"][gi] * oph["nrm"][oi], axis=1) > 0.999) & (dpos < moved_at)
    moved = (len(g) + len(o) - 2 * len(common) + 2 * int(np.sum(~same))) / n
    po = np.abs(oph["power"][oi][same])
    dpw = np.abs(gph["power"][gi][same] - oph["power"][oi][same]) / (po + 1e-6 * np.median(po))
    return moved, dpos[same], dpw


def both_maps(sdd, orc, sc, lams, n, seed, center, radius, distance, r, max_depth=16, n_sub=None):
    h = sdd.SceneHandle(sc, n_subdomains=n_sub)
    gm = sdd.PhotonMaps(h.h, lams, n, seed, center, radius, distance, r, max_depth=max_depth)
    om = orc.OracleScene(sc).photon_maps(lams, n, seed, center=center, radius=radius, distance=distance,
                                         gather_radius=r, max_depth=max_depth)
    return h, gm, om


def check_sets(gm, om, min_counts=(1, 1), pos_tol=1e-4, moved_max=2e-3):
    """pos_tol: 1e-4 m where the coordinates (emitter included) stay within ~20 m; FP32
    positions carry ~1e-7 of the coordinates' magnitude per operation, so a scene whose
    coordinates reach ~100 m takes ten times that."""
    for m in (CAUSTIC, GLOBAL):
        gph, oph = gm.photons(m), om.photons(m)
        assert oph["pos"].shape[0] >= min_counts[m], (m, oph["pos"].shape[0])
        assert abs(gph["pos"].shape[0] - oph["pos"].shape[0]) <= 0.002 * oph["pos"].shape[0] + 5, m
        # the caustic map stores a photon before its first diffuse bounce (seq 0); the oracle's
        # per-photon rank counts only the stores of that map, the GPU's seq counts diffuse
        # surfaces met: global photons are stored from the second surface on (seq >= 1)
        moved, dpos, dpw = compare_sets(gph, oph, global_offset=1 if m == GLOBAL else 0, moved_at=10 * pos_tol)
        assert moved <= moved_max, (m, moved)
        assert np.quantile(dpos, 0.999) < pos_tol, (m, np.quantile(dpos, 0.999))
        assert np.quantile(dpw, 0.999) < 1e-4, (m, np.quantile(dpw, 0.999))


@pytest.fixture(scope="module")
def nave():
    return S.nave_scene(seed=1)


@pytest.fixture(scope="module")
def court_maps(sdd, orc):
    return both_maps(sdd, orc, court(), LAMS, 200000, 17, (0.0, 0.0, 0.5), 5.0, 20.0, 0.1)


def test_photon_sets_match_the_oracle(court_maps):
    _, gm, om = court_maps
    check_sets(gm, om, min_counts=(50000, 30000))


def floor_and_wall_queries(n_side=24):
    g = (np.arange(n_side) + 0.5) / n_side * 5.6 - 2.8
    x, y = np.meshgrid(g, g)
    floor = np.column_stack([x.ravel(), y.ravel(), np.zeros(x.size)])
    xw, zw = np.meshgrid(g, (np.arange(8) + 0.5) / 8 * 2.8)
    wall = np.column_stack([xw.ravel(), np.full(xw.size, 3.0), zw.ravel()])
    pts = np.vstack([floor, wall, floor[:64]])
    nrm = np.vstack([np.tile([0, 0, 1.0], (floor.shape[0], 1)), np.tile([0, -1.0, 0], (wall.shape[0], 1)),
                     np.tile([0, 0, -1.0], (64, 1))])  # the last 64 look at the floor from below
    lam = (np.arange(pts.shape[0]) % LAMS.size).astype(np.int32)
    return pts, nrm, lam


def brute_gather(ph, x, nrm, lam, r):
    """The density estimate's definition over a photon list, FP32 distances as the kernel."""
    p = ph["pos"].astype(np.float32)
    out = np.zeros(x.shape[0])
    for i in range(x.shape[0]):
        d = p - x[i].astype(np.float32)
        d2 = (d * d).sum(axis=1, dtype=np.float32)
        sel = (d2 < np.float32(r) * np.float32(r)) & (ph["lam"] == lam[i]) & ((ph["nrm"] @ nrm[i]) > 0)
        out[i] = ph["power"][sel].astype(np.float64).sum() / (math.pi * r * r)
    return out


def test_gather_matches_its_definition_and_the_oracle(sdd, court_maps):
    _, gm, om = court_maps
    r = 0.1
    pts, nrm, lam = floor_and_wall_queries()
    dx = torch.from_numpy(pts.astype(np.float32)).cuda()
    dn = torch.from_numpy(nrm.astype(np.float32)).cuda()
    dl = torch.from_numpy(lam).cuda()
    ec, eg = torch.empty(len(lam), device="cuda"), torch.empty(len(lam), device="cuda")
    gm.gather(dx, dn, dl, ec, eg)
    ec, eg = ec.cpu().numpy().astype(np.float64), eg.cpu().numpy().astype(np.float64)
    assert np.all(ec[-64:] == 0) and np.all(eg[-64:] == 0)  # photons that arrived on the other side
    for m, e in ((CAUSTIC, ec), (GLOBAL, eg)):
        ref = brute_gather(gm.photons(m), pts, nrm, lam, r)
        one = np.max(gm.photons(m)["power"]) / (math.pi * r * r)  # one photon's contribution
        close = np.abs(e - ref) <= 1e-5 * np.abs(ref) + 1e-30
        assert np.mean(close) >= 0.995, (m, np.mean(close))
        assert np.all(np.abs(e - ref) <= 1.01 * one + 1e-5 * np.abs(ref)), m
        assert ref.mean() > 0, m
    oc, og = om.gather(pts, nrm, lam)
    for e, o in ((ec, oc), (eg, og)):
        assert np.abs(e - o).mean() <= 3e-3 * np.abs(o).mean(), (np.abs(e - o).mean(), np.abs(o).mean())


def test_render_with_photon_maps_matches_the_oracle(sdd, orc, court_maps):
    h, gm, om = court_maps
    sc = court()
    cam = S.CameraData(pos=(0.0, -5.0, 4.0), look_at=(0.0, 0.5, 0.0), up=(0, 0, 1), vfov_deg=60.0, width=24,
                       height=16)
    spec = S.RenderSpec(lambda_nm=LAMS, spp=8, seed=5, max_depth=8, mode=S.RENDER_MC, rr_start_depth=3)
    gpu, _, gp, gh = render_gpu(sdd, h, cam, spec, paths=True, photon_maps=gm)
    ref, rp, rh = orc.OracleScene(sc).render(cam, spec, want_paths=True, photons=om)
    flips = float(np.mean(gh != rh))
    assert flips <= 1e-3, flips
    assert mean_rel_image_error(gpu, ref) <= 2e-3, mean_rel_image_error(gpu, ref)
    plain, _ = render_gpu(sdd, h, cam, spec)
    assert np.abs(plain - gpu).sum() > 1e-3 * np.abs(gpu).sum()  # the maps do change the image


def test_render_with_photon_maps_in_bundles_and_the_graph_form(sdd, orc, court_maps):
    """Spectral bundles (the three wavelengths share one ray while their decisions agree, the
    oracle tracing each as its own chain on the bundle's draws): host-driven against the
    oracle path by path, and the graph form equal to the host-driven form bit for bit."""
    h, gm, om = court_maps
    sc = court()
    cam = S.CameraData(pos=(0.0, -5.0, 4.0), look_at=(0.0, 0.5, 0.0), up=(0, 0, 1), vfov_deg=60.0, width=24,
                       height=16)
    spec = S.RenderSpec(lambda_nm=LAMS, spp=8, seed=5, max_depth=8, mode=S.RENDER_MC, rr_start_depth=3, bundle=3)
    gpu, gx, gp, gh = render_gpu(sdd, h, cam, spec, paths=True, photon_maps=gm, batched=0)
    ref, rp, rh = orc.OracleScene(sc).render(cam, spec, want_paths=True, photons=om)
    assert float(np.mean(gh != rh)) <= 1e-3, float(np.mean(gh != rh))
    assert mean_rel_image_error(gpu, ref) <= 2e-3, mean_rel_image_error(gpu, ref)
    g2, gx2, gp2, gh2 = render_gpu(sdd, h, cam, spec, paths=True, photon_maps=gm, batched=2)
    assert np.array_equal(g2, gpu) and np.array_equal(gx2, gx) and np.array_equal(gp2, gp) and np.array_equal(gh2, gh)
    one = S.RenderSpec(**{**spec.__dict__, "bundle": 1})
    u0, _ = render_gpu(sdd, h, cam, one, photon_maps=gm, batched=0)
    u2, _ = render_gpu(sdd, h, cam, one, photon_maps=gm, batched=2)
    assert np.array_equal(u0, u2)


def test_photon_buffers_grow_when_photons_are_stored_many_times(sdd, orc):
    """A closed white room (albedo 0.7) with the emitter disc inside it: a photon is stored
    about 2.3 times, past the first buffer size (one entry per photon), so the build traces
    again with larger buffers.  The sun is tilted so that no face of the glass block is met
    at grazing incidence (where FP32 refraction amplifies rounding beyond the position bar)."""
    tris = box_tris((-2, -2, 0), (2, 2, 3), 0)
    tris += box_tris((-0.6, -0.6, 0.4), (0.6, 0.6, 0.5), 1)
    ones = np.ones(LAMS.size)
    s = np.array([0.3, 0.2, 0.93])
    sc = scene_from(tris, [S.MAT_DIFFUSE, S.MAT_SOLID], [ones, S.cauchy_n(LAMS, 1.5, 0.004)], [0 * ones, 1e-7 * ones],
                    [0, 0], [0.7 * ones, 0 * ones], s / np.linalg.norm(s), n_sub=3)
    n = 30000
    h, gm, om = both_maps(sdd, orc, sc, LAMS[:1], n, 3, (0.0, 0.0, 2.3), 1.5, 0.0, 0.1, max_depth=32)
    assert gm.count(GLOBAL) > 2 * n
    check_sets(gm, om, min_counts=(1000, 2 * n))


@pytest.fixture(scope="module")
def nave_maps(sdd, orc, nave):
    sc, _, _ = nave
    lams = sc.table_nm[::10].astype(np.float32)
    return lams, both_maps(sdd, orc, sc, lams, 40000, 9, (30.0, 0.0, 7.0), 31.0, 60.0, 0.25)


def test_photon_maps_in_the_nave(nave_maps):
    """The nave (184,864 triangles, 8 subdomains): sunlight through the thin-slab windows of
    the sunward wall; 9 of the 81 wavelengths."""
    _, (h, gm, om) = nave_maps
    check_sets(gm, om, min_counts=(1, 1000), pos_tol=1e-3)  # coordinates up to ~100 m


def test_render_with_photon_maps_in_the_nave(sdd, orc, nave, nave_maps):
    """300 seeded pixels of the 1024 x 768 nave frame at 4 spp with its photon maps (9
    wavelengths): the graph form with bundles of 9 and the host-driven form with one wavelength
    per path, each against the oracle's render with its own maps, path by path."""
    sc, cam, spec = nave
    lams, (h, gm, om) = nave_maps
    pixels = np.sort(np.random.default_rng(23).choice(cam.width * cam.height, 300, replace=False)).astype(np.int32)
    for bundle, batched in ((9, 2), (1, 0)):
        sp = S.RenderSpec(**{**spec.__dict__, "lambda_nm": lams, "spp": 4, "bundle": bundle})
        gpu, _, gp, gh = render_gpu(sdd, h, cam, sp, pixels=pixels, paths=True, photon_maps=gm, batched=batched)
        ref, rp, rh = orc.OracleScene(sc).render(cam, sp, pixels=pixels, want_paths=True, photons=om)
        flips = float(np.mean(gh != rh))
        assert flips <= 1e-3, (bundle, flips)
        assert mean_rel_image_error(gpu, ref) <= 2e-3, (bundle, mean_rel_image_error(gpu, ref))


def test_photon_maps_through_heterogeneous_tiles(sdd, orc):
    """Sunlight through the brute-force-traced window of heterogeneous tiles (height-field back
    faces, air bubbles) of the tiled room: each photon meeting a tile takes one ray through it
    on the photon tile stream.  Tile rays flip at FP32 rounding for ~0.2% of rays (the tile
    parity tests), so up to 0.5% of the photons may end elsewhere, and a ray's dozens of
    refractions and bubble scatterings in a tile carry FP32 rounding into its exit direction:
    positions to 1 mm after the metres to the floor."""
    sc, _, _ = S.tile_room_scene()
    lams = sc.table_nm[::10].astype(np.float32)
    h, gm, om = both_maps(sdd, orc, sc, lams, 20000, 13, (3.0, 0.0, 2.0), 0.8, 5.0, 0.1)
    check_sets(gm, om, min_counts=(20000, 20000), pos_tol=1e-3, moved_max=5e-3)


def test_photon_maps_with_out_of_core_subdomains(sdd, court_maps):
    """With at most one of the court's four subdomain BVHs in device memory the photons are
    the all-resident ones bit for bit (in another order: their slots follow the appends)."""
    h, gm, _ = court_maps
    sdd.sdd_set_tuning(h.h, {**sdd.sdd_get_tuning(h.h), "resident_subdomains": 1})
    try:
        loads = sdd.sdd_get_stats(h.h)["subdomain_loads"]
        gs = sdd.PhotonMaps(h.h, LAMS, 200000, 17, (0.0, 0.0, 0.5), 5.0, 20.0, 0.1)
        assert sdd.sdd_get_stats(h.h)["subdomain_loads"] > loads  # the subdomains were streamed in
    finally:
        sdd.sdd_set_tuning(h.h, {**sdd.sdd_get_tuning(h.h), "resident_subdomains": 0})
    for m in (CAUSTIC, GLOBAL):
        a, b = gm.photons(m), gs.photons(m)
        ka = np.lexsort((a["seq"], a["id"], a["lam"]))
        kb = np.lexsort((b["seq"], b["id"], b["lam"]))
        for k in ("pos", "nrm", "power", "lam", "id", "seq"):
            assert np.array_equal(a[k][ka], b[k][kb]), (m, k)


def test_invalid_photon_map_use_is_rejected(sdd, court_maps):
    h, gm, _ = court_maps
    cam = S.CameraData(pos=(0.0, -5.0, 4.0), look_at=(0.0, 0.5, 0.0), up=(0, 0, 1), vfov_deg=60.0, width=4, height=4)
    spec = S.RenderSpec(lambda_nm=LAMS, spp=1, seed=5, max_depth=8, mode=S.RENDER_MC, rr_start_depth=3)
    with pytest.raises(sdd.SddError, match="batched = 0 or 2"):
        render_gpu(sdd, h, cam, spec, photon_maps=gm, batched=1)
    other = S.RenderSpec(**{**spec.__dict__, "lambda_nm": LAMS + 1.0})
    with pytest.raises(sdd.SddError, match="wavelength"):
        render_gpu(sdd, h, cam, other, photon_maps=gm)
    dark = court()
    dark.sun = None
    hd = sdd.SceneHandle(dark)
    with pytest.raises(sdd.SddError, match="sun"):
        sdd.PhotonMaps(hd.h, LAMS, 10, 1, (0, 0, 0), 1.0, 1.0, 0.1)
    with pytest.raises(sdd.SddError, match="gather_radius"):
        sdd.PhotonMaps(h.h, LAMS, 10, 1, (0, 0, 0), 1.0, 1.0, 0.0)
