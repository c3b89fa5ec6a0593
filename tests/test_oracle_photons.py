"""Pins of the oracle's photon maps (Sec. 3.2, Jensen's photon mapping; no GPU).

A floor (Lambertian, albedo rho) lies under a glass plate of infinite extent, lit by the sun at
elevation e.  Closed forms, with the plate's transmittance T(theta) and its cosine-weighted
hemispherical reflectance R_h from the tests' own real-arithmetic Fresnel form and explicit
bounce sums (not the oracle's functions):
  * sun irradiance on the floor through the plate      E_d = L_sun pi sin^2(a) sin(e) T(90 - e)
  * light the floor sends up and the plate sends back  E_ind = E_d rho R_h / (1 - rho R_h)
A solid plate refracts the sunlight (specular events that change direction), so the floor's
first-hit photons are caustic photons: the caustic map must estimate E_d.  A thin slab passes
it straight through: that light is direct (the renderer's sun NEE counts it) and must not be
stored.  Photons after a diffuse bounce are global photons: the global map must estimate
E_ind under either plate.  Estimates are averaged over query points 2 r apart (disjoint photon
discs), against 4 standard errors of that mean.
"""
import math

import numpy as np
import pytest

from paper_1912_05494_gb300 import scenes as S
from test_oracle_pins import box_tris, custom_scene, fresnel_real_form, quad, slab_by_bounce_sum

F32 = lambda x: float(np.float32(x))  # noqa: E731


def plate_RT(theta, n, k, d, lam):
    R, _, _ = fresnel_real_form(theta, n, k)
    cos_t = math.sqrt(1.0 - (math.sin(theta) / n) ** 2)
    return slab_by_bounce_sum(R, math.exp(-4.0 * math.pi * k * d / cos_t / (lam * 1e-9)))


def hemispherical(f, m=3000):
    """2 * integral_0^{pi/2} f(theta) cos(theta) sin(theta) d theta (midpoint rule)."""
    th = (np.arange(m) + 0.5) * (0.5 * math.pi / m)
    return float(sum(f(t) * math.cos(t) * math.sin(t) for t in th) * 2.0 * (0.5 * math.pi / m))


N_, K_, D_, LAM = 1.5, 2e-5, 5e-3, 550.0
RHO, L_SUN, ELEV, HALF = 0.7, 1.0e4, math.radians(55.0), math.radians(0.2665)
GAP = 0.05  # plate bottom above the floor (m): bounced light returns within a few tens of cm


def scene(kind):
    big = 100.0
    tris = quad((-big, -big, 0), (big, -big, 0), (big, big, 0), (-big, big, 0), 0)
    if kind == S.MAT_SOLID:
        tris += box_tris((-big, -big, GAP), (big, big, GAP + D_), 1)
    else:
        tris += quad((-big, -big, GAP), (big, -big, GAP), (big, big, GAP), (-big, big, GAP), 1)
    sdir = (0.0, -math.cos(ELEV), math.sin(ELEV))
    mats = [{"kind": S.MAT_DIFFUSE, "albedo": RHO}, {"kind": kind, "n": N_, "k": K_, "d": D_}]
    return custom_scene(tris, mats, sky=0.0, sky_mode=1, sun=L_SUN, sun_dir=sdir, half=HALF, lam=LAM)


def closed_forms():
    n, k, d = F32(N_), F32(K_), F32(D_)
    T = lambda th: plate_RT(th, n, k, d, LAM)[1]  # noqa: E731
    R = lambda th: plate_RT(th, n, k, d, LAM)[0]  # noqa: E731
    R_h = hemispherical(R)
    E_d = F32(L_SUN) * math.pi * math.sin(F32(HALF)) ** 2 * math.sin(ELEV) * T(0.5 * math.pi - ELEV)
    return E_d, E_d * RHO * R_h / (1.0 - RHO * R_h), T, R


def queries(r):
    g = np.arange(-3, 4) * 2.2 * r
    x, y = np.meshgrid(g, g)
    return np.column_stack([x.ravel(), y.ravel(), np.zeros(x.size)])


def maps(orc, kind, n=300000, r=0.15):
    osc = orc.OracleScene(scene(kind))
    pm = osc.photon_maps(np.array([LAM], np.float32), n, seed=31, center=(0.0, 0.0, 0.0), radius=4.0, distance=30.0,
                         gather_radius=r)
    return osc, pm


def mean_se(v):
    return float(v.mean()), float(v.std(ddof=1) / math.sqrt(v.size))


def test_direct_light_is_not_stored(orc):
    """Open floor under the sun: the first hit is direct light and the bounce escapes: both
    maps are empty.  Under a thin slab, straight transmission is direct light too: no caustic
    photon."""
    big = 100.0
    tris = quad((-big, -big, 0), (big, -big, 0), (big, big, 0), (-big, big, 0), 0)
    sc = custom_scene(tris, [{"kind": S.MAT_DIFFUSE, "albedo": RHO}], sky=0.0, sky_mode=1, sun=L_SUN,
                      sun_dir=(0.0, -math.cos(ELEV), math.sin(ELEV)), half=HALF, lam=LAM)
    pm = orc.OracleScene(sc).photon_maps(np.array([LAM], np.float32), 20000, seed=1, center=(0, 0, 0), radius=2.0,
                                         distance=30.0, gather_radius=0.1)
    assert pm.count(orc.MAP_CAUSTIC) == 0 and pm.count(orc.MAP_GLOBAL) == 0
    _, pm = maps(orc, S.MAT_SLAB, n=20000)
    assert pm.count(orc.MAP_CAUSTIC) == 0 and pm.count(orc.MAP_GLOBAL) > 0


def test_caustic_and_global_maps_under_a_solid_plate(orc):
    E_d, E_ind, _, _ = closed_forms()
    _, pm = maps(orc, S.MAT_SOLID)
    q = queries(0.15)
    ec, eg = pm.gather(q, (0.0, 0.0, 1.0), 0)
    m, se = mean_se(ec)
    assert abs(m - E_d) < 4 * se and se < 0.02 * E_d, (m, E_d, se)
    m, se = mean_se(eg)
    assert abs(m - E_ind) < 4 * se and se < 0.1 * E_ind, (m, E_ind, se)
    ph = pm.photons(orc.MAP_CAUSTIC)
    assert np.allclose(ph["pos"][:, 2], 0.0, atol=1e-9) and np.all(ph["nrm"][:, 2] > 0.99)  # all on the floor


def test_global_map_under_a_thin_slab(orc):
    E_d, E_ind, _, _ = closed_forms()
    _, pm = maps(orc, S.MAT_SLAB)
    ec, eg = pm.gather(queries(0.15), (0.0, 0.0, 1.0), 0)
    assert np.all(ec == 0.0)
    m, se = mean_se(eg)
    assert abs(m - E_ind) < 4 * se and se < 0.1 * E_ind, (m, E_ind, se)
    # photons arriving on the other side of a surface do not count
    ec2, eg2 = pm.gather(queries(0.15), (0.0, 0.0, -1.0), 0)
    assert np.all(eg2 == 0.0)


def test_render_with_photon_maps(orc):
    """A camera looks straight down through the solid plate at the floor (no sky): the sun
    reaches the floor only through the refracting plate, so only the maps light it.  Each
    pixel equals T(0) rho / pi (E_caustic + E_global) of the maps at its floor point; and the
    render without maps is black (the sun NEE is blocked by solid glass)."""
    osc, pm = maps(orc, S.MAT_SOLID)
    cam = S.CameraData(pos=(0, 0, 1.0), look_at=(0, 0, 0), up=(0, 1, 0), vfov_deg=1.0, width=6, height=6, ortho=1,
                       ortho_height=1.2)
    spec = S.RenderSpec(lambda_nm=np.array([LAM], np.float32), spp=1024, seed=3, max_depth=12, mode=1,
                        rr_start_depth=3)
    film, paths, _ = osc.render(cam, spec, want_paths=True, photons=pm)
    plain, _, _ = osc.render(cam, spec)
    assert np.all(plain == 0.0)
    # the floor points the pixels see (straight down, no lateral shift at normal incidence)
    h = 1.2 / 2
    c = (np.arange(6) + 0.5) / 6 * 2 - 1
    xs, ys = np.meshgrid(c * h, -c * h)
    pts = np.column_stack([xs.ravel(), ys.ravel(), np.zeros(36)])
    ec, eg = pm.gather(pts, (0.0, 0.0, 1.0), 0)
    _, _, T, _ = closed_forms()
    want = T(0.0) * RHO / math.pi * (ec + eg)
    se = paths.std(axis=1).ravel() / math.sqrt(spec.spp)
    # pixels jitter over their footprint while the gather point is the centre: compare means
    assert abs(film.mean() - want.mean()) < 4 * math.sqrt((se**2).sum()) / 36 + 0.02 * want.mean(), (
        film.mean(), want.mean())
    E_d, E_ind, _, _ = closed_forms()
    assert abs(film.mean() / (T(0.0) * RHO / math.pi * (E_d + E_ind)) - 1.0) < 0.05
