"""Pins of the oracle's Monte Carlo integrator inside scenes (no GPU): Russian roulette,
heterogeneous tiles placed in a scene, and the sphere optics of air bubbles.

Russian roulette (Sec. 3.2 Monte Carlo with random rays; survival q = min(0.95, throughput),
throughput / q) is checked against two references that do not use it: the deterministic split
tree of two glass plates (Sec. 3.1), and the closed-form radiosity of a Lambertian floor under
an infinite horizontal glass slab lit by sky and sun (Eq. 3 with the slab series of Sec. 2).
A tile placed in a scene (`tile_frame`, the tile branches of `trace_mc` and `shadow_rec`, the
1-degree ballistic shadow rule) is checked against the thin-slab material, which closed forms
pin elsewhere: a flat, bubble-free tile is the thin slab.  The bubble optics
(`bubble_scatter`, Sec. 1 air micro-bubbles) are checked against textbook sphere-scattering
deviations and an independent 2-D model written with polar angles.
"""
import math

import numpy as np
import pytest

from paper_1912_05494_gb300 import scenes as S
from test_oracle_pins import box_tris, custom_scene, fresnel_real_form, quad, slab_by_bounce_sum

F32 = lambda x: float(np.float32(x))  # noqa: E731  (scene tables are float32)


def _slab_RT(theta, n, k, d, lam):
    """Thin-slab R and T from the real-arithmetic Fresnel form and an explicit bounce sum."""
    R, _, _ = fresnel_real_form(theta, n, k)
    cos_t = math.sqrt(1.0 - (math.sin(theta) / n) ** 2)
    tau = math.exp(-4.0 * math.pi * k * d / cos_t / (lam * 1e-9))
    return slab_by_bounce_sum(R, tau)


def _hemispherical(f, m=4000):
    """2 * integral_0^{pi/2} f(theta) cos(theta) sin(theta) d theta (midpoint rule)."""
    th = (np.arange(m) + 0.5) * (0.5 * math.pi / m)
    return float(sum(f(t) * math.cos(t) * math.sin(t) for t in th) * 2.0 * (0.5 * math.pi / m))


def _rr_kill_fraction(h_rr, h_off):
    """Paths whose event hash differs from the same draws without roulette: roulette draws use a
    word nothing else reads, so a path changes its events only where roulette killed it."""
    return float(np.mean(h_rr != h_off))


# ----------------------------------------------------------------------------- Russian roulette
def test_russian_roulette_unbiased_against_split_tree():
    """Two absorbing glass plates one behind the other, seen obliquely: Monte Carlo with roulette
    from interaction 1, 2 or 3 averages to the deterministic split tree of the same depth, and
    roulette kills more than 20% of the paths (throughput ~0.5 behind each plate)."""
    from oracle import oracle as orc
    n, k, d = 1.55, 1e-5, 3e-3
    tris = box_tris((-0.5, 0.0, -0.5), (0.5, d, 0.5), 0) + box_tris((-0.5, 0.02, -0.5), (0.5, 0.02 + d, 0.5), 0)
    osc = orc.OracleScene(custom_scene(tris, [{"kind": S.MAT_SOLID, "n": n, "k": k}]))
    th = math.radians(40.0)
    cam = S.CameraData(pos=(0.0, -math.cos(th), math.sin(th)), look_at=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0),
                       vfov_deg=1.0, width=2, height=2, ortho=1, ortho_height=0.02)
    lam = np.array([550.0], np.float32)
    depth = 10
    det, _, _ = osc.render(cam, S.RenderSpec(lambda_nm=lam, spp=1, seed=0, max_depth=depth, mode=0))
    _, _, h_off = osc.render(cam, S.RenderSpec(lambda_nm=lam, spp=20000, seed=21, max_depth=depth, mode=1),
                             want_paths=True)
    for start in (1, 2, 3):
        mc, paths, h = osc.render(cam, S.RenderSpec(lambda_nm=lam, spp=20000, seed=21, max_depth=depth, mode=1,
                                                    rr_start_depth=start), want_paths=True)
        kill = _rr_kill_fraction(h, h_off)
        assert kill > 0.2, (start, kill)
        se = paths.std() / math.sqrt(paths.size)
        assert abs(mc.mean() - det.mean()) < 4 * se + 1e-9, (start, mc.mean(), det.mean(), se)


def test_russian_roulette_unbiased_on_floor_under_glass():
    """An infinite Lambertian floor (albedo rho) under an infinite horizontal thin slab, sky
    L_sky above and a sun disc at elevation e; an orthographic camera looks straight down
    through the slab.  Floor radiance solves
        L_f = [rho/pi E_d + rho L_sky T_h] / (1 - rho R_h),
        E_d = L_sun pi sin^2(a) sin(e) T(90 deg - e),
    with T_h, R_h the slab's cosine-weighted hemispherical transmittance and reflectance; the
    pixel is R(0) L_sky + T(0) L_f.  Monte Carlo with and without roulette matches it; with
    roulette from interaction 1, 2 or 3 more than 20% of paths are killed."""
    from oracle import oracle as orc
    rho, L_sky, L_sun = 0.5, 1.0, 2.0e4
    n, k, d, lam = 1.52, 4e-6, 4e-3, 550.0
    elev, a = math.radians(35.0), math.radians(0.2665)
    sdir = (0.0, -math.cos(elev), math.sin(elev))
    big = 100.0
    tris = (quad((-big, -big, 0), (big, -big, 0), (big, big, 0), (-big, big, 0), 0)
            + quad((-big, -big, 0.5), (big, -big, 0.5), (big, big, 0.5), (-big, big, 0.5), 1))
    mats = [{"kind": S.MAT_DIFFUSE, "albedo": rho}, {"kind": S.MAT_SLAB, "n": n, "k": k, "d": d}]
    osc = orc.OracleScene(custom_scene(tris, mats, sky=L_sky, sky_mode=1, sun=L_sun, sun_dir=sdir, half=a))
    cam = S.CameraData(pos=(0, 0, 1.0), look_at=(0, 0, 0), up=(0, 1, 0), vfov_deg=1.0, width=8, height=8,
                       ortho=1, ortho_height=0.5)
    n32, k32, d32 = F32(n), F32(k), F32(d)
    T = lambda th: _slab_RT(th, n32, k32, d32, lam)[1]  # noqa: E731
    R = lambda th: _slab_RT(th, n32, k32, d32, lam)[0]  # noqa: E731
    T_h, R_h = _hemispherical(T), _hemispherical(R)
    E_d = F32(L_sun) * math.pi * math.sin(F32(a)) ** 2 * math.sin(elev) * T(0.5 * math.pi - elev)
    L_f = (rho / math.pi * E_d + rho * L_sky * T_h) / (1.0 - rho * R_h)
    want = R(0.0) * L_sky + T(0.0) * L_f
    spec = dict(lambda_nm=np.array([lam], np.float32), spp=1500, seed=5, max_depth=40, mode=1)
    _, _, h_off = osc.render(cam, S.RenderSpec(**spec), want_paths=True)
    for start in (1 << 30, 1, 2, 3):
        film, paths, h = osc.render(cam, S.RenderSpec(**spec, rr_start_depth=start), want_paths=True)
        se = paths.std() / math.sqrt(paths.size)
        assert abs(film.mean() - want) < 4 * se, (start, film.mean(), want, se)
        if start < 1 << 30:
            assert _rr_kill_fraction(h, h_off) > 0.2, start
    assert abs(film.mean() - (R(0.0) + T(0.0) * rho * L_sky)) > 10 * se  # sun and inter-reflection matter


# ----------------------------------------------------------------------------- tiles in a scene
def _window_scene(kind, n, k, d, lam, sun, sdir, half):
    """Floor + one obliquely placed 3x3 m window (30 tile periods across) between the floor
    and the sun; the window is a thin slab or a flat, bubble-free heterogeneous tile."""
    nw = np.array([0.35, -1.0, 0.45])
    nw /= np.linalg.norm(nw)
    e1 = np.cross(nw, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nw, e1)
    c = np.array([0.3, -2.0, 1.6])
    corners = [tuple(c + 1.5 * (sx * e1 + sy * e2)) for sx, sy in ((-1, -1), (1, -1), (1, 1), (-1, 1))]
    big = 100.0
    tris = quad((-big, -big, 0), (big, -big, 0), (big, big, 0), (-big, big, 0), 0) + quad(*corners, 1)
    mats = [{"kind": S.MAT_DIFFUSE, "albedo": 0.5}, {"kind": kind, "n": n, "k": k, "d": d}]
    sc = custom_scene(tris, mats, sky=1.0, sky_mode=1, sun=sun, sun_dir=sdir, half=half, lam=lam)
    if kind == S.MAT_TILE:
        sc.tiles = [{"d_mean": float(np.float32(d)), "amp": 0.0, "rho": 0.0, "seed": 3}]
        sc.mat_tile = np.array([-1, 0], np.int32)
    return sc, nw, c, e1, e2


def _ortho(pos, look, up, w=12, h=12, size=0.3):
    return S.CameraData(pos=tuple(pos), look_at=tuple(look), up=tuple(up), vfov_deg=1.0, width=w, height=h,
                        ortho=1, ortho_height=size)


def test_flat_tile_in_scene_equals_thin_slab():
    """A flat, bubble-free tile window placed obliquely renders, in expectation, what the thin-
    slab window renders: the floor lit by the sun through it (the NEE ballistic rule), a
    camera looking through it at the sun (entering through the back face: the exit direction
    must map back exactly onto the sun's disc) and one looking through it from the sun's side
    onto the floor (entering through the front face).  The window spans 30 tile periods, so
    hit positions wrap many times; the tracer's cell lookup is itself periodic, the wrap in
    `tile_frame` only keeps tile coordinates small."""
    from oracle import oracle as orc
    n, k, d, lam = 1.53, 3e-6, 3.5e-3, 550.0
    elev, half, sun = math.radians(35.0), math.radians(0.2665), 2.0e4
    sdir = np.array([0.0, -math.cos(elev), math.sin(elev)])
    scenes = {kind: _window_scene(kind, n, k, d, lam, sun, sdir, half) for kind in (S.MAT_SLAB, S.MAT_TILE)}
    _, nw, c, e1, e2 = scenes[S.MAT_SLAB]
    # every shadow ray of the floor patch and every camera ray below crosses the window
    for p in ([-0.2, -0.2, 0.0], [0.2, 0.2, 0.0], [0.0, -0.15, 0.2], [0.0, 0.15, 0.4]):
        t = np.dot(nw, c - p) / np.dot(nw, sdir)
        q = np.asarray(p) + t * sdir - c
        assert t > 0 and abs(np.dot(q, e1)) < 1.3 and abs(np.dot(q, e2)) < 1.3
    assert abs(np.dot(nw, sdir)) < 0.95  # oblique: 18+ degrees off the window normal
    cams = {
        "floor": _ortho([0, 0, 1.0], [0, 0, 0], [0, 1, 0]),
        # origins at z = 0.3 +- 0.1: clear of the floor
        "to_sun": _ortho([0, 0, 0.3], list(np.array([0, 0, 0.3]) + sdir), [1, 0, 0], size=0.2),
        "from_sun": _ortho(list(np.array([0, 0, 0.3]) + 4.0 * sdir), [0, 0, 0.3], [1, 0, 0], size=0.2),
    }
    spec = S.RenderSpec(lambda_nm=np.array([lam], np.float32), spp=300, seed=13, max_depth=12, mode=1,
                        rr_start_depth=3)
    for name, cam in cams.items():
        res = {}
        for kind, (sc, *_) in scenes.items():
            film, paths, _ = orc.OracleScene(sc).render(cam, spec, want_paths=True)
            res[kind] = (film.mean(), paths.std() / math.sqrt(paths.size))
        (ms, ss), (mt, st) = res[S.MAT_SLAB], res[S.MAT_TILE]
        assert abs(ms - mt) < 4 * math.hypot(ss, st) and ss < 0.01 * ms, (name, ms, mt, ss, st)
        if name == "to_sun":  # the sun seen through the window
            theta = math.acos(abs(float(np.dot(nw, sdir))))
            T = _slab_RT(theta, F32(n), F32(k), F32(d), lam)[1]
            assert abs(mt / (T * (F32(sun) + 1.0)) - 1.0) < 0.03, (mt, T)


# ----------------------------------------------------------------------------- bubble optics
def _bubble_angle_model(sin_i, n, chain):
    """Independent 2-D model of a ray meeting a unit circle of air in glass of index n: the ray
    travels in direction angle 0 and meets the circle at polar angle pi - theta_i; each surface
    takes 'R' (reflect) or 'T' (refract; reflect when Snell has no solution).  Returns the exit
    direction angle and the number of surfaces met."""
    th_i = math.asin(sin_i)
    alpha, phi, inside, met = math.pi - th_i, 0.0, False, 0
    wrap = lambda x: (x + math.pi) % (2.0 * math.pi) - math.pi  # noqa: E731
    for c in chain:
        met += 1
        normal = alpha + math.pi if not inside else alpha  # normal pointing along the travel
        inc = wrap(phi - normal)
        s_t = (n if not inside else 1.0 / n) * math.sin(inc)
        if c == "T" and abs(s_t) < 1.0:
            phi = normal + math.asin(s_t)
            inside = not inside
        else:
            phi = 2.0 * alpha + math.pi - phi
        if not inside:
            return phi, met
        alpha = 2.0 * phi + math.pi - alpha  # across the chord
    raise AssertionError("chain ended inside the bubble")


@pytest.mark.parametrize("n", [1.5, 1.33])
def test_bubble_sphere_optics(n):
    """Exit directions of a bubble met at impact parameter b/r = sin(theta_i), with the surface
    choices forced: external reflection leaves at pi - 2 theta_i from the incident direction;
    straight refraction (in, out) at 2 (theta_r - theta_i), sin theta_r = n sin theta_i, bent
    away from the centre; chains with internal reflections against the 2-D angle model; in
    random 3-D orientations, in the plane of d and the impact direction."""
    from oracle import oracle as orc
    rng = np.random.default_rng(17)
    N = 300
    d = rng.normal(size=(N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = rng.normal(size=(N, 3))
    rad -= np.sum(rad * d, axis=1, keepdims=True) * d
    rad /= np.linalg.norm(rad, axis=1, keepdims=True)
    sin_i = rng.uniform(0.02, 0.98, N)
    force = {"R": 0.0, "T": 1.0 - 1e-15}
    for chain in ("R", "TT", "TRT", "TRRT", "TRRRT"):
        u = np.tile([force[ch] for ch in chain], (N, 1))
        out, met = orc.bubble_scatter(d, rad, sin_i, u, n)
        for i in range(N):
            phi, m = _bubble_angle_model(sin_i[i], n, chain)
            want = math.cos(phi) * d[i] + math.sin(phi) * rad[i]
            assert met[i] == m, (chain, i, met[i], m)
            assert np.allclose(out[i], want, atol=1e-12), (chain, sin_i[i], out[i], want)
    th_i = np.arcsin(sin_i)
    out, met = orc.bubble_scatter(d, rad, sin_i, np.zeros((N, 1)), n)
    assert np.all(met == 1)
    assert np.allclose(np.sum(out * d, axis=1), np.cos(np.pi - 2 * th_i), atol=1e-12)
    ok = n * sin_i < 0.95  # below the critical angle of glass -> air
    out, met = orc.bubble_scatter(d[ok], rad[ok], sin_i[ok], np.full((ok.sum(), 2), 1 - 1e-15), n)
    th_r = np.arcsin(n * sin_i[ok])
    assert np.all(met == 2)
    assert np.allclose(np.sum(out * d[ok], axis=1), np.cos(2 * (th_r - th_i[ok])), atol=1e-12)
    assert np.all(np.sum(out * rad[ok], axis=1) > 0)  # diverging: away from the centre
    tir = n * sin_i > 1.0  # total internal reflection at the first surface whatever the draw
    out, met = orc.bubble_scatter(d[tir], rad[tir], sin_i[tir], np.full((tir.sum(), 2), 1 - 1e-15), n)
    assert tir.sum() > 10 and np.all(met == 1)
    assert np.allclose(np.sum(out * d[tir], axis=1), np.cos(np.pi - 2 * th_i[tir]), atol=1e-12)
