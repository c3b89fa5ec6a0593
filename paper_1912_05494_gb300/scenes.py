"""Seeded synthetic scenes: the inputs that both the CUDA renderer and the CPU oracle read.

This module only builds input arrays (triangles, per-material n(lambda)/k(lambda) tables and
thicknesses, illuminant spectra, camera, wavelength set).  It performs none of the
renderer's arithmetic and imports nothing else from this package.

The paper's own inputs -- the Royaumont abbey model and the Maubuisson / Saint-Just glass
measurements (Sec. 1, Sec. 2, Sec. 6) -- are not available, so these procedural scenes
stand in for them:

* ``slab_scene``: one 1 m x 1 m x 3 mm glass slab in front of a uniform sky of radiance 1,
  n = 1.52 + 0.0042/lambda^2 (lambda in um), k = 5e-7 (1 + 0.5 Gaussian bump), 16
  wavelengths 380-730 nm, 64x64 pinhole camera at normal incidence, deterministic
  reflect+transmit splitting to depth 6.
* ``nave_scene``: a box nave 60 x 12 x 20 m (walls to 14 m under a semicircular vault),
  24 lancet windows of 200 thin-slab glass tiles (Cauchy n, banded k, 2-5 mm) with lead
  came, 22 piers, a 6500 K sky and a sun at 35 degrees elevation, 81 wavelengths
  380-780 nm (Sec. 4's spectral grid), 1024x768, 16 spp, depth 12.
* ``tiny_scene``: a few random triangles for intersection tests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAT_SOLID, MAT_SLAB, MAT_TILE, MAT_DIFFUSE, MAT_OPAQUE = 0, 1, 2, 3, 4
RENDER_DETERMINISTIC, RENDER_MC = 0, 1

SPECTRAL_GRID_81 = np.arange(380.0, 780.0 + 1e-9, 5.0, dtype=np.float32)  # Sec. 4: 81 samples


@dataclasses.dataclass
class SceneData:
    vertices: np.ndarray          # float32 [V, 3] metres
    indices: np.ndarray           # uint32 [T, 3]
    tri_material: np.ndarray      # uint16 [T]
    mat_kind: np.ndarray          # int32 [M]
    mat_thickness: np.ndarray     # float32 [M] metres
    table_nm: np.ndarray          # float32 [Lt] wavelength grid of every table below
    mat_n: np.ndarray             # float32 [M, Lt]
    mat_k: np.ndarray             # float32 [M, Lt]
    mat_albedo: np.ndarray        # float32 [M, Lt]
    sky: np.ndarray               # float32 [Lt]
    sky_mode: int                 # 0 every direction, 1 upper hemisphere (z > 0) only
    sun_dir: np.ndarray           # float32 [3] unit, toward the sun
    sun_half_angle: float         # radians; 0 = no sun
    sun: np.ndarray | None        # float32 [Lt]
    ray_eps: float                # spawn offset along the geometric normal (m)
    n_subdomains: int = 1
    split_axis: int = 0
    info: dict = dataclasses.field(default_factory=dict)
    tiles: list | None = None      # heterogeneous tile parameters (dicts d_mean, amp, rho, seed)
    mat_tile: np.ndarray | None = None  # int32 [M] tile index of HETERO_TILE materials, -1 otherwise
    tile_grid: int = 64
    tile_size: float = 0.1
    slab_polarisation: int = 0    # thin slabs: 0 series on the unpolarised R, 1 per polarisation

    @property
    def n_triangles(self) -> int:
        return int(self.indices.shape[0])


@dataclasses.dataclass
class CameraData:
    pos: tuple
    look_at: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int
    ortho: int = 0
    ortho_height: float = 0.0


@dataclasses.dataclass
class RenderSpec:
    lambda_nm: np.ndarray         # float32 [L]
    spp: int
    seed: int
    max_depth: int
    mode: int                     # RENDER_DETERMINISTIC or RENDER_MC
    rr_start_depth: int = 1 << 30
    bundle: int = 1               # Monte Carlo: consecutive wavelengths that share their draws

    @property
    def n_lambda(self) -> int:
        return int(self.lambda_nm.shape[0])


# ----------------------------------------------------------------------------- spectra
def cauchy_n(lambda_nm, a, b_um2):
    """Cauchy dispersion n = A + B / lambda^2 with lambda in micrometres."""
    lam_um = np.asarray(lambda_nm, np.float64) * 1e-3
    return a + b_um2 / lam_um**2


def planck(lambda_nm, temp_k):
    """Planck spectral radiance B(lambda, T) in W sr^-1 m^-3 (CODATA constants)."""
    h, c, kb = 6.62607015e-34, 2.99792458e8, 1.380649e-23
    lam = np.asarray(lambda_nm, np.float64) * 1e-9
    return 2.0 * h * c**2 / lam**5 / np.expm1(h * c / (lam * kb * temp_k))


def blackbody_normalised(lambda_nm, temp_k=6500.0, at_nm=560.0):
    """Blackbody spectrum scaled to 1 at ``at_nm``."""
    return planck(lambda_nm, temp_k) / planck(np.array([at_nm]), temp_k)[0]


# ----------------------------------------------------------------------------- geometry
class _Mesh:
    def __init__(self):
        self.v: list = []
        self.t: list = []
        self.m: list = []

    def tri(self, a, b, c, mat):
        base = len(self.v)
        self.v.extend([a, b, c])
        self.t.append((base, base + 1, base + 2))
        self.m.append(mat)

    def quad(self, a, b, c, d, mat):
        """Quad a-b-c-d (counter-clockwise seen from the side its normal points to)."""
        base = len(self.v)
        self.v.extend([a, b, c, d])
        self.t.append((base, base + 1, base + 2))
        self.t.append((base, base + 2, base + 3))
        self.m.extend([mat, mat])

    def box(self, lo, hi, mat):
        """Axis-aligned box with outward-facing triangles (12 triangles)."""
        x0, y0, z0 = lo
        x1, y1, z1 = hi
        p = [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
             (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]
        for a, b, c, d in ((0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4),
                           (2, 3, 7, 6), (1, 2, 6, 5), (0, 4, 7, 3)):
            self.quad(p[a], p[b], p[c], p[d], mat)

    def arrays(self):
        v = np.asarray(self.v, np.float32).reshape(-1, 3)
        t = np.asarray(self.t, np.uint32).reshape(-1, 3)
        m = np.asarray(self.m, np.uint16)
        return v, t, m


def _grid(mesh, origin, eu, ev, nu, nv, mat, skip=None):
    """Tessellate the parallelogram origin + [0,nu]*eu + [0,nv]*ev into nu*nv quads."""
    o = np.asarray(origin, np.float64)
    eu = np.asarray(eu, np.float64)
    ev = np.asarray(ev, np.float64)
    for i in range(nu):
        for j in range(nv):
            if skip is not None and skip(i, j):
                continue
            a = o + i * eu + j * ev
            mesh.quad(tuple(a), tuple(a + eu), tuple(a + eu + ev), tuple(a + ev), mat)


# ----------------------------------------------------------------------------- scenes
def slab_scene(seed: int = 0):
    """One glass slab (12 triangles) in front of a uniform sky of radiance 1."""
    rng = np.random.default_rng(seed)
    lam = (380.0 + np.arange(16) * (350.0 / 15.0)).astype(np.float32)
    mu = 550.0 + rng.uniform(-50.0, 50.0)
    n = cauchy_n(lam, 1.52, 0.0042)
    k = 5e-7 * (1.0 + 0.5 * np.exp(-((lam - mu) ** 2) / (2.0 * 50.0**2)))
    mesh = _Mesh()
    mesh.box((-0.5, 0.0, -0.5), (0.5, 0.003, 0.5), 0)
    v, t, m = mesh.arrays()
    scene = SceneData(
        vertices=v, indices=t, tri_material=m,
        mat_kind=np.array([MAT_SOLID], np.int32),
        mat_thickness=np.array([0.003], np.float32),
        table_nm=lam,
        mat_n=n[None, :].astype(np.float32), mat_k=k[None, :].astype(np.float32),
        mat_albedo=np.zeros((1, lam.size), np.float32),
        sky=np.ones(lam.size, np.float32), sky_mode=0,
        sun_dir=np.array([0, 0, 1], np.float32), sun_half_angle=0.0, sun=None,
        ray_eps=1e-5, n_subdomains=1, split_axis=1,
        info={"k_bump_center_nm": float(mu), "triangles": int(t.shape[0])},
    )
    cam = CameraData(pos=(0.0, -1.0, 0.0), look_at=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0),
                     vfov_deg=60.0, width=64, height=64)
    spec = RenderSpec(lambda_nm=lam, spp=1, seed=seed, max_depth=6, mode=RENDER_DETERMINISTIC)
    return scene, cam, spec


def nave_scene(seed: int = 1, cell: float = 0.25, windows_per_wall: int = 12,
               tiles_x: int = 10, tiles_z: int = 20, length: float = 60.0,
               n_subdomains: int = 8, width: int = 1024, height: int = 768, spp: int = 16,
               max_depth: int = 12, rr_start_depth: int = 3, pier_sides: int = 16,
               sills=(6.0,), hetero_tiles: int = 0, tile_seed: int = 3):
    """Procedural nave with stained-glass windows of thin-slab tiles.

    Nave 60 m (x) x 12 m (y); walls up to z = 14 m under a semicircular barrel vault
    (apex 20 m).  Windows: 1 m x 2 m lancets (tiles_x x tiles_z tiles of 10 cm) with their
    sill at 6 m, centred every 5 m along both long walls; lead came is 6 mm x 10 mm boxes on
    the tile grid.  22 octagonal-ish piers (``pier_sides``-gons of radius 0.4 m).
    """
    rng = np.random.default_rng(seed)
    lam = SPECTRAL_GRID_81.copy()
    mesh = _Mesh()
    STONE, CAME = 0, 1
    wall_h, width_y = 14.0, 12.0
    nx = int(round(length / cell))
    tile = 0.1
    win_w, win_h = tiles_x * tile, tiles_z * tile
    spacing = length / windows_per_wall
    win_x0 = [spacing * (i + 0.5) - 0.5 * win_w for i in range(windows_per_wall)]

    def in_window(x_lo, z_lo):
        if not any(sl - 1e-6 <= z_lo < sl + win_h - 1e-6 for sl in sills):
            return False
        return any(x0 - 1e-6 <= x_lo < x0 + win_w - 1e-6 for x0 in win_x0)

    # floor (normal +z) and long walls (normals toward the interior)
    _grid(mesh, (0, 0, 0), (cell, 0, 0), (0, cell, 0), nx, int(round(width_y / cell)), STONE)
    nz = int(round(wall_h / cell))
    _grid(mesh, (0, 0, 0), (0, 0, cell), (cell, 0, 0), nz, nx, STONE,
          skip=lambda i, j: in_window(j * cell, i * cell))
    _grid(mesh, (0, width_y, 0), (cell, 0, 0), (0, 0, cell), nx, nz, STONE,
          skip=lambda i, j: in_window(i * cell, j * cell))
    # end walls up to the vault apex
    ny = int(round(width_y / cell))
    nze = int(round(20.0 / cell))
    _grid(mesh, (0, 0, 0), (0, cell, 0), (0, 0, cell), ny, nze, STONE)
    _grid(mesh, (length, 0, 0), (0, 0, cell), (0, cell, 0), nze, ny, STONE)
    # semicircular vault over y in [0, 12], centred at (y=6, z=14)
    n_arc = int(round(math.pi * 6.0 / cell))
    for a in range(n_arc):
        t0, t1 = math.pi * a / n_arc, math.pi * (a + 1) / n_arc
        y0, z0 = 6.0 - 6.0 * math.cos(t0), wall_h + 6.0 * math.sin(t0)
        y1, z1 = 6.0 - 6.0 * math.cos(t1), wall_h + 6.0 * math.sin(t1)
        for i in range(nx):
            xa, xb = i * cell, (i + 1) * cell
            mesh.quad((xa, y0, z0), (xa, y1, z1), (xb, y1, z1), (xb, y0, z0), STONE)
    # piers
    n_rings = int(round(wall_h / cell))
    for side_y in (1.0, width_y - 1.0):
        for i in range(1, windows_per_wall):
            cx = spacing * i
            for r in range(n_rings):
                za, zb = r * cell, (r + 1) * cell
                for s in range(pier_sides):
                    a0 = 2 * math.pi * s / pier_sides
                    a1 = 2 * math.pi * (s + 1) / pier_sides
                    p0 = (cx + 0.4 * math.cos(a0), side_y + 0.4 * math.sin(a0))
                    p1 = (cx + 0.4 * math.cos(a1), side_y + 0.4 * math.sin(a1))
                    mesh.quad((p0[0], p0[1], za), (p1[0], p1[1], za), (p1[0], p1[1], zb),
                              (p0[0], p0[1], zb), STONE)
    # windows: thin-slab tiles (one material each) and lead came
    n_tiles = 2 * len(sills) * windows_per_wall * tiles_x * tiles_z
    tile_mat0 = 2
    tm = tile_mat0
    half_w, half_d = 0.003, 0.005
    for wall_y, sill, x0 in [(wy, sl, x) for wy in (0.0, width_y) for sl in sills for x in win_x0]:
        if True:
            for i in range(tiles_x):
                for j in range(tiles_z):
                    xa, za = x0 + i * tile, sill + j * tile
                    mesh.quad((xa, wall_y, za), (xa + tile, wall_y, za),
                              (xa + tile, wall_y, za + tile), (xa, wall_y, za + tile), tm)
                    tm += 1
            for i in range(tiles_x + 1):
                xc = x0 + i * tile
                mesh.box((xc - half_w, wall_y - half_d, sill), (xc + half_w, wall_y + half_d, sill + win_h), CAME)
            for j in range(tiles_z + 1):
                zc = sill + j * tile
                mesh.box((x0, wall_y - half_d, zc - half_w), (x0 + win_w, wall_y + half_d, zc + half_w), CAME)
    v, t, m = mesh.arrays()

    # materials: stone, came, then one thin slab per tile (distribution map of n, k, d)
    n_mat = tile_mat0 + n_tiles
    kind = np.full(n_mat, MAT_SLAB, np.int32)
    kind[STONE] = MAT_DIFFUSE
    kind[CAME] = MAT_DIFFUSE
    thick = np.zeros(n_mat, np.float32)
    mat_n = np.ones((n_mat, lam.size), np.float32)
    mat_k = np.zeros((n_mat, lam.size), np.float32)
    albedo = np.zeros((n_mat, lam.size), np.float32)
    albedo[STONE] = 0.5
    albedo[CAME] = 0.05
    thick[tile_mat0:] = rng.uniform(2e-3, 5e-3, n_tiles)
    a = rng.uniform(1.50, 1.58, n_tiles)
    b = rng.uniform(0.003, 0.006, n_tiles)
    mat_n[tile_mat0:] = cauchy_n(lam[None, :], a[:, None], b[:, None])
    base = np.exp(rng.uniform(np.log(1e-7), np.log(1e-5), n_tiles))
    centre = rng.uniform(400.0, 700.0, (n_tiles, 3))
    sigma = rng.uniform(15.0, 60.0, (n_tiles, 3))
    amp = rng.uniform(0.5, 3.0, (n_tiles, 3))
    bumps = (amp[:, :, None] * np.exp(-((lam[None, None, :] - centre[:, :, None]) ** 2)
                                      / (2.0 * sigma[:, :, None] ** 2))).sum(axis=1)
    mat_k[tile_mat0:] = base[:, None] * (1.0 + bumps)

    sky = blackbody_normalised(lam).astype(np.float32)
    elev = math.radians(35.0)
    sun_dir = np.array([0.0, -math.cos(elev), math.sin(elev)], np.float32)
    tiles = mat_tile = None
    if hetero_tiles:
        # heterogeneous tiles: each window tile takes one of the tile set's tiles in turn
        tiles, tn, tk = tile_set(tile_seed, hetero_tiles)
        mat_tile = np.full(n_mat, -1, np.int32)
        ids = np.arange(n_tiles) % hetero_tiles
        mat_tile[tile_mat0:] = ids
        kind[tile_mat0:] = MAT_TILE
        thick[tile_mat0:] = np.array([tiles[i]["d_mean"] for i in ids], np.float32)
        mat_n[tile_mat0:] = tn[ids]
        mat_k[tile_mat0:] = tk[ids]
    scene = SceneData(
        vertices=v, indices=t, tri_material=m, mat_kind=kind, mat_thickness=thick,
        table_nm=lam, mat_n=mat_n, mat_k=mat_k, mat_albedo=albedo,
        sky=sky, sky_mode=1, sun_dir=sun_dir, sun_half_angle=math.radians(0.2665),
        sun=(5e4 * sky).astype(np.float32), ray_eps=2e-6 * length,
        n_subdomains=n_subdomains, split_axis=0,
        info={"triangles": int(t.shape[0]), "tiles": n_tiles, "materials": n_mat},
        tiles=tiles, mat_tile=mat_tile,
    )
    cam = CameraData(pos=(3.0, 6.0, 1.7), look_at=(4.0, 6.0, 1.7), up=(0.0, 0.0, 1.0),
                     vfov_deg=50.0, width=width, height=height)
    spec = RenderSpec(lambda_nm=lam, spp=spp, seed=seed, max_depth=max_depth, mode=RENDER_MC,
                      rr_start_depth=rr_start_depth)
    return scene, cam, spec


def large_nave_scene(seed: int = 5, n_subdomains: int = 8, spp: int = 64):
    """The large batched frame: the procedural nave refined to ~1.07M triangles (0.1 m wall
    cells) with 96 windows (two rows of 24 per long wall, sills at 2 m and 8 m) of 10 x 40
    heterogeneous tiles each (38,400 tiles drawing on the 512-tile set of seed 3);
    3840 x 2160, 81 wavelengths, depth 16, Russian roulette from depth 3."""
    return nave_scene(seed=seed, cell=0.1, windows_per_wall=24, tiles_x=10, tiles_z=40, sills=(2.0, 8.0),
                      hetero_tiles=512, tile_seed=3, n_subdomains=n_subdomains, width=3840, height=2160, spp=spp,
                      max_depth=16, rr_start_depth=3)


def tile_room_scene(seed: int = 2, n_tiles: int = 16, width: int = 48, height: int = 32, spp: int = 4):
    """A 6 x 6 x 4 m room whose y = 0 wall holds a 1 m x 1 m window of 10 x 10 heterogeneous
    tiles (tiles drawn from a seeded tile set), lit by the sky and a sun at 35 degrees that
    shines through the window onto the floor; camera inside looking at the window."""
    tiles, tn, tk = tile_set(seed, n_tiles)
    lam = SPECTRAL_GRID_81.copy()
    mesh = _Mesh()
    STONE = 0
    c = 0.25
    _grid(mesh, (0, 0, 0), (c, 0, 0), (0, c, 0), 24, 24, STONE)                 # floor
    _grid(mesh, (0, 0, 4), (0, c, 0), (c, 0, 0), 24, 24, STONE)                 # ceiling
    _grid(mesh, (0, 6, 0), (c, 0, 0), (0, 0, c), 24, 16, STONE)                 # back wall
    _grid(mesh, (0, 0, 0), (0, 0, c), (0, c, 0), 16, 24, STONE)                 # x = 0
    _grid(mesh, (6, 0, 0), (0, c, 0), (0, 0, c), 24, 16, STONE)                 # x = 6
    win = lambda i, j: 10 <= i < 14 and 6 <= j < 10  # noqa: E731  (x in [2.5, 3.5), z in [1.5, 2.5))
    _grid(mesh, (0, 0, 0), (0, 0, c), (c, 0, 0), 16, 24, STONE, skip=lambda i, j: win(j, i))
    tm = 1
    for i in range(10):
        for j in range(10):
            xa, za = 2.5 + 0.1 * i, 1.5 + 0.1 * j
            mesh.quad((xa, 0.0, za), (xa + 0.1, 0.0, za), (xa + 0.1, 0.0, za + 0.1), (xa, 0.0, za + 0.1), tm)
            tm += 1
    v, t, m = mesh.arrays()
    n_mat = tm
    ids = np.arange(100) % n_tiles
    kind = np.full(n_mat, MAT_TILE, np.int32)
    kind[STONE] = MAT_DIFFUSE
    mat_tile = np.full(n_mat, -1, np.int32)
    mat_tile[1:] = ids
    thick = np.zeros(n_mat, np.float32)
    thick[1:] = [tiles[i]["d_mean"] for i in ids]
    mat_n = np.ones((n_mat, lam.size), np.float32)
    mat_k = np.zeros((n_mat, lam.size), np.float32)
    mat_n[1:] = tn[ids]
    mat_k[1:] = tk[ids]
    albedo = np.zeros((n_mat, lam.size), np.float32)
    albedo[STONE] = 0.5
    sky = blackbody_normalised(lam).astype(np.float32)
    elev = math.radians(35.0)
    scene = SceneData(
        vertices=v, indices=t, tri_material=m, mat_kind=kind, mat_thickness=thick, table_nm=lam,
        mat_n=mat_n, mat_k=mat_k, mat_albedo=albedo, sky=sky, sky_mode=1,
        sun_dir=np.array([0.0, -math.cos(elev), math.sin(elev)], np.float32), sun_half_angle=math.radians(0.2665),
        sun=(5e4 * sky).astype(np.float32), ray_eps=1e-5, n_subdomains=2, split_axis=0,
        info={"triangles": int(t.shape[0])}, tiles=tiles, mat_tile=mat_tile,
    )
    cam = CameraData(pos=(3.0, 4.5, 1.2), look_at=(3.0, 0.0, 1.6), up=(0.0, 0.0, 1.0), vfov_deg=70.0,
                     width=width, height=height)
    spec = RenderSpec(lambda_nm=lam, spp=spp, seed=seed, max_depth=8, mode=RENDER_MC, rr_start_depth=3)
    return scene, cam, spec


def tile_set(seed: int = 3, n_tiles: int = 512):
    """Heterogeneous tiles: mean thickness U[2.5, 4.5] mm, thickness variation U[0.5, 3] mm
    peak to peak (the field is clamped to 2-5 mm), bubble density 1e4 per cm^3 scaled by
    U[0.5, 1.5], and per-tile Cauchy n(lambda) / banded k(lambda) on the 81-sample grid."""
    rng = np.random.default_rng(seed)
    lam = SPECTRAL_GRID_81
    tiles = [{"d_mean": float(rng.uniform(2.5e-3, 4.5e-3)), "amp": float(rng.uniform(0.5e-3, 3e-3)),
              "rho": float(1e10 * rng.uniform(0.5, 1.5)), "seed": int(rng.integers(1, 2**31))}
             for _ in range(n_tiles)]
    a = rng.uniform(1.50, 1.58, n_tiles)
    b = rng.uniform(0.003, 0.006, n_tiles)
    n = cauchy_n(lam[None, :], a[:, None], b[:, None])
    base = np.exp(rng.uniform(np.log(1e-7), np.log(1e-5), n_tiles))
    centre = rng.uniform(400.0, 700.0, (n_tiles, 3))
    sigma = rng.uniform(15.0, 60.0, (n_tiles, 3))
    amp = rng.uniform(0.5, 3.0, (n_tiles, 3))
    k = base[:, None] * (1.0 + (amp[:, :, None] * np.exp(-((lam[None, None, :] - centre[:, :, None]) ** 2)
                                                          / (2.0 * sigma[:, :, None] ** 2))).sum(axis=1))
    return tiles, n.astype(np.float32), k.astype(np.float32)


def tile_queries(seed: int, n_samples: int, n_tiles: int, tile_n, tile_k):
    """Seeded surrogate queries: |cos(theta_in)| ~ U(0, 1] with either face equally likely (the
    sign: > 0 the flat front face, < 0 the rough back), phi_in ~ U[0, 2 pi), lambda uniform on the
    81-sample grid, tile uniform; n and k looked up from the tile's tables."""
    rng = np.random.default_rng(seed)
    cos_in = (1.0 - rng.uniform(0.0, 1.0, n_samples)) * np.where(rng.uniform(0.0, 1.0, n_samples) < 0.5, 1.0, -1.0)
    cos_in = cos_in.astype(np.float32)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_samples).astype(np.float32)
    li = rng.integers(0, SPECTRAL_GRID_81.size, n_samples)
    tile = rng.integers(0, n_tiles, n_samples).astype(np.int32)
    return {"cos_in": cos_in, "phi_in": phi, "lambda_nm": SPECTRAL_GRID_81[li].astype(np.float32),
            "lambda_index": li.astype(np.int32), "n": tile_n[tile, li].astype(np.float32),
            "k": tile_k[tile, li].astype(np.float32), "tile": tile}


def surrogate_init(seed: int = 4):
    """Initial state of the tile-BTDF network: Fourier matrix B [16, 7] ~ N(0, 1) and layer
    weights W [in, out] ~ U(-a, a), a = sqrt(6 / (in + out)) (Glorot), biases 0.  Layer
    widths 48 -> 128 -> 128 -> 128 -> 128 -> 16."""
    rng = np.random.default_rng(seed)
    B = rng.normal(0.0, 1.0, (16, 7))
    params = []
    for n_in, n_out in ((48, 128), (128, 128), (128, 128), (128, 128), (128, 16)):
        a = math.sqrt(6.0 / (n_in + n_out))
        params.append((rng.uniform(-a, a, (n_in, n_out)), np.zeros(n_out)))
    return B, params


def tiny_scene(seed: int = 0, n_triangles: int = 32, kinds=(MAT_DIFFUSE,)):
    """A few random triangles inside the unit cube, for intersection tests."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, (n_triangles, 1, 3))
    v = (centres + rng.normal(0.0, 0.15, (n_triangles, 3, 3))).reshape(-1, 3).astype(np.float32)
    t = np.arange(3 * n_triangles, dtype=np.uint32).reshape(-1, 3)
    lam = np.array([550.0], np.float32)
    nm = len(kinds)
    m = rng.integers(0, nm, n_triangles).astype(np.uint16)
    return SceneData(
        vertices=v, indices=t, tri_material=m, mat_kind=np.asarray(kinds, np.int32),
        mat_thickness=np.full(nm, 0.003, np.float32), table_nm=lam,
        mat_n=np.full((nm, 1), 1.5, np.float32), mat_k=np.full((nm, 1), 1e-6, np.float32),
        mat_albedo=np.full((nm, 1), 0.5, np.float32), sky=np.ones(1, np.float32), sky_mode=0,
        sun_dir=np.array([0, 0, 1], np.float32), sun_half_angle=0.0, sun=None, ray_eps=1e-5,
    )


def random_rays(seed: int, n: int, lo=-0.2, hi=1.2):
    """Rays from random points toward random points of the unit cube (float32)."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(lo, hi, (n, 3))
    target = rng.uniform(0.2, 0.8, (n, 3))
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)
