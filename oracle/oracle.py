"""ctypes binding of the FP64 CPU oracle (``sdd_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the bench's CPU-baseline leg
are the only users.  The CUDA library never loads it, and it never loads the CUDA library.
``build()`` compiles the shared library with the host C++ compiler (no GPU needed).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdd_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++, -O2, portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class OrcScene(C.Structure):
    _fields_ = [
        ("n_vertices", C.c_int), ("vertices", C.c_void_p),
        ("n_triangles", C.c_int), ("indices", C.c_void_p), ("tri_material", C.c_void_p),
        ("n_materials", C.c_int), ("mat_kind", C.c_void_p), ("mat_thickness", C.c_void_p),
        ("n_table", C.c_int), ("table_nm", C.c_void_p),
        ("mat_n", C.c_void_p), ("mat_k", C.c_void_p), ("mat_albedo", C.c_void_p),
        ("sky", C.c_void_p), ("sky_mode", C.c_int),
        ("sun_dir", C.c_float * 3), ("sun_half_angle", C.c_float), ("sun", C.c_void_p),
        ("ray_eps", C.c_float), ("n_tiles", C.c_int), ("tiles", C.c_void_p), ("mat_tile", C.c_void_p),
        ("tile_grid", C.c_int), ("tile_size", C.c_double), ("slab_polarisation", C.c_int),
    ]


class OrcCamera(C.Structure):
    _fields_ = [
        ("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
        ("vfov_deg", C.c_float), ("width", C.c_int), ("height", C.c_int),
        ("ortho", C.c_int), ("ortho_height", C.c_float),
    ]


class OrcOpts(C.Structure):
    _fields_ = [
        ("n_lambda", C.c_int), ("lambda_nm", C.c_void_p), ("spp", C.c_int),
        ("seed", C.c_uint64), ("max_depth", C.c_int), ("mode", C.c_int),
        ("rr_start_depth", C.c_int), ("n_pixels", C.c_int), ("pixels", C.c_void_p),
        ("n_threads", C.c_int), ("bundle", C.c_int), ("photons", C.c_void_p),
    ]


class OrcPhotonOpts(C.Structure):
    _fields_ = [
        ("n_per_lambda", C.c_int), ("seed", C.c_uint64), ("max_depth", C.c_int), ("center", C.c_float * 3),
        ("radius", C.c_float), ("distance", C.c_float), ("gather_radius", C.c_float), ("n_threads", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_scene_create.restype = C.c_void_p
        _lib.orc_scene_create.argtypes = [C.POINTER(OrcScene)]
        _lib.orc_scene_destroy.argtypes = [C.c_void_p]
        _lib.orc_render.restype = C.c_int
        _lib.orc_render.argtypes = [C.c_void_p, C.POINTER(OrcCamera), C.POINTER(OrcOpts),
                                    C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_closest.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p, C.c_void_p]
        _lib.orc_beer_lambert.restype = C.c_double
        _lib.orc_beer_lambert.argtypes = [C.c_double, C.c_double, C.c_double]
        _lib.orc_cone_dir.argtypes = [C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
        _lib.orc_hardware_threads.restype = C.c_int
        _lib.orc_photons_trace.restype = C.c_void_p
        _lib.orc_photons_trace.argtypes = [C.c_void_p, C.POINTER(OrcPhotonOpts), C.c_int, C.c_void_p]
        _lib.orc_photons_destroy.argtypes = [C.c_void_p]
        _lib.orc_photons_count.restype = C.c_int64
        _lib.orc_photons_count.argtypes = [C.c_void_p, C.c_int]
        _lib.orc_photons_get.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 5
        _lib.orc_photons_gather.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 5
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ----------------------------------------------------------------------------- physics
def philox(ctr, key):
    ctr = _c(ctr, np.uint32).reshape(-1, 4)
    key = _c(key, np.uint32).reshape(2)
    out = np.zeros_like(ctr)
    lib().orc_philox(ctr.shape[0], _p(ctr), _p(key), _p(out))
    return out


def fresnel(cos_i, n1, n2_re, n2_im):
    """Unpolarised, s and p reflectance: returns (R, Rs, Rp)."""
    cos_i, n1, n2_re, n2_im = np.broadcast_arrays(*(np.asarray(x, np.float64) for x in (cos_i, n1, n2_re, n2_im)))
    args = [_c(x, np.float64).ravel() for x in (cos_i, n1, n2_re, n2_im)]
    n = args[0].size
    R, Rs, Rp = (np.zeros(n) for _ in range(3))
    lib().orc_fresnel(n, *(_p(a) for a in args), _p(R), _p(Rs), _p(Rp))
    shp = cos_i.shape
    return R.reshape(shp), Rs.reshape(shp), Rp.reshape(shp)


def slab(cos_i, n, k, d_m, lambda_nm, pol=0):
    """Thin-slab (R, T); pol = 1 runs the series for s and p separately and averages."""
    arrs = np.broadcast_arrays(*(np.asarray(x, np.float64) for x in (cos_i, n, k, d_m, lambda_nm)))
    args = [_c(x, np.float64).ravel() for x in arrs]
    m = args[0].size
    R, T = np.zeros(m), np.zeros(m)
    lib().orc_slab(m, *(_p(a) for a in args), int(pol), _p(R), _p(T))
    return R.reshape(arrs[0].shape), T.reshape(arrs[0].shape)


def beer_lambert(k, len_m, lambda_nm):
    return lib().orc_beer_lambert(float(k), float(len_m), float(lambda_nm))


def cmf(lambda_nm):
    lam = _c(lambda_nm, np.float64).ravel()
    out = np.zeros((lam.size, 3))
    lib().orc_cmf(lam.size, _p(lam), _p(out))
    return out


def cosine_dir(nrm, u):
    nrm = _c(nrm, np.float64).reshape(-1, 3)
    u = _c(u, np.float64).reshape(-1, 2)
    out = np.zeros_like(nrm)
    lib().orc_cosine_dir(nrm.shape[0], _p(nrm), _p(u), _p(out))
    return out


def cone_dir(axis, h, u):
    axis = _c(axis, np.float64).reshape(-1, 3)
    u = _c(u, np.float64).reshape(-1, 2)
    out = np.zeros_like(axis)
    lib().orc_cone_dir(axis.shape[0], _p(axis), C.c_double(h), _p(u), _p(out))
    return out


def xyz(film, lambda_nm):
    film = _c(film, np.float64)
    lam = _c(lambda_nm, np.float32)
    npx = film.size // lam.size
    out = np.zeros((npx, 3))
    lib().orc_xyz(npx, lam.size, _p(lam), _p(film), _p(out))
    return out


class OrcTile(C.Structure):
    _fields_ = [("d_mean", C.c_double), ("amp", C.c_double), ("rho", C.c_double), ("seed", C.c_uint32)]


TILE_BINS = 8
TILE_STAT_COLS = 4 + 2 * TILE_BINS


def _tiles(tiles):
    arr = (OrcTile * len(tiles))()
    for i, t in enumerate(tiles):
        arr[i].d_mean, arr[i].amp, arr[i].rho, arr[i].seed = t["d_mean"], t["amp"], t["rho"], t["seed"]
    return arr


def tile_heights(tile, G=64, L=0.1):
    """Tile thickness at the (G+1)^2 grid vertices (row j, column i), metres."""
    h = np.zeros((G + 1) * (G + 1))
    lib().orc_tile_heights(_tiles([tile]), G, C.c_double(L), _p(h))
    return h.reshape(G + 1, G + 1)


def tile_trace(tile, heights, xy, dirs, n_re, k, lambda_nm, px, sample, bounce=1, lam=0, seed=0, max_events=64,
               G=64, L=0.1):
    """Trace rays through one tile; returns dict of side, w, dir, bubbles, events."""
    h = _c(heights, np.float64).ravel()
    xy = _c(xy, np.float64).reshape(-1, 2)
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    n = xy.shape[0]
    px = _c(np.broadcast_to(px, (n,)), np.uint32)
    sample = _c(np.broadcast_to(sample, (n,)), np.uint32)
    side = np.zeros(n, np.int32)
    w = np.zeros(n)
    dout = np.zeros((n, 3))
    bub = np.zeros(n, np.int32)
    ev = np.zeros(n, np.int32)
    lib().orc_tile_trace(_tiles([tile]), G, C.c_double(L), _p(h), n, _p(xy), _p(dirs), C.c_double(n_re),
                         C.c_double(k), C.c_double(lambda_nm), _p(px), _p(sample), C.c_uint32(bounce),
                         C.c_uint32(lam), C.c_uint64(seed), max_events, _p(side), _p(w), _p(dout), _p(bub), _p(ev))
    return {"side": side, "w": w, "dir": dout, "bubbles": bub, "events": ev}


def tile_samples(tiles, heights, cos_in, phi_in, lambda_nm, n_re, k, tile, rays=256, seed=0, max_events=64,
                 n_threads=0, G=64, L=0.1):
    """Per-sample statistics [n, 20]: T, R, absorbed, bubbles/ray, then the fraction of T and of R
    in each of 8 deflection-angle bins (edges 0, 1, 2, 4, 8, 16, 32, 64, 180 degrees).
    cos_in > 0 enters through the tile's flat front face, < 0 through its rough back face."""
    hs = _c(heights, np.float64).ravel()
    args = [_c(x, np.float64).ravel() for x in (cos_in, phi_in, lambda_nm, n_re, k)]
    t = _c(tile, np.int32).ravel()
    ns = t.size
    out = np.zeros((ns, TILE_STAT_COLS))
    lib().orc_tile_samples(len(tiles), _tiles(tiles), G, C.c_double(L), _p(hs), ns, *(_p(a) for a in args), _p(t),
                           rays, C.c_uint64(seed), max_events, n_threads, _p(out))
    return out


def hardware_threads() -> int:
    return int(lib().orc_hardware_threads())


# ----------------------------------------------------------------------------- scenes
class OracleScene:
    """An oracle-side copy of a ``scenes.SceneData`` (median-split BVH built on creation)."""

    def __init__(self, sd):
        self._keep = []

        def keep(a, dt):
            a = _c(a, dt)
            self._keep.append(a)
            return _p(a)

        d = OrcScene()
        d.n_vertices = sd.vertices.shape[0]
        d.vertices = keep(sd.vertices, np.float32)
        d.n_triangles = sd.indices.shape[0]
        d.indices = keep(sd.indices, np.uint32)
        d.tri_material = keep(sd.tri_material, np.uint16)
        d.n_materials = sd.mat_kind.shape[0]
        d.mat_kind = keep(sd.mat_kind, np.int32)
        d.mat_thickness = keep(sd.mat_thickness, np.float32)
        d.n_table = sd.table_nm.shape[0]
        d.table_nm = keep(sd.table_nm, np.float32)
        d.mat_n = keep(sd.mat_n, np.float32)
        d.mat_k = keep(sd.mat_k, np.float32)
        d.mat_albedo = keep(sd.mat_albedo, np.float32)
        d.sky = keep(sd.sky, np.float32)
        d.sky_mode = int(sd.sky_mode)
        for i in range(3):
            d.sun_dir[i] = float(sd.sun_dir[i])
        d.sun_half_angle = float(sd.sun_half_angle)
        d.sun = keep(sd.sun, np.float32) if sd.sun is not None else None
        d.ray_eps = float(sd.ray_eps)
        d.slab_polarisation = int(getattr(sd, "slab_polarisation", 0))
        if getattr(sd, "tiles", None):
            arr = _tiles(sd.tiles)
            self._keep.append(arr)
            d.n_tiles = len(sd.tiles)
            d.tiles = C.cast(arr, C.c_void_p)
            d.mat_tile = keep(sd.mat_tile, np.int32)
            d.tile_grid = int(sd.tile_grid)
            d.tile_size = float(sd.tile_size)
        self.h = lib().orc_scene_create(C.byref(d))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_destroy(self.h)
            self.h = None

    def closest(self, org, dirs, brute=False):
        org = _c(org, np.float64).reshape(-1, 3)
        dirs = _c(dirs, np.float64).reshape(-1, 3)
        n = org.shape[0]
        t = np.zeros(n)
        prim = np.zeros(n, np.int32)
        lib().orc_closest(self.h, n, _p(org), _p(dirs), int(brute), _p(t), _p(prim))
        return t, prim

    def photon_maps(self, lambda_nm, n_per_lambda, seed, center, radius, distance, gather_radius, max_depth=16,
                    n_threads=0):
        """Caustic and global photon maps of the sun (Sec. 3.2) for the given wavelengths."""
        return PhotonMaps(self, lambda_nm, n_per_lambda, seed, center, radius, distance, gather_radius, max_depth,
                          n_threads)

    def render(self, cam, spec, pixels=None, n_threads=0, want_paths=False, photons=None):
        """Returns (film [n_px, L], path_L [n_px, spp, L] or None, hash or None)."""
        c = OrcCamera()
        for i in range(3):
            c.pos[i], c.look_at[i], c.up[i] = cam.pos[i], cam.look_at[i], cam.up[i]
        c.vfov_deg = cam.vfov_deg
        c.width, c.height = cam.width, cam.height
        c.ortho, c.ortho_height = cam.ortho, cam.ortho_height
        lam = _c(spec.lambda_nm, np.float32)
        px = None if pixels is None else _c(pixels, np.int32)
        o = OrcOpts()
        o.n_lambda, o.lambda_nm, o.spp = lam.size, _p(lam), spec.spp
        o.seed, o.max_depth, o.mode = spec.seed, spec.max_depth, spec.mode
        o.rr_start_depth = spec.rr_start_depth
        o.n_pixels = 0 if px is None else px.size
        o.pixels = _p(px)
        o.n_threads = n_threads
        o.bundle = getattr(spec, "bundle", 1)
        o.photons = photons.h if photons is not None else None
        npx = cam.width * cam.height if px is None else px.size
        film = np.zeros((npx, lam.size))
        path_L = np.zeros((npx, spec.spp, lam.size)) if want_paths else None
        path_h = np.zeros((npx, spec.spp, lam.size), np.uint32) if want_paths else None
        rc = lib().orc_render(self.h, C.byref(c), C.byref(o), _p(film), _p(path_L), _p(path_h))
        if rc != 0:
            raise ValueError("oracle rejected the render arguments")
        return film, path_L, path_h


def bubble_scatter(d, rad, sin_i, u, n_re, k=0.0, r=50e-6):
    """Sphere optics of one air bubble with the surface choices given: d, rad [n, 3], sin_i [n],
    u [n, m] uniforms taken one per surface met.  Returns (exit direction [n, 3], surfaces met,
    or -1 where the m uniforms ran out inside the bubble)."""
    d = _c(d, np.float64).reshape(-1, 3)
    n = d.shape[0]
    rad = _c(rad, np.float64).reshape(n, 3)
    sin_i = _c(np.broadcast_to(sin_i, (n,)), np.float64)
    u = _c(u, np.float64).reshape(n, -1)
    out = np.zeros((n, 3))
    ev = np.zeros(n, np.int32)
    lib().orc_bubble_scatter(n, _p(d), _p(rad), _p(sin_i), C.c_double(r), C.c_double(n_re), C.c_double(k),
                             u.shape[1], _p(u), _p(out), _p(ev))
    return out, ev


MAP_CAUSTIC, MAP_GLOBAL = 0, 1


class PhotonMaps:
    """Oracle photon maps (a handle of orc_photons_trace)."""

    def __init__(self, osc, lambda_nm, n_per_lambda, seed, center, radius, distance, gather_radius, max_depth,
                 n_threads):
        self.lambda_nm = _c(lambda_nm, np.float32)
        o = OrcPhotonOpts()
        o.n_per_lambda, o.seed, o.max_depth = int(n_per_lambda), int(seed), int(max_depth)
        for i in range(3):
            o.center[i] = float(center[i])
        o.radius, o.distance, o.gather_radius, o.n_threads = radius, distance, gather_radius, n_threads
        self._osc = osc
        self.h = lib().orc_photons_trace(osc.h, C.byref(o), self.lambda_nm.size, _p(self.lambda_nm))
        if not self.h:
            raise ValueError("oracle rejected the photon-map arguments")
        self.radius = float(gather_radius)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_photons_destroy(self.h)
            self.h = None

    def count(self, which):
        return int(lib().orc_photons_count(self.h, which))

    def photons(self, which):
        """dict of pos [n, 3], nrm [n, 3], power [n], lam [n], id [n] of one map."""
        n = self.count(which)
        pos, nrm, pw = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        lam, pid = np.zeros(n, np.int32), np.zeros(n, np.uint32)
        lib().orc_photons_get(self.h, which, _p(pos), _p(nrm), _p(pw), _p(lam), _p(pid))
        return {"pos": pos, "nrm": nrm, "power": pw, "lam": lam, "id": pid}

    def gather(self, x, nrm, lam):
        """Irradiance estimates (caustic, global) at points x [n, 3] with normals nrm [n, 3]."""
        x = _c(x, np.float64).reshape(-1, 3)
        nrm = _c(np.broadcast_to(nrm, x.shape), np.float64)
        lam = _c(np.broadcast_to(lam, (x.shape[0],)), np.int32)
        ec, eg = np.zeros(x.shape[0]), np.zeros(x.shape[0])
        lib().orc_photons_gather(self.h, x.shape[0], _p(x), _p(nrm), _p(lam), _p(ec), _p(eg))
        return ec, eg
