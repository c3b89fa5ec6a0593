"""ctypes binding of libsdd (include/sdd.h).  Argument marshalling only: every step of the
render runs in the library's CUDA kernels.  Loading fails loudly when the library has not
been built; there is no CPU fallback.

Functions keep the C names.  Device buffers are passed as torch CUDA tensors (their data
pointers), host inputs as numpy arrays, streams as torch streams (or None for the current
stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsdd.so")
_lib = None

SDD_MODE_DETERMINISTIC = 0
SDD_MODE_MONTE_CARLO = 1
STATUS_NAMES = {0: "SDD_OK", -1: "SDD_ERR_ARG", -2: "SDD_ERR_OOM", -3: "SDD_ERR_CUDA",
                -4: "SDD_ERR_QUEUE_OVERFLOW", -5: "SDD_ERR_TIMEOUT", -6: "SDD_ERR_STATE", -7: "SDD_ERR_STACK"}


class SddError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sdd_material(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_lambda", C.c_int), ("lambda_nm", C.c_void_p),
                ("n", C.c_void_p), ("k", C.c_void_p), ("thickness_m", C.c_float),
                ("albedo", C.c_void_p), ("tile_param_id", C.c_int)]


class sdd_illuminant(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("lambda_nm", C.c_void_p), ("sky_radiance", C.c_void_p),
                ("sky_mode", C.c_int), ("sun_dir", C.c_float * 3), ("sun_half_angle_rad", C.c_float),
                ("sun_radiance", C.c_void_p)]


class sdd_scene_desc(C.Structure):
    _fields_ = [("n_vertices", C.c_int), ("vertices", C.c_void_p), ("n_triangles", C.c_int),
                ("indices", C.c_void_p), ("material_of_triangle", C.c_void_p),
                ("n_materials", C.c_int), ("materials", C.c_void_p), ("illum", sdd_illuminant),
                ("n_subdomains", C.c_int), ("split_axis", C.c_int), ("ray_epsilon_m", C.c_float),
                ("tiles", C.c_void_p), ("slab_polarisation", C.c_int)]


class sdd_camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("orthographic", C.c_int), ("ortho_height_m", C.c_float)]


class sdd_render_opts(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("lambda_nm", C.c_void_p), ("spp", C.c_int),
                ("seed", C.c_uint64), ("max_depth", C.c_int), ("mode", C.c_int),
                ("rr_start_depth", C.c_int), ("use_surrogate", C.c_int), ("batched", C.c_int),
                ("n_pixels", C.c_int), ("pixels", C.c_void_p), ("wave_paths", C.c_int),
                ("path_radiance_out", C.c_void_p), ("path_hash_out", C.c_void_p), ("surrogate", C.c_void_p),
                ("bundle", C.c_int), ("photon_maps", C.c_void_p)]


class sdd_photon_opts(C.Structure):
    _fields_ = [("n_lambda", C.c_int), ("lambda_nm", C.c_void_p), ("n_per_lambda", C.c_int), ("seed", C.c_uint64),
                ("max_depth", C.c_int), ("center", C.c_float * 3), ("radius_m", C.c_float),
                ("distance_m", C.c_float), ("gather_radius_m", C.c_float)]


class sdd_stats(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("ms_raygen", "ms_traverse", "ms_shade", "ms_shadow", "ms_film",
                                           "ms_total")] + \
               [(n, C.c_int64) for n in ("launches_raygen", "launches_traverse", "launches_shade",
                                          "launches_shadow", "launches_film", "launches_total", "rays_closest",
                                          "rays_shadow", "node_visits", "tri_tests", "shadow_node_visits",
                                          "shadow_tri_tests", "crossings", "paths", "waves", "bytes_ray_state")] + \
               [("ms_persistent", C.c_double), ("launches_persistent", C.c_int64), ("graph_replays", C.c_int64),
                ("ms_tile", C.c_double), ("launches_tile", C.c_int64), ("tile_shaded", C.c_int64),
                ("wave_splits", C.c_int64), ("subdomain_loads", C.c_int64), ("bytes_streamed", C.c_int64)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class sdd_train_opts(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("seed", C.c_uint64)]


class sdd_tileset_desc(C.Structure):
    _fields_ = [("n_tiles", C.c_int), ("d_mean_m", C.c_void_p), ("amplitude_m", C.c_void_p),
                ("bubble_density_m3", C.c_void_p), ("seed", C.c_void_p), ("grid", C.c_int),
                ("tile_size_m", C.c_float)]


class sdd_tuning(C.Structure):
    _fields_ = [("traverse_block", C.c_int), ("top_nodes", C.c_int), ("wave_paths", C.c_int), ("no_graph", C.c_int),
                ("queue_capacity", C.c_int), ("block_chunks", C.c_int), ("resident_subdomains", C.c_int)]


class sdd_scene_info(C.Structure):
    _fields_ = [("n_triangles", C.c_int), ("n_subdomains", C.c_int), ("split_axis", C.c_int),
                ("bvh_max_depth", C.c_int), ("n_tri_refs", C.c_int64), ("n_nodes", C.c_int64),
                ("device_bytes", C.c_int64), ("planes", C.c_float * 65)]


class sdd_bvh_info(C.Structure):
    _fields_ = [("n_subdomains", C.c_int), ("split_axis", C.c_int), ("bvh_max_depth", C.c_int),
                ("stack_need", C.c_int), ("n_nodes", C.c_int64), ("n_tri_records", C.c_int64),
                ("slop", C.c_float)]


def lib():
    """Load libsdd.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(the renderer has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32 = C.c_void_p, C.c_int
        L.sdd_scene_create.argtypes = [C.POINTER(sdd_scene_desc), C.POINTER(vp)]
        L.sdd_scene_destroy.argtypes = [vp]
        L.sdd_scene_destroy.restype = None
        L.sdd_render.argtypes = [vp, C.POINTER(sdd_camera), C.POINTER(sdd_render_opts), vp, vp, vp]
        L.sdd_render_to_host.argtypes = [vp, C.POINTER(sdd_camera), C.POINTER(sdd_render_opts), vp, vp, vp]
        L.sdd_set_profiling.argtypes = [vp, i32]
        L.sdd_get_stats.argtypes = [vp, C.POINTER(sdd_stats)]
        L.sdd_set_tuning.argtypes = [vp, C.POINTER(sdd_tuning)]
        L.sdd_get_tuning.argtypes = [vp, C.POINTER(sdd_tuning)]
        L.sdd_scene_get_info.argtypes = [vp, C.POINTER(sdd_scene_info)]
        L.sdd_bvh_build_host.argtypes = [C.POINTER(sdd_scene_desc), C.POINTER(sdd_bvh_info), vp, C.c_int64, vp,
                                         C.c_int64, vp, vp, vp]
        L.sdd_trace_closest.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.sdd_trace_closest_noalloc.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.sdd_eval_optics.argtypes = [i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
        L.sdd_philox.argtypes = [i32, vp, C.c_uint64, vp, vp]
        L.sdd_tileset_create.argtypes = [C.POINTER(sdd_tileset_desc), C.POINTER(vp)]
        L.sdd_tileset_destroy.argtypes = [vp]
        L.sdd_tileset_destroy.restype = None
        L.sdd_tileset_heights.argtypes = [vp, i32, vp]
        u32, u64, f32 = C.c_uint32, C.c_uint64, C.c_float
        L.sdd_tile_trace_rays.argtypes = [vp, i32, i32, vp, vp, f32, f32, f32, vp, vp, u32, u32, u64, i32, vp, vp, vp,
                                          vp, vp, vp]
        L.sdd_tile_generate.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, i32, u64, i32, vp, vp]
        L.sdd_surrogate_param_count.restype = i32
        L.sdd_surrogate_create.argtypes = [vp, vp, i32, i32, C.POINTER(vp)]
        L.sdd_surrogate_destroy.argtypes = [vp]
        L.sdd_surrogate_destroy.restype = None
        L.sdd_surrogate_get_params.argtypes = [vp, vp, i32]
        L.sdd_surrogate_set_params.argtypes = [vp, vp, i32]
        L.sdd_surrogate_gradients.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.sdd_surrogate_train_step.argtypes = [vp, i32, vp, vp, f32, vp, vp]
        L.sdd_surrogate_infer.argtypes = [vp, i32, vp, vp, vp]
        L.sdd_surrogate_train.argtypes = [vp, i32, vp, vp, C.POINTER(sdd_train_opts), vp, vp]
        L.sdd_surrogate_get_weights.argtypes = [vp, vp, C.c_size_t]
        L.sdd_surrogate_set_weights.argtypes = [vp, vp, C.c_size_t]
        L.sdd_photon_maps_build.argtypes = [vp, C.POINTER(sdd_photon_opts), C.POINTER(vp), vp]
        L.sdd_photon_maps_destroy.argtypes = [vp]
        L.sdd_photon_maps_destroy.restype = None
        L.sdd_photon_maps_count.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.sdd_photon_maps_get.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.sdd_photon_gather.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.sdd_last_error.restype = C.c_char_p
        L.sdd_version.restype = C.c_char_p
        for name in ("sdd_scene_create", "sdd_render", "sdd_render_to_host", "sdd_set_profiling", "sdd_get_stats",
                     "sdd_scene_get_info", "sdd_trace_closest", "sdd_trace_closest_noalloc", "sdd_eval_optics",
                     "sdd_philox", "sdd_set_tuning", "sdd_get_tuning", "sdd_tileset_create", "sdd_tileset_heights",
                     "sdd_tile_trace_rays", "sdd_tile_generate", "sdd_surrogate_create", "sdd_surrogate_get_params",
                     "sdd_surrogate_set_params", "sdd_surrogate_gradients", "sdd_surrogate_train_step",
                     "sdd_surrogate_infer", "sdd_watchdog_selftest", "sdd_surrogate_train",
                     "sdd_surrogate_get_weights", "sdd_surrogate_set_weights", "sdd_photon_maps_build",
                     "sdd_photon_maps_count", "sdd_photon_maps_get", "sdd_photon_gather"):
            getattr(L, name).restype = C.c_int
        L.sdd_watchdog_selftest.argtypes = [C.c_int]
        _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise SddError(st, lib().sdd_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ----------------------------------------------------------------------------- scene
def _scene_desc(sd, n_subdomains=None, split_axis=None, ray_epsilon_m=None, tileset=None):
    """The sdd_scene_desc of a ``scenes.SceneData`` and the arrays it points into (keep them
    alive while the descriptor is in use)."""
    keep = []

    def P(a, dt):
        a = _c(a, dt)
        keep.append(a)
        return C.c_void_p(a.ctypes.data)

    M = int(sd.mat_kind.shape[0])
    mats = (sdd_material * M)()
    lam = P(sd.table_nm, np.float32)
    nt = int(sd.table_nm.shape[0])
    mat_n = _c(sd.mat_n, np.float32)
    mat_k = _c(sd.mat_k, np.float32)
    alb = _c(sd.mat_albedo, np.float32)
    keep += [mat_n, mat_k, alb]
    for m in range(M):
        mats[m].kind = int(sd.mat_kind[m])
        mats[m].n_lambda = nt
        mats[m].lambda_nm = lam
        mats[m].n = C.c_void_p(mat_n.ctypes.data + 4 * nt * m)
        mats[m].k = C.c_void_p(mat_k.ctypes.data + 4 * nt * m)
        mats[m].albedo = C.c_void_p(alb.ctypes.data + 4 * nt * m)
        mats[m].thickness_m = float(sd.mat_thickness[m])
        mats[m].tile_param_id = int(sd.mat_tile[m]) if sd.mat_tile is not None else 0
    d = sdd_scene_desc()
    d.n_vertices = int(sd.vertices.shape[0])
    d.vertices = P(sd.vertices, np.float32)
    d.n_triangles = int(sd.indices.shape[0])
    d.indices = P(sd.indices, np.uint32)
    d.material_of_triangle = P(sd.tri_material, np.uint16)
    d.n_materials = M
    d.materials = C.cast(mats, C.c_void_p)
    il = d.illum
    il.n_lambda = nt
    il.lambda_nm = lam
    il.sky_radiance = P(sd.sky, np.float32)
    il.sky_mode = int(sd.sky_mode)
    for i in range(3):
        il.sun_dir[i] = float(sd.sun_dir[i])
    il.sun_half_angle_rad = float(sd.sun_half_angle)
    il.sun_radiance = P(sd.sun, np.float32) if sd.sun is not None else None
    d.n_subdomains = int(sd.n_subdomains if n_subdomains is None else n_subdomains)
    d.split_axis = int(sd.split_axis if split_axis is None else split_axis)
    d.ray_epsilon_m = float(sd.ray_eps if ray_epsilon_m is None else ray_epsilon_m)
    d.tiles = tileset
    d.slab_polarisation = int(getattr(sd, "slab_polarisation", 0))
    keep.append(mats)
    return d, keep


def sdd_scene_create(sd, n_subdomains=None, split_axis=None, ray_epsilon_m=None, tileset=None):
    """Create a device scene from a ``scenes.SceneData``; returns the opaque handle.  Scenes
    with heterogeneous tiles need ``tileset`` (an sdd_tileset handle built from sd.tiles)."""
    d, keep = _scene_desc(sd, n_subdomains, split_axis, ray_epsilon_m, tileset)
    h = C.c_void_p()
    _check(lib().sdd_scene_create(C.byref(d), C.byref(h)))
    return h


# Layout of the BVH node and triangle record sdd_bvh_build_host returns (child c in element c).
BVH_NODE = np.dtype([("lo_x", "<f4", 4), ("hi_x", "<f4", 4), ("lo_y", "<f4", 4), ("hi_y", "<f4", 4),
                     ("lo_z", "<f4", 4), ("hi_z", "<f4", 4), ("link", "<i4", 4), ("count", "<i4", 4)])
BVH_TRI = np.dtype([("v0", "<f4", 3), ("prim", "<u4"), ("v1", "<f4", 3), ("pad1", "<u4"), ("v2", "<f4", 3),
                    ("pad2", "<u4")])


def sdd_bvh_build_host(sd, n_subdomains=None, split_axis=None, ray_epsilon_m=None) -> dict:
    """The subdomain split and BVHs sdd_scene_create would build for ``sd``, built on the host
    (no device): info fields, nodes (BVH_NODE), triangle records (BVH_TRI), per-subdomain root
    and node count, and the planes."""
    d, keep = _scene_desc(sd, n_subdomains, split_axis, ray_epsilon_m)
    info = sdd_bvh_info()
    L = lib()
    _check(L.sdd_bvh_build_host(C.byref(d), C.byref(info), None, 0, None, 0, None, None, None))
    n_sub = info.n_subdomains
    nodes = np.zeros(info.n_nodes, BVH_NODE)
    tris = np.zeros(info.n_tri_records, BVH_TRI)
    root = np.zeros(n_sub, np.int32)
    nn = np.zeros(n_sub, np.int32)
    planes = np.zeros(n_sub + 1, np.float32)
    _check(L.sdd_bvh_build_host(C.byref(d), C.byref(info), nodes.ctypes.data, nodes.size, tris.ctypes.data,
                                tris.size, root.ctypes.data, nn.ctypes.data, planes.ctypes.data))
    out = {f[0]: getattr(info, f[0]) for f in info._fields_}
    out.update(nodes=nodes, tris=tris, root=root, n_nodes_sub=nn, planes=planes)
    return out


def sdd_scene_destroy(h):
    lib().sdd_scene_destroy(h)


def sdd_scene_get_info(h) -> dict:
    info = sdd_scene_info()
    _check(lib().sdd_scene_get_info(h, C.byref(info)))
    out = {f[0]: getattr(info, f[0]) for f in info._fields_ if f[0] != "planes"}
    out["planes"] = [info.planes[i] for i in range(info.n_subdomains + 1)]
    return out


def make_camera(cam) -> sdd_camera:
    c = sdd_camera()
    for i in range(3):
        c.pos[i], c.look_at[i], c.up[i] = cam.pos[i], cam.look_at[i], cam.up[i]
    c.vfov_deg = cam.vfov_deg
    c.width, c.height = cam.width, cam.height
    c.orthographic = cam.ortho
    c.ortho_height_m = cam.ortho_height
    return c


def make_opts(spec, pixels=None, wave_paths=0, batched=0, path_radiance_out=None, path_hash_out=None,
              use_surrogate=0, surrogate=None, photon_maps=None):
    keep = []
    o = sdd_render_opts()
    lam = _c(spec.lambda_nm, np.float32)
    keep.append(lam)
    o.n_lambda = lam.size
    o.lambda_nm = C.c_void_p(lam.ctypes.data)
    o.spp = spec.spp
    o.seed = spec.seed
    o.max_depth = spec.max_depth
    o.mode = spec.mode
    o.rr_start_depth = min(spec.rr_start_depth, 2**31 - 1)
    o.use_surrogate = use_surrogate
    o.batched = batched
    if pixels is not None:
        px = _c(pixels, np.int32)
        keep.append(px)
        o.n_pixels = px.size
        o.pixels = C.c_void_p(px.ctypes.data)
    o.wave_paths = wave_paths
    o.path_radiance_out = _ptr(path_radiance_out)
    o.path_hash_out = _ptr(path_hash_out)
    o.surrogate = surrogate.h if surrogate is not None else None
    o.bundle = getattr(spec, "bundle", 1)
    o.photon_maps = photon_maps.h if photon_maps is not None else None
    o._keep = keep
    return o


def sdd_render(h, cam, spec, spectral_out, xyz_out=None, stream=None, **kw):
    """Render into device tensors spectral_out [n_px, L] and xyz_out [n_px, 3] (float32)."""
    c = make_camera(cam)
    o = make_opts(spec, **kw)
    _check(lib().sdd_render(h, C.byref(c), C.byref(o), _ptr(spectral_out), _ptr(xyz_out), _stream(stream)))


def sdd_render_to_host(h, cam, spec, spectral_out, xyz_out=None, stream=None, **kw):
    """Render into HOST buffers (numpy arrays or pinned CPU tensors); the library copies back."""
    c = make_camera(cam)
    o = make_opts(spec, **kw)
    _check(lib().sdd_render_to_host(h, C.byref(c), C.byref(o), _ptr(spectral_out), _ptr(xyz_out), _stream(stream)))


def sdd_set_profiling(h, level: int):
    _check(lib().sdd_set_profiling(h, int(level)))


def sdd_watchdog_selftest(timeout_ms: int = 200):
    """Runs the batched form's grid barrier with one block that never arrives; raises
    SddError(SDD_ERR_TIMEOUT) when the watchdog fired (the expected outcome)."""
    _check(lib().sdd_watchdog_selftest(int(timeout_ms)))


def sdd_set_tuning(h, tuning: dict):
    t = sdd_tuning(**{k: int(v) for k, v in tuning.items()})
    _check(lib().sdd_set_tuning(h, C.byref(t)))


def sdd_get_tuning(h) -> dict:
    t = sdd_tuning()
    _check(lib().sdd_get_tuning(h, C.byref(t)))
    return {f[0]: getattr(t, f[0]) for f in t._fields_}


def sdd_get_stats(h) -> dict:
    s = sdd_stats()
    _check(lib().sdd_get_stats(h, C.byref(s)))
    return s.as_dict()


def sdd_trace_closest(h, org, dirs, t_out, prim_out, stream=None):
    """Closest hit of n rays: device float [n,3] origins/directions -> t [n], prim [n] (int32)."""
    n = int(org.shape[0])
    _check(lib().sdd_trace_closest(h, n, _ptr(org), _ptr(dirs), _ptr(t_out), _ptr(prim_out), _stream(stream)))


def sdd_trace_closest_noalloc(h, org, dirs, t_out, prim_out, stream=None):
    """As sdd_trace_closest, but out of the library's fixed static scratch (no allocation)."""
    n = int(org.shape[0])
    _check(lib().sdd_trace_closest_noalloc(h, n, _ptr(org), _ptr(dirs), _ptr(t_out), _ptr(prim_out),
                                           _stream(stream)))


def sdd_eval_optics(cos_i, n_re, k, d, lam, R, Rs, Ts, stream=None, slab_polarisation=0):
    n = int(cos_i.numel())
    _check(lib().sdd_eval_optics(n, _ptr(cos_i), _ptr(n_re), _ptr(k), _ptr(d), _ptr(lam), int(slab_polarisation),
                                 _ptr(R), _ptr(Rs), _ptr(Ts), _stream(stream)))


def sdd_philox(ctr, key: int, out, stream=None):
    n = int(ctr.shape[0])
    _check(lib().sdd_philox(n, _ptr(ctr), C.c_uint64(key), _ptr(out), _stream(stream)))


# ----------------------------------------------------------------------------- tiles
def sdd_tileset_create(tiles, grid=64, tile_size_m=0.1):
    """tiles: list of dicts with d_mean, amp, rho, seed (host values)."""
    keep = [np.ascontiguousarray([t[key] for t in tiles], dtype=dt)
            for key, dt in (("d_mean", np.float32), ("amp", np.float32), ("rho", np.float32), ("seed", np.uint32))]
    d = sdd_tileset_desc(len(tiles), *(C.c_void_p(a.ctypes.data) for a in keep), grid, tile_size_m)
    h = C.c_void_p()
    _check(lib().sdd_tileset_create(C.byref(d), C.byref(h)))
    return h


def sdd_tileset_destroy(h):
    lib().sdd_tileset_destroy(h)


def sdd_tileset_heights(h, tile, grid=64):
    out = np.zeros((grid + 1) * (grid + 1), np.float32)
    _check(lib().sdd_tileset_heights(h, int(tile), C.c_void_p(out.ctypes.data)))
    return out.reshape(grid + 1, grid + 1)


def sdd_tile_trace_rays(h, tile, xy, dirs, n_re, k, lambda_nm, px, sample, bounce, lam, seed, max_events, side, w,
                        dir_out, bubbles, events, stream=None):
    n = int(xy.shape[0])
    _check(lib().sdd_tile_trace_rays(h, int(tile), n, _ptr(xy), _ptr(dirs), float(n_re), float(k), float(lambda_nm),
                                     _ptr(px), _ptr(sample), int(bounce), int(lam), int(seed), int(max_events),
                                     _ptr(side), _ptr(w), _ptr(dir_out), _ptr(bubbles), _ptr(events), _stream(stream)))


def sdd_tile_generate(h, cos_in, phi_in, lambda_nm, n_re, k, tile, rays, seed, max_events, out, stream=None):
    n = int(cos_in.shape[0])
    _check(lib().sdd_tile_generate(h, n, _ptr(cos_in), _ptr(phi_in), _ptr(lambda_nm), _ptr(n_re), _ptr(k), _ptr(tile),
                                   int(rays), int(seed), int(max_events), _ptr(out), _stream(stream)))


class TileSetHandle:
    def __init__(self, tiles, grid=64, tile_size_m=0.1):
        self.h = sdd_tileset_create(tiles, grid, tile_size_m)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            sdd_tileset_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- surrogate
def flatten_params(params):
    """[(W [in, out], b [out]), ...] -> flat float32 array in the library's layout."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32)])
                           for W, b in params]).astype(np.float32)


def unflatten_params(flat, shapes=((48, 128), (128, 128), (128, 128), (128, 128), (128, 16))):
    out, o = [], 0
    for n_in, n_out in shapes:
        W = flat[o:o + n_in * n_out].reshape(n_in, n_out)
        o += n_in * n_out
        b = flat[o:o + n_out]
        o += n_out
        out.append((W, b))
    return out


class Surrogate:
    """The tile-BTDF network on the GPU (thin wrapper of the sdd_surrogate_* calls)."""

    def __init__(self, fourier_B, params, max_batch=65536):
        flat = flatten_params(params)
        Bm = np.ascontiguousarray(fourier_B, np.float32)
        self.n_params = int(lib().sdd_surrogate_param_count())
        h = C.c_void_p()
        _check(lib().sdd_surrogate_create(C.c_void_p(Bm.ctypes.data), C.c_void_p(flat.ctypes.data), flat.size,
                                          max_batch, C.byref(h)))
        self.h = h

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(lib().sdd_surrogate_get_params(self.h, C.c_void_p(out.ctypes.data), self.n_params))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        _check(lib().sdd_surrogate_set_params(self.h, C.c_void_p(flat.ctypes.data), flat.size))

    def gradients(self, raw, y, stream=None):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        _check(lib().sdd_surrogate_gradients(self.h, int(raw.shape[0]), _ptr(raw), _ptr(y), C.c_void_p(g.ctypes.data),
                                             C.byref(loss), _stream(stream)))
        return float(loss.value), g

    def train_step(self, raw, y, lr=1e-3, stream=None):
        loss = C.c_float()
        _check(lib().sdd_surrogate_train_step(self.h, int(raw.shape[0]), _ptr(raw), _ptr(y), C.c_float(lr),
                                              C.byref(loss), _stream(stream)))
        return float(loss.value)

    def train(self, raw, y, steps, batch=65536, lr=1e-3, seed=4, stream=None):
        """A whole training run through sdd_surrogate_train; returns the per-step losses."""
        n = int(raw.shape[0])
        o = sdd_train_opts(int(steps), int(min(batch, n)), float(lr), int(seed))
        losses = np.zeros(int(steps), np.float32)
        _check(lib().sdd_surrogate_train(self.h, n, _ptr(raw), _ptr(y), C.byref(o), C.c_void_p(losses.ctypes.data),
                                         _stream(stream)))
        return losses

    def weights(self) -> bytes:
        buf = C.create_string_buffer(4 * self.n_params)
        _check(lib().sdd_surrogate_get_weights(self.h, buf, C.c_size_t(4 * self.n_params)))
        return buf.raw

    def set_weights(self, data: bytes):
        buf = C.create_string_buffer(bytes(data), len(data))
        _check(lib().sdd_surrogate_set_weights(self.h, buf, C.c_size_t(len(data))))

    def infer(self, raw, out, stream=None):
        _check(lib().sdd_surrogate_infer(self.h, int(raw.shape[0]), _ptr(raw), _ptr(out), _stream(stream)))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sdd_surrogate_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MAP_CAUSTIC, MAP_GLOBAL = 0, 1


class PhotonMaps:
    """Caustic and global photon maps of a scene (Sec. 3.2), built on the device by
    sdd_photon_maps_build; pass as ``photon_maps=`` to a render."""

    def __init__(self, scene_h, lambda_nm, n_per_lambda, seed, center, radius, distance, gather_radius, max_depth=16,
                 stream=None):
        lam = _c(lambda_nm, np.float32)
        o = sdd_photon_opts()
        o.n_lambda = lam.size
        o.lambda_nm = C.c_void_p(lam.ctypes.data)
        o.n_per_lambda = int(n_per_lambda)
        o.seed = int(seed)
        o.max_depth = int(max_depth)
        o.center[:] = [float(c) for c in center]
        o.radius_m = float(radius)
        o.distance_m = float(distance)
        o.gather_radius_m = float(gather_radius)
        self.h = C.c_void_p()
        _check(lib().sdd_photon_maps_build(scene_h, C.byref(o), C.byref(self.h), _stream(stream)))

    def count(self, m: int) -> int:
        a, b = C.c_int64(), C.c_int64()
        _check(lib().sdd_photon_maps_count(self.h, C.byref(a), C.byref(b)))
        return int(a.value if m == MAP_CAUSTIC else b.value)

    def photons(self, m: int) -> dict:
        """The photons of map m as host arrays, in no particular order."""
        n = self.count(m)
        out = {"pos": np.zeros((n, 3), np.float32), "nrm": np.zeros((n, 3), np.float32),
               "power": np.zeros(n, np.float32), "lam": np.zeros(n, np.int32), "id": np.zeros(n, np.uint32),
               "seq": np.zeros(n, np.uint32)}
        if n:
            _check(lib().sdd_photon_maps_get(self.h, int(m), *(C.c_void_p(out[k].ctypes.data)
                                                               for k in ("pos", "nrm", "power", "lam", "id", "seq"))))
        return out

    def gather(self, x, nrm, lam, e_caustic, e_global, stream=None):
        """Density estimates at device points x [n, 3] with unit normals nrm [n, 3] and
        wavelength indices lam [n] (int32) into device e_caustic [n], e_global [n]."""
        _check(lib().sdd_photon_gather(self.h, int(lam.numel()), _ptr(x), _ptr(nrm), _ptr(lam), _ptr(e_caustic),
                                       _ptr(e_global), _stream(stream)))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sdd_photon_maps_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sdd_last_error() -> str:
    return lib().sdd_last_error().decode(errors="replace")


def sdd_version() -> str:
    return lib().sdd_version().decode()


class SceneHandle:
    """RAII wrapper around an sdd_scene handle (and the tile set of its heterogeneous tiles)."""

    def __init__(self, sd, **kw):
        self.tiles = None
        if sd.tiles:
            self.tiles = sdd_tileset_create(sd.tiles, sd.tile_grid, sd.tile_size)
            kw["tileset"] = self.tiles
        self.h = sdd_scene_create(sd, **kw)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            sdd_scene_destroy(self.h)
        self.h = None
        if getattr(self, "tiles", None) is not None and self.tiles.value:
            sdd_tileset_destroy(self.tiles)
        self.tiles = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
