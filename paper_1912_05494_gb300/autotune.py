"""Autotuner for the renderer's launch shape: subdomain count, traversal block size, BVH
levels staged in shared memory and wave size.

The paper's experiment (Sec. 6, Table 1) varies the number of sub-domains at a fixed number
of threads and finds that speed keeps growing with it on their cluster; on one GB300 the best
count depends on the scene, so it is measured.  The tuner times a reduced frame (a seeded
subset of pixels, fewer samples) of the caller's scene for each candidate, by coordinate
descent: subdomain count first (each candidate rebuilds the scene's BVHs), then block size,
then staged top nodes, then wave size.  Results are cached in a JSON file keyed by a hash of
the scene, the frame shape and the device name.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import scenes as S
from . import sdd

DEFAULT_CACHE = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "sdd", "autotune.json")


def scene_key(sd, cam, spec, device_name: str, extra: str = "") -> str:
    h = hashlib.sha256()
    for a in (sd.vertices, sd.indices, sd.tri_material, sd.mat_kind, sd.mat_thickness, sd.mat_n, sd.mat_k):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(json.dumps([cam.width, cam.height, spec.spp, spec.n_lambda, spec.max_depth, spec.mode,
                         device_name, extra]).encode())
    return h.hexdigest()[:24]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, db):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_frame(h, cam, spec, pixels, tuning, repeats=2, render_kw=None):
    """Median seconds of `repeats` renders of the reduced frame with the given tuning."""
    import torch
    kw = render_kw or {}
    sdd.sdd_set_tuning(h, tuning)
    n_px = len(pixels)
    out = torch.empty((n_px, spec.n_lambda), device="cuda", dtype=torch.float32)
    sdd.sdd_render(h, cam, spec, out, pixels=pixels, **kw)  # warm-up (workspace, caches, graph)
    ts = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sdd.sdd_render(h, cam, spec, out, pixels=pixels, **kw)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def autotune(sd, cam, spec, *, subdomains=(1, 2, 4, 8, 16, 32, 64), blocks=(64, 128, 256),
             top_nodes=(0, 63, 255), wave_paths=(1 << 22, 1 << 24, 1 << 26), sample_pixels=65536,
             sample_spp=None, cache_path=DEFAULT_CACHE, use_cache=True, log=None, render_kw=None):
    """Pick the fastest launch shape for rendering `sd` with `cam` / `spec` on this GPU.
    render_kw: extra sdd_render options of the form being tuned (batched, use_surrogate, ...);
    a network passed there is not part of the cache key.

    Returns {"n_subdomains", "tuning": {...}, "seconds", "trials": [...]}.
    """
    import torch
    dev = torch.cuda.get_device_name()
    form = {k: v for k, v in (render_kw or {}).items() if isinstance(v, (int, float, str))}
    key = scene_key(sd, cam, spec, dev, json.dumps([list(subdomains), list(blocks), list(top_nodes),
                                                    list(wave_paths), sample_pixels, sample_spp, form],
                                                   sort_keys=True))
    db = _load(cache_path) if use_cache else {}
    if use_cache and key in db:
        return db[key]
    rng = np.random.default_rng(12345)
    n_all = cam.width * cam.height
    pixels = np.sort(rng.choice(n_all, min(sample_pixels, n_all), replace=False)).astype(np.int32)
    spec_s = S.RenderSpec(**{**spec.__dict__, "spp": sample_spp or spec.spp})
    trials = []

    def note(msg):
        if log:
            log(msg)

    base = {"traverse_block": 128, "top_nodes": 0, "wave_paths": 0, "no_graph": 0}
    best = None
    best_sub = None
    for ns in subdomains:
        h = sdd.SceneHandle(sd, n_subdomains=ns)
        t = time_frame(h.h, cam, spec_s, pixels, base, render_kw=render_kw)
        trials.append({"n_subdomains": ns, **base, "seconds": t})
        note(f"S={ns}: {t * 1e3:.1f} ms")
        if best is None or t < best:
            best, best_sub = t, ns
        h.close()
    h = sdd.SceneHandle(sd, n_subdomains=best_sub)
    cur = dict(base)
    for knob, values in (("traverse_block", blocks), ("top_nodes", top_nodes), ("wave_paths", wave_paths)):
        for v in values:
            cand = {**cur, knob: v}
            if cand == cur and any(t["n_subdomains"] == best_sub and all(t[k] == cur[k] for k in cur) for t in trials):
                continue
            t = time_frame(h.h, cam, spec_s, pixels, cand, render_kw=render_kw)
            trials.append({"n_subdomains": best_sub, **cand, "seconds": t})
            note(f"S={best_sub} {knob}={v}: {t * 1e3:.1f} ms")
            if t < best:
                best, cur = t, cand
    h.close()
    res = {"n_subdomains": best_sub, "tuning": cur, "seconds": best, "device": dev, "sample_pixels": int(len(pixels)),
           "sample_spp": spec_s.spp, "trials": trials}
    if use_cache:
        db[key] = res
        _store(cache_path, db)
    return res
