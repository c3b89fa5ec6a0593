"""The C-ABI library loads on a machine without a GPU and exports every symbol that
include/sdd.h declares; argument validation that needs no device is exercised here too."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd
    return sdd


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdd_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sdd_render" in names and "sdd_scene_create" in names
    L = lib.lib()
    for n in names:
        assert hasattr(L, n), n


def test_null_arguments_are_rejected_without_a_device(lib):
    L = lib.lib()
    out = C.c_void_p()
    assert L.sdd_scene_create(None, C.byref(out)) == -1
    assert b"NULL" in L.sdd_last_error()
    assert L.sdd_render(None, None, None, None, None, None) == -1
    assert L.sdd_trace_closest(None, 1, None, None, None, None, None) == -1
    assert L.sdd_philox(-1, None, 0, None, None) == -1


def test_bad_scene_descriptions_are_rejected(lib):
    from paper_1912_05494_gb300 import scenes as S
    sc, _, _ = S.slab_scene(0)
    bad = S.SceneData(**{**sc.__dict__})
    bad.indices = sc.indices.copy()
    bad.indices[0, 0] = 10**6
    with pytest.raises(lib.SddError, match="index out of range"):
        lib.sdd_scene_create(bad)
    bad2 = S.SceneData(**{**sc.__dict__})
    bad2.mat_n = np.full_like(sc.mat_n, 0.5)
    with pytest.raises(lib.SddError, match="n must be >= 1"):
        lib.sdd_scene_create(bad2)
    with pytest.raises(lib.SddError, match="n_subdomains"):
        lib.sdd_scene_create(sc, n_subdomains=65)
    bad3 = S.SceneData(**{**sc.__dict__})
    bad3.table_nm = sc.table_nm[::-1].copy()
    with pytest.raises(lib.SddError, match="ascending"):
        lib.sdd_scene_create(bad3)


def declared_arity():
    """Parameter count of every function include/sdd.h declares."""
    text = open(os.path.join(ROOT, "include", "sdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(sdd_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    """Every ctypes declaration of the binding takes as many arguments as the C declaration."""
    L = lib.lib()
    arity = declared_arity()
    assert len(arity) >= 30
    checked = 0
    for name, n in arity.items():
        f = getattr(L, name)
        if f.argtypes is not None:
            assert len(f.argtypes) == n, (name, len(f.argtypes), n)
            checked += 1
    assert checked >= 25


def test_bad_slab_polarisation_is_rejected(lib):
    from paper_1912_05494_gb300 import scenes as S
    sc, _, _ = S.slab_scene(0)
    bad = S.SceneData(**{**sc.__dict__})
    bad.slab_polarisation = 2
    with pytest.raises(lib.SddError, match="slab_polarisation"):
        lib.sdd_scene_create(bad)


def test_photon_map_entry_points_reject_null_arguments(lib):
    L = lib.lib()
    out = C.c_void_p()
    assert L.sdd_photon_maps_build(None, None, C.byref(out), None) == -1
    assert L.sdd_photon_gather(None, 1, None, None, None, None, None, None) == -1
    a, b = C.c_int64(), C.c_int64()
    assert L.sdd_photon_maps_count(None, C.byref(a), C.byref(b)) == -1
    assert L.sdd_photon_maps_get(None, 0, None, None, None, None, None, None) == -1
    L.sdd_photon_maps_destroy(None)


def test_binding_structures_match_the_header_layout(lib, tmp_path):
    """The ctypes structures have the size and field offsets that a C compiler gives the
    header's structures (compiled here with gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sdd_render_opts": lib.sdd_render_opts, "sdd_photon_opts": lib.sdd_photon_opts,
               "sdd_scene_desc": lib.sdd_scene_desc, "sdd_camera": lib.sdd_camera, "sdd_tuning": lib.sdd_tuning,
               "sdd_stats": lib.sdd_stats, "sdd_tileset_desc": lib.sdd_tileset_desc,
               "sdd_train_opts": lib.sdd_train_opts, "sdd_scene_info": lib.sdd_scene_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sdd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'  printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])
