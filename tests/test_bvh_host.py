"""The subdomain split and the per-subdomain 4-wide BVHs (Sec. 5: the geometry is split once,
every sub-domain keeps its own hierarchy), built on the host by sdd_bvh_build_host exactly as
sdd_scene_create builds them, checked against their definition with numpy (no GPU):

* every triangle whose box overlaps a slab (widened by the slop) is referenced exactly once in
  that slab's tree, and by no other slab's tree it does not overlap;
* a leaf child's box contains its triangles' boxes clipped to the widened slab, an inner
  child's box contains its node's child boxes, and the records hold the scene's vertices;
* each subdomain's nodes form one block, every node reached once from the root, inner children
  after their parent (breadth-first), children packed first in a node, at most four, and four
  wherever the node has an inner child (the collapse opens inner children until four);
* the deepest traversal stack (k - 1 pushes at a node with k inner children) recomputed here
  equals the reported bound, which stays within the kernels' 64 entries.
"""
import numpy as np
import pytest

from paper_1912_05494_gb300 import scenes as S

ERR_ARG = -1  # SDD_ERR_ARG of include/sdd.h


@pytest.fixture(scope="module")
def sdd():
    from paper_1912_05494_gb300 import sdd as m
    m.lib()
    return m


def tri_boxes(sc):
    v = sc.vertices.astype(np.float32)[sc.indices.astype(np.int64)]  # [n][3 corners][3]
    return v.min(axis=1), v.max(axis=1), v


def check(sdd, sc, n_sub, max_leaf=4):
    r = sdd.sdd_bvh_build_host(sc, n_subdomains=n_sub)
    nodes, tris, root, nn, planes = r["nodes"], r["tris"], r["root"], r["n_nodes_sub"], r["planes"]
    axis, slop = r["split_axis"], np.float32(r["slop"])
    assert r["n_subdomains"] == n_sub and planes[0] == -np.inf and planes[-1] == np.inf
    assert np.all(np.diff(planes) > 0)
    blo, bhi, verts = tri_boxes(sc)
    assert np.array_equal(np.sort(root), root) and root[0] == 0 and int(nn.sum()) == nodes.size
    assert np.array_equal(root[1:], np.cumsum(nn)[:-1])
    boxes = ("lo_x", "hi_x", "lo_y", "hi_y", "lo_z", "hi_z")
    stack_need = 0
    fan = []
    for s in range(n_sub):
        lo_s = np.float32(planes[s]) - slop
        hi_s = np.float32(planes[s + 1]) + slop
        want = ~((bhi[:, axis] < lo_s) | (blo[:, axis] > hi_s))
        # the references' boxes: clipped to the widened slab along the split axis
        clo, chi = blo.copy(), bhi.copy()
        clo[:, axis] = np.maximum(clo[:, axis], lo_s)
        chi[:, axis] = np.minimum(chi[:, axis], hi_s)
        seen = np.zeros(nn[s], np.int64)
        refs = []
        need = {}

        def walk(i):
            seen[i - root[s]] += 1
            n = nodes[i]
            k = int(np.sum(n["link"] >= 0))
            assert np.all(n["link"][:k] >= 0) and np.all(n["link"][k:] < 0) and np.all(n["count"][k:] == 0)
            assert 1 <= k <= 4 or nn[s] == 1
            # the collapse opens inner children until a node holds four: a node with fewer
            # children has leaves only
            assert k == 4 or np.all(n["count"][:k] > 0) or nn[s] == 1
            fan.append(k)
            below, k_in = 0, 0
            for c in range(k):
                lo = np.array([n["lo_x"][c], n["lo_y"][c], n["lo_z"][c]], np.float32)
                hi = np.array([n["hi_x"][c], n["hi_y"][c], n["hi_z"][c]], np.float32)
                link, cnt = int(n["link"][c]), int(n["count"][c])
                if cnt > 0:
                    assert cnt <= max_leaf
                    rec = tris[link:link + cnt]
                    p = rec["prim"].astype(np.int64)
                    refs.extend(p.tolist())
                    assert np.array_equal(rec["v0"], verts[p, 0]) and np.array_equal(rec["v1"], verts[p, 1])
                    assert np.array_equal(rec["v2"], verts[p, 2])
                    assert np.all(clo[p] >= lo) and np.all(chi[p] <= hi)
                else:
                    assert root[s] <= link < root[s] + nn[s] and link > i  # breadth-first, own block
                    m = nodes[link]
                    km = int(np.sum(m["link"] >= 0))
                    for f in range(0, 6, 2):
                        assert np.all(m[boxes[f]][:km] >= lo[f // 2]) and np.all(m[boxes[f + 1]][:km] <= hi[f // 2])
                    k_in += 1
                    below = max(below, walk(link))
            need[i] = k_in - 1 + below if k_in > 0 else 0
            return need[i]

        stack_need = max(stack_need, walk(int(root[s])))
        assert np.all(seen == 1), "every node of the block reached once"
        refs = np.array(refs, np.int64)
        assert np.unique(refs).size == refs.size, "a triangle referenced twice in one slab"
        assert np.array_equal(np.sort(refs), np.flatnonzero(want))
    assert stack_need == r["stack_need"] <= 64
    return r, np.array(fan)


def test_nave_split_and_trees(sdd):
    sc, _, _ = S.nave_scene(seed=1)
    r, fan = check(sdd, sc, 8)
    # four children wherever an inner child was left to open (the nodes above the bottom);
    # a binary tree would have two everywhere
    assert fan.mean() > 3.0, fan.mean()
    assert r["bvh_max_depth"] < 60


@pytest.mark.parametrize("n_sub", [1, 3, 64])
def test_random_triangles(sdd, n_sub):
    sc = S.tiny_scene(3, n_triangles=500)
    check(sdd, sc, n_sub)


def test_coincident_triangles_and_empty_slabs(sdd):
    """Thirty copies of one triangle at one end of the scene (their centroids coincide, so no
    SAH split separates them and the builder splits them by count into small leaves) and a
    single triangle at the other, in five slabs: the middle slabs hold no geometry and get a
    root without children."""
    sc = S.tiny_scene(3, n_triangles=2)
    v = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [10, 0, 0], [10.1, 0, 0], [10, 0.1, 0]], np.float32)
    idx = np.array([[0, 1, 2]] * 30 + [[3, 4, 5]], np.uint32)
    sc = S.SceneData(**{**sc.__dict__, "vertices": v, "indices": idx,
                        "tri_material": np.zeros(idx.shape[0], np.uint16)})
    r, fan = check(sdd, sc, 5)
    nodes, root, nn = r["nodes"], r["root"], r["n_nodes_sub"]
    for s in (1, 2, 3):
        assert nn[s] == 1 and np.all(nodes[root[s]]["link"] < 0)
    assert nn[0] > 1  # thirty references do not fit one node's leaves
    last = nodes[root[4]]  # one triangle: a root over one leaf
    assert int(last["count"][0]) == 1 and np.all(last["link"][1:] < 0)


def test_invalid_geometry_is_refused(sdd):
    sc = S.tiny_scene(3, n_triangles=8)
    with pytest.raises(sdd.SddError):
        sdd.sdd_bvh_build_host(sc, n_subdomains=0)
    bad = S.SceneData(**{**sc.__dict__, "indices": np.full_like(sc.indices, 10 ** 6)})
    with pytest.raises(sdd.SddError):
        sdd.sdd_bvh_build_host(bad, n_subdomains=2)


def test_too_small_buffers_are_refused(sdd):
    """Buffers below the sizes the first call reports are refused with SDD_ERR_ARG."""
    import ctypes as C
    sc = S.tiny_scene(3, n_triangles=40)
    d, keep = sdd._scene_desc(sc, n_subdomains=2)
    info = sdd.sdd_bvh_info()
    L = sdd.lib()
    assert L.sdd_bvh_build_host(C.byref(d), C.byref(info), None, 0, None, 0, None, None, None) == 0
    nodes = np.zeros(info.n_nodes, sdd.BVH_NODE)
    tris = np.zeros(info.n_tri_records, sdd.BVH_TRI)
    short = L.sdd_bvh_build_host(C.byref(d), C.byref(info), nodes.ctypes.data, nodes.size - 1, None, 0, None, None,
                                 None)
    assert short == ERR_ARG and b"nodes buffer too small" in L.sdd_last_error()
    short = L.sdd_bvh_build_host(C.byref(d), C.byref(info), None, 0, tris.ctypes.data, tris.size - 1, None, None,
                                 None)
    assert short == ERR_ARG and b"tris buffer too small" in L.sdd_last_error()
    assert L.sdd_bvh_build_host(C.byref(d), None, None, 0, None, 0, None, None, None) == ERR_ARG
