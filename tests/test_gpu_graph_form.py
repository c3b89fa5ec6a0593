"""The graph form (sdd_render_opts.batched = 2) on the GPU, through the C ABI.

Its kernels read their queue counts on the device; per generation the closest-hit and shadow
passes run in conditional 'while' nodes of a CUDA graph captured once per frame shape (a
fixed n_sub + 1 passes when the graph is off); the per-ray device code is the host-driven form's, so images,
per-path radiance and event hashes must equal the host-driven form's bit for bit (brute-force
tiles excepted: their tracer is inlined into differently register-bounded kernels, and the
compiler may contract its arithmetic differently, so there at most 0.1 % of branch
decisions may flip).
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
    assert torch.cuda.is_available()
    return m


def render(sdd, h, cam, spec, **kw):
    n = cam.width * cam.height
    out = torch.empty((n, spec.n_lambda), device="cuda")
    xyz = torch.empty((n, 3), device="cuda")
    pr = torch.empty((n, spec.spp, spec.n_lambda), device="cuda")
    ph = torch.empty((n, spec.spp, spec.n_lambda), device="cuda", dtype=torch.int32)
    sdd.sdd_render(h.h, cam, spec, out, xyz, path_radiance_out=pr, path_hash_out=ph, **kw)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), xyz.cpu().numpy(), pr.cpu().numpy(), ph.cpu().numpy().view(np.uint32))


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("bundle,n_sub", [(1, 8), (14, 8), (9, 3), (1, 1), (41, 8), (64, 5)])
def test_graph_form_equals_host_driven_on_the_nave(sdd, bundle, n_sub):
    sc, cam, spec = S.nave_scene(seed=1)
    cam = S.CameraData(**{**cam.__dict__, "width": 64, "height": 40})
    spec = S.RenderSpec(**{**spec.__dict__, "spp": 3, "bundle": bundle})
    h = sdd.SceneHandle(sc, n_subdomains=n_sub)
    a = render(sdd, h, cam, spec)
    b = render(sdd, h, cam, spec, batched=2)
    c = render(sdd, h, cam, spec, batched=2)  # replayed graph
    assert same(a, b) and same(b, c)
    st = sdd.sdd_get_stats(h.h)
    assert st["graph_replays"] >= 1
    # each generation's passes run in a conditional loop of two passes per iteration, until
    # the queues drain (a ray crosses each of the n_sub slabs at most once)
    loops = st["waves"] * (spec.max_depth + 2)
    for k in ("launches_traverse", "launches_shadow"):
        assert st[k] % 2 == 0 and 2 * loops <= st[k] <= (n_sub // 2 + 2) * 2 * loops, (k, st[k], loops)
    # without a graph the same sequence runs with n_sub + 1 passes per generation
    tun = sdd.sdd_get_tuning(h.h)
    sdd.sdd_set_tuning(h.h, {**tun, "no_graph": 1})
    d = render(sdd, h, cam, spec, batched=2)
    sdd.sdd_set_tuning(h.h, tun)
    assert same(a, d)
    assert sdd.sdd_get_stats(h.h)["launches_traverse"] == loops * (n_sub + 1)


def test_graph_form_with_several_waves_and_profiling(sdd):
    """Several waves per frame and per-launch timing: the timing events are nodes of the
    graph and are read back after every replay."""
    sc, cam, spec = S.nave_scene(seed=1)
    cam = S.CameraData(**{**cam.__dict__, "width": 48, "height": 32})
    spec = S.RenderSpec(**{**spec.__dict__, "spp": 4, "bundle": 14})
    h = sdd.SceneHandle(sc)
    a = render(sdd, h, cam, spec, wave_paths=3000)
    sdd.sdd_set_profiling(h.h, 1)
    for _ in range(2):
        b = render(sdd, h, cam, spec, batched=2, wave_paths=3000)
        st = sdd.sdd_get_stats(h.h)
        assert st["waves"] > 1
        assert st["ms_traverse"] > 0 and st["ms_shade"] > 0 and st["ms_shadow"] > 0
        assert same(a, b)
    sdd.sdd_set_profiling(h.h, 0)


@pytest.mark.parametrize("bundle", [1, 8, 41])
def test_graph_form_with_network_tiles(sdd, bundle):
    """Heterogeneous tiles shaded by the network (weights as initialised: the comparison is
    of the two forms, not of the network's quality)."""
    sc, cam, spec = S.tile_room_scene(width=40, height=24, spp=4)
    spec = S.RenderSpec(**{**spec.__dict__, "bundle": bundle})
    B, params = S.surrogate_init(4)
    net = sdd.Surrogate(B, params, max_batch=4096)
    h = sdd.SceneHandle(sc)
    kw = {"use_surrogate": 1, "surrogate": net}
    a = render(sdd, h, cam, spec, **kw)
    b = render(sdd, h, cam, spec, batched=2, **kw)
    assert same(a, b)
    assert sdd.sdd_get_stats(h.h)["launches_tile"] > 0


def test_graph_form_with_brute_force_tiles(sdd):
    sc, cam, spec = S.tile_room_scene(width=40, height=24, spp=4)
    h = sdd.SceneHandle(sc)
    a = render(sdd, h, cam, spec)
    b = render(sdd, h, cam, spec, batched=2)
    assert float(np.mean(a[3] != b[3])) <= 1e-3
    assert float(np.abs(a[0] - b[0]).sum() / np.abs(a[0]).sum()) <= 1e-3


def test_graph_form_splits_waves_when_bundles_outgrow_the_queues(sdd):
    sc, cam, spec = S.slab_scene(0)
    cam = S.CameraData(**{**cam.__dict__, "width": 24, "height": 24})
    spec = S.RenderSpec(**{**spec.__dict__, "mode": S.RENDER_MC, "spp": 16, "bundle": 16, "rr_start_depth": 3,
                           "max_depth": 8})
    h = sdd.SceneHandle(sc)
    a = render(sdd, h, cam, spec)
    b = render(sdd, h, cam, spec, batched=2)
    assert sdd.sdd_get_stats(h.h)["wave_splits"] > 0
    assert same(a, b)


def test_graph_form_argument_check(sdd):
    sc, cam, spec = S.slab_scene(0)
    h = sdd.SceneHandle(sc)
    out = torch.empty((cam.width * cam.height, spec.n_lambda), device="cuda")
    with pytest.raises(sdd.SddError, match="batched"):
        sdd.sdd_render(h.h, cam, spec, out, batched=3)
