"""Out-of-core subdomains (sdd_tuning.resident_subdomains): Sec. 5 loads sub-domains according
to the memory available and unloads them when few rays remain.  With at most C of the S
subdomain BVHs in device memory, the host-driven passes make the C subdomains with the most
queued rays resident before each pass and leave the other queues waiting; the traversal code
and the BVH are the same, so images, per-path radiance and path hashes must equal the
all-resident render's bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1912_05494_gb300 import scenes as S  # noqa: E402
from test_gpu_parity import render_gpu  # noqa: E402


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd as m
    assert torch.cuda.is_available()
    return m


def set_resident(sdd, h, c):
    sdd.sdd_set_tuning(h.h, {**sdd.sdd_get_tuning(h.h), "resident_subdomains": c})


@pytest.mark.parametrize("bundle", [1, 14])
def test_streamed_render_is_bit_identical(sdd, bundle):
    sc, cam, spec = S.nave_scene(seed=1)  # 8 subdomains along the nave
    cam = S.CameraData(**{**cam.__dict__, "width": 64, "height": 48})
    spec = S.RenderSpec(**{**spec.__dict__, "spp": 2, "bundle": bundle})
    h = sdd.SceneHandle(sc)
    ref, rx, rp, rh = render_gpu(sdd, h, cam, spec, paths=True, batched=0)
    for cap in (4, 2, 1):
        set_resident(sdd, h, cap)
        assert sdd.sdd_get_tuning(h.h)["resident_subdomains"] == cap
        img, x, pr, ph = render_gpu(sdd, h, cam, spec, paths=True, batched=0)
        st = sdd.sdd_get_stats(h.h)
        assert np.array_equal(img, ref) and np.array_equal(x, rx), cap
        assert np.array_equal(pr, rp) and np.array_equal(ph, rh), cap
        assert st["subdomain_loads"] >= 8 and st["bytes_streamed"] > 0, (cap, st["subdomain_loads"])
    set_resident(sdd, h, 0)
    img, _ = render_gpu(sdd, h, cam, spec, batched=2)  # all resident again: every form works
    b, _ = render_gpu(sdd, h, cam, spec, batched=0)
    assert np.array_equal(b, ref)


def test_streamed_closest_hit_queries(sdd):
    sc, _, _ = S.nave_scene(seed=1)
    h = sdd.SceneHandle(sc)
    rng = np.random.default_rng(3)
    n = 50000
    o = np.column_stack([rng.uniform(0.5, 59.5, n), rng.uniform(0.5, 11.5, n), rng.uniform(0.2, 13.5, n)])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    do, dd = torch.from_numpy(o.astype(np.float32)).cuda(), torch.from_numpy(d.astype(np.float32)).cuda()
    out = []
    for cap in (0, 3):
        set_resident(sdd, h, cap)
        t = torch.empty(n, device="cuda")
        p = torch.empty(n, device="cuda", dtype=torch.int32)
        sdd.sdd_trace_closest(h.h, do, dd, t, p)
        torch.cuda.synchronize()
        out.append((t.cpu().numpy(), p.cpu().numpy()))
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][0], out[1][0])


def test_other_forms_refuse_while_streaming(sdd):
    sc, cam, spec = S.nave_scene(seed=1)
    cam = S.CameraData(**{**cam.__dict__, "width": 16, "height": 8})
    spec = S.RenderSpec(**{**spec.__dict__, "spp": 1})
    h = sdd.SceneHandle(sc)
    set_resident(sdd, h, 2)
    out = torch.empty((16 * 8, spec.n_lambda), device="cuda")
    for form in (1, 2):
        with pytest.raises(sdd.SddError, match="host-driven"):
            sdd.sdd_render(h.h, cam, spec, out, None, batched=form)
    e = torch.empty((4, 3), device="cuda")
    t = torch.empty(4, device="cuda")
    p = torch.empty(4, device="cuda", dtype=torch.int32)
    with pytest.raises(sdd.SddError, match="resident"):
        sdd.sdd_trace_closest_noalloc(h.h, e, e, t, p)
    set_resident(sdd, h, 0)
    sdd.sdd_render(h.h, cam, spec, out, None, batched=2)
    torch.cuda.synchronize()
