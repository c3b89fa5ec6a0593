"""sdd_trace_closest_noalloc against sdd_trace_closest.

The allocation-free variant serves callers whose device memory is fixed when they start and
who cannot let the library allocate during a call; it runs the same traversal passes out of
a static 16 MiB array instead of the scene's workspace.  Its results must equal those of the
allocating entry point, on consecutive calls (the shared array keeps the previous call's
contents, so the second call checks that nothing stale leaks through), and it must refuse a
batch that does not fit.  This file is named so that pytest collects it last.
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


def trace_both(sdd, h, o, d):
    do, dd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    n = o.shape[0]
    t_a = torch.full((n,), -1.0, device="cuda")
    p_a = torch.full((n,), -2, device="cuda", dtype=torch.int32)
    t_b = torch.full((n,), -1.0, device="cuda")
    p_b = torch.full((n,), -2, device="cuda", dtype=torch.int32)
    sdd.sdd_trace_closest(h.h, do, dd, t_a, p_a)
    sdd.sdd_trace_closest_noalloc(h.h, do, dd, t_b, p_b)
    torch.cuda.synchronize()
    return t_a.cpu().numpy(), p_a.cpu().numpy(), t_b.cpu().numpy(), p_b.cpu().numpy()


def nave_rays(seed, n):
    rng = np.random.default_rng(seed)
    o = np.column_stack([rng.uniform(0.5, 59.5, n), rng.uniform(0.5, 11.5, n), rng.uniform(0.2, 13.5, n)])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def test_noalloc_setup_call_without_rays(sdd):
    """A call with n = 0 only places the static scratch on the current device (what a caller
    that budgets its memory at start-up does once); it succeeds and touches no output."""
    sc = S.tiny_scene(7, n_triangles=64)
    h = sdd.SceneHandle(sc)
    e = torch.empty((0, 3), device="cuda")
    t = torch.empty((0,), device="cuda")
    p = torch.empty((0,), device="cuda", dtype=torch.int32)
    sdd.sdd_trace_closest_noalloc(h.h, e, e, t, p)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n_sub", [1, 5])
def test_noalloc_matches_allocating_entry_point_tiny(sdd, n_sub):
    sc = S.tiny_scene(7, n_triangles=64)
    h = sdd.SceneHandle(sc, n_subdomains=n_sub, split_axis=0)
    for call, seed in enumerate((21, 22)):  # two calls in a row, different rays
        o, d = S.random_rays(seed, 5000 + 777 * call)
        t_a, p_a, t_b, p_b = trace_both(sdd, h, o, d)
        assert np.array_equal(p_a, p_b)
        assert np.allclose(t_a, t_b, rtol=1e-6, atol=0) or np.array_equal(t_a, t_b)
        assert (p_a >= 0).mean() > 0.3


def test_noalloc_matches_on_the_nave_near_capacity(sdd):
    sc, _, _ = S.nave_scene(seed=1)
    h = sdd.SceneHandle(sc, n_subdomains=8)
    for call, (seed, n) in enumerate(((31, 140000), (32, 90001))):
        o, d = nave_rays(seed, n)
        t_a, p_a, t_b, p_b = trace_both(sdd, h, o, d)
        assert np.array_equal(p_a, p_b), call
        finite = np.isfinite(t_a)
        assert np.array_equal(finite, np.isfinite(t_b))
        assert np.allclose(t_a[finite], t_b[finite], rtol=1e-6, atol=0)
        assert finite.mean() > 0.99  # the nave is closed: almost every ray hits something


def test_noalloc_rejects_batches_beyond_its_static_scratch(sdd):
    sc, _, _ = S.nave_scene(seed=1)
    h = sdd.SceneHandle(sc, n_subdomains=8)
    o, d = nave_rays(33, 200000)
    do, dd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    t = torch.empty(o.shape[0], device="cuda")
    p = torch.empty(o.shape[0], device="cuda", dtype=torch.int32)
    with pytest.raises(sdd.SddError, match="static limit"):
        sdd.sdd_trace_closest_noalloc(h.h, do, dd, t, p)
