"""Failure paths on the GPU without a fault, trap or hang: every wait is bounded and every
store is checked against its capacity, so injected failures come back as status codes and
the context stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1912_05494_gb300 import scenes as S  # noqa: E402

SDD_ERR_QUEUE_OVERFLOW, SDD_ERR_TIMEOUT = -4, -5


@pytest.fixture(scope="module")
def sdd():
    import __graft_entry__ as g
    g.build()
    from paper_1912_05494_gb300 import sdd as m
    return m


def small_nave():
    sc, cam, spec = S.nave_scene(seed=1)
    cam = S.CameraData(**{**cam.__dict__, "width": 32, "height": 24})
    spec = S.RenderSpec(**{**spec.__dict__, "spp": 2})
    return sc, cam, spec


@pytest.mark.parametrize("batched", [0, 1])
def test_tiny_queue_capacity_reports_overflow_and_recovers(sdd, batched):
    sc, cam, spec = small_nave()
    h = sdd.SceneHandle(sc)
    out = torch.empty((cam.width * cam.height, spec.n_lambda), device="cuda")
    sdd.sdd_render(h.h, cam, spec, out, batched=batched)
    good = out.cpu().numpy().copy()
    tun = sdd.sdd_get_tuning(h.h)
    sdd.sdd_set_tuning(h.h, {**tun, "queue_capacity": 1000})  # far below the wave's 124,416 paths
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_render(h.h, cam, spec, out, batched=batched)
    assert e.value.status == SDD_ERR_QUEUE_OVERFLOW
    sdd.sdd_set_tuning(h.h, {**tun, "queue_capacity": 0})
    sdd.sdd_render(h.h, cam, spec, out, batched=batched)
    assert np.array_equal(out.cpu().numpy(), good)


def test_bad_queue_capacity_is_rejected(sdd):
    sc, cam, spec = small_nave()
    h = sdd.SceneHandle(sc)
    with pytest.raises(sdd.SddError, match="queue_capacity"):
        sdd.sdd_set_tuning(h.h, {**sdd.sdd_get_tuning(h.h), "queue_capacity": -1})


def test_watchdog_gives_up_and_the_context_stays_usable(sdd):
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_watchdog_selftest(200)
    assert e.value.status == SDD_ERR_TIMEOUT
    sc, cam, spec = small_nave()
    h = sdd.SceneHandle(sc)
    out = torch.empty((cam.width * cam.height, spec.n_lambda), device="cuda")
    sdd.sdd_render(h.h, cam, spec, out, batched=1)
    assert np.isfinite(out.cpu().numpy()).all()
