"""Where the GPU path computes in FP64, and what FP32 would cost there, measured against the
FP64 oracle.

* Near-grazing thin slab (cos theta < 1/16): the renderer evaluates the Fresnel terms and the
  slab series in FP64 and rounds the result to FP32.  Compared with the oracle it stays at
  float rounding (<= 2e-7 relative in T); the same expressions evaluated in FP32 (complex64
  Fresnel, FP32 series) lose up to ~7e-4 relative in T near cos theta = 1e-4, where 1 - R and
  1 - R^2 tau^2 cancel.
* Film: per (pixel, wavelength) the renderer sums the samples' FP32 path radiance in FP64 in
  sample order and divides once.  An FP32 running sum of the same path radiances at 16 spp
  differs from it by at most ~1e-6 relative; the FP64 sum matches the FP64 mean of the
  per-path values to float rounding of the final division.
"""
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


def slab_fp32(cos_i, n, k, d, lam):
    """The thin-slab series with every step in FP32 (complex64 Fresnel)."""
    f = np.float32
    c = cos_i.astype(f)
    n2 = (n.astype(f) + 1j * k.astype(f)).astype(np.complex64)
    sin2 = (f(1) - c * c).astype(f)
    eta = (f(1) / n2).astype(np.complex64)
    ct = np.sqrt((f(1) - eta * eta * sin2).astype(np.complex64))
    rs = (c - n2 * ct) / (c + n2 * ct)
    rp = (n2 * c - ct) / (n2 * c + ct)
    R = (f(0.5) * (np.abs(rs) ** 2 + np.abs(rp) ** 2)).astype(f)
    cos_t = np.sqrt(f(1) - sin2 / (n.astype(f) ** 2)).astype(f)
    tau = np.exp(-f(12.566370614359172) * k.astype(f) * d.astype(f) / (lam.astype(f) * f(1e-9) * cos_t)).astype(f)
    omr, rt = f(1) - R, R * tau
    den = (f(1) - rt) * (f(1) + rt)
    return R + omr * omr * R * tau * tau / den, omr * omr * tau / den


def test_near_grazing_slab_fp64_branch(sdd, orc):
    rng = np.random.default_rng(21)
    m = 4000
    cos_i = np.exp(rng.uniform(np.log(1e-4), np.log(0.0625), m)).astype(np.float32)
    nre = rng.uniform(1.45, 1.65, m).astype(np.float32)
    k = np.exp(rng.uniform(np.log(1e-8), np.log(1e-5), m)).astype(np.float32)
    d = rng.uniform(2e-3, 5e-3, m).astype(np.float32)
    lam = rng.uniform(380, 780, m).astype(np.float32)
    t = [torch.from_numpy(x).cuda() for x in (cos_i, nre, k, d, lam)]
    R, Rs, Ts = (torch.empty(m, device="cuda") for _ in range(3))
    sdd.sdd_eval_optics(*t, R, Rs, Ts)
    Rs_ref, Ts_ref = orc.slab(cos_i, nre, k, d, lam)
    gpu_T = np.abs(Ts.cpu().numpy() - Ts_ref) / Ts_ref
    gpu_R = np.abs(Rs.cpu().numpy() - Rs_ref) / Rs_ref
    R32, T32 = slab_fp32(cos_i, nre, k, d, lam)
    f32_T = np.abs(T32 - Ts_ref) / Ts_ref
    print(f"near grazing: GPU (FP64 branch) max rel err T {gpu_T.max():.2e}, R {gpu_R.max():.2e}; "
          f"FP32 evaluation max rel err T {f32_T.max():.2e} (mean {f32_T.mean():.2e})")
    assert gpu_T.max() <= 2e-7 and gpu_R.max() <= 2e-7
    assert f32_T.max() > 20 * gpu_T.max()  # what the FP64 branch buys


def test_film_fp64_sum_against_fp32_accumulation(sdd):
    sc, cam, spec = S.nave_scene(seed=1)
    cam = S.CameraData(**{**cam.__dict__, "width": 64, "height": 48})
    h = sdd.SceneHandle(sc)
    film, _, pr, _ = render_gpu(sdd, h, cam, spec, paths=True)  # 16 spp, 81 wavelengths
    p32 = pr.astype(np.float32)
    acc = np.zeros(p32[:, 0, :].shape, np.float32)
    for s in range(spec.spp):  # FP32 running sum in sample order
        acc = (acc + p32[:, s, :]).astype(np.float32)
    f32_mean = (acc / np.float32(spec.spp)).astype(np.float64)
    f64_mean = pr.sum(axis=1) / spec.spp
    nz = f64_mean > 0
    e32 = np.abs(f32_mean[nz] - f64_mean[nz]) / f64_mean[nz]
    e_film = np.abs(film[nz] - f64_mean[nz]) / f64_mean[nz]
    print(f"film at 16 spp: FP32 accumulation max rel err {e32.max():.2e} (mean {e32.mean():.2e}); "
          f"FP64 film max rel err {e_film.max():.2e}")
    assert e_film.max() <= 1.2e-7  # the final FP32 rounding of the FP64 mean
    assert e32.max() <= 4e-6
