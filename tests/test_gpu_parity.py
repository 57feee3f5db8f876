"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance: relative L2 of the complex field <= 1e-5 (FP32 path); the
intensity PSNR is computed and reported alongside.  Cases span several FFT
tiles and ragged shapes: square and rectangular holograms, full and partial
views on and off the full view's pixel lattice, and both output kinds.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.configs import SMALL_512, SMALL_512_MM, WA_4096, WA_4096_MM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def psnr(i_gpu, i_ref):
    mse = float(np.mean((i_gpu.astype(np.float64) - i_ref) ** 2))
    return 10 * math.log10(float(i_ref.max()) ** 2 / mse) if mse > 0 else float("inf")


def gpu_run(nf, H, lam, pitch, view_kw):
    ny, nx = H.shape
    h = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    plan = nf.Plan(lam, pitch, nx, ny, h)
    vf = nf.View(kind=nf.OUT_FIELD, **view_kw)
    vi = nf.View(kind=nf.OUT_INTENSITY, **view_kw)
    f = plan.reconstruct(vf)
    i = plan.reconstruct(vi)
    torch.cuda.synchronize()
    out = f.cpu().numpy(), i.cpu().numpy()
    plan.close()
    return out


def oracle_run(H, lam, pitch, kw):
    return oracle.reconstruct(H, lam, pitch, kw["z"], kw.get("center_x", 0.0),
                              kw.get("center_y", 0.0), kw.get("width", 0.0), kw.get("height", 0.0),
                              kw.get("out_nx", 0), kw.get("out_ny", 0))


def check(nf, H, lam, pitch, kw, tol=TOL):
    f_gpu, i_gpu = gpu_run(nf, H, lam, pitch, kw)
    f_ref, i_ref = oracle_run(H, lam, pitch, kw)
    e = rel_l2(f_gpu, f_ref)
    p = psnr(i_gpu, i_ref)
    print("rel_l2=%.3e psnr=%.1f dB" % (e, p))
    assert f_gpu.shape == f_ref.shape
    assert e <= tol, e
    # intensity is |field|^2 of the same computation
    assert rel_l2(i_gpu, i_ref) <= 3 * tol
    return e, p


def random_holo(ny, nx, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex64)


def test_small_random_square(nf):
    check(nf, random_holo(64, 64, 1), 532e-9, 0.4e-6, dict(z=0.3e-3))


def test_small_random_rectangular(nf):
    check(nf, random_holo(96, 160, 2), 532e-9, 0.35e-6, dict(z=0.5e-3))


def test_pointcloud_512_full_view(nf):
    w = SMALL_512
    H = w.make_hologram()
    e, p = check(nf, H, w.wavelength, w.pitch, dict(z=w.z_view))
    assert p > 60


def test_partial_view_on_lattice(nf):
    lam, pitch, n, z = 532e-9, 0.4e-6, 256, 1e-3
    H = synth.hologram(synth.points(11, 6, (0.6e-3, 1.4e-3), synth.tan_half_fov(lam, pitch)),
                       lam, pitch, n, n)
    B = oracle.plan_view(lam, pitch, n, n, z)["width"]
    p = B / n
    kw = dict(z=z, center_x=(180 - n / 2) * p, center_y=(70 - n / 2) * p, width=48 * p,
              height=80 * p, out_nx=48, out_ny=80)
    assert nf.view_plan(lam, pitch, n, n, nf.View(**kw))["on_full_view_lattice"] == 1
    check(nf, H, lam, pitch, kw)


def test_partial_view_off_lattice(nf):
    lam, pitch, n, z = 532e-9, 0.4e-6, 256, 1e-3
    H = random_holo(n, n, 3)
    kw = dict(z=z, center_x=1.234e-4, center_y=-0.71e-4, width=2.1e-4, height=1.3e-4, out_nx=70,
              out_ny=44)
    assert nf.view_plan(lam, pitch, n, n, nf.View(**kw))["on_full_view_lattice"] == 0
    check(nf, H, lam, pitch, kw)


def test_ultra_wide_angle_small(nf):
    # 120 deg FoV geometry (pitch 0.307 um at 532 nm): evanescent spectrum corners
    lam, pitch, n = 532e-9, 0.307e-6, 128
    H = random_holo(n, n, 4)
    check(nf, H, lam, pitch, dict(z=0.2e-3))


def test_zero_hologram_gives_zero(nf):
    H = np.zeros((64, 64), np.complex64)
    f, i = gpu_run(nf, H, 532e-9, 0.4e-6, dict(z=0.3e-3))
    assert np.all(f == 0) and np.all(i == 0)


def test_point_source_refocus_and_peak(nf):
    lam, pitch, n, z = 532e-9, 0.4e-6, 256, 1e-3
    B = oracle.plan_view(lam, pitch, n, n, z)["width"]
    p = B / n
    for ix, iy in [(128, 128), (230, 40)]:
        H = synth.hologram(np.array([[(ix - n / 2) * p, (iy - n / 2) * p, z, 1.0, 0.0]]), lam,
                           pitch, n, n)
        _, I = gpu_run(nf, H, lam, pitch, dict(z=z))
        j, i = np.unravel_index(np.argmax(I), I.shape)
        assert (i, j) == (ix, iy)
        if ix == 128:
            assert abs(I.max() / n ** 4 - 1) < 5e-3


@pytest.mark.slow
def test_pointcloud_4096_full_view(nf):
    """The wide-angle FP32 workload at full size at the paper's depths (4096^2,
    2000 points at 0.5-1.5 m, full view at 0.85 m)."""
    w = WA_4096
    H = w.make_hologram()
    check(nf, H, w.wavelength, w.pitch, dict(z=w.z_view))


def test_pointcloud_512_mm_full_view(nf):
    """512^2 at 0.4 um, 8 unit-amplitude points at z in [0.5, 2] mm, full view
    at z = 1 mm (N' = 640), field within 1e-5 of the oracle."""
    w = SMALL_512_MM
    H = w.make_hologram()
    e, p = check(nf, H, w.wavelength, w.pitch, dict(z=w.z_view))
    assert p > 60


@pytest.mark.slow
def test_pointcloud_4096_mm_full_view(nf):
    """The wide-angle FP32 workload at its stated depths: 4096^2 at 0.5 um,
    2000 points at z in [1, 5] mm, full view at z = 3 mm (N' = 4608), field
    within 1e-5 of the oracle."""
    w = WA_4096_MM
    H = w.make_hologram()
    check(nf, H, w.wavelength, w.pitch, dict(z=w.z_view))
