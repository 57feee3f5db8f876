"""The 16384^2 ultra-wide-angle geometry (120 deg FoV, view at 0.8 m) at full
size on the GPU.

* Full view in the benchmark's launch configuration (plan.load of a new
  hologram, then the full 16384^2 intensity view, FP32 path): point sources
  placed on full-view pixels at the view distance refocus on exactly those
  pixels, and the on-axis one reaches |sum of N^2 unit phasors|^2 = N^4 --
  properties that hold at any size (the oracle meets them at 1024^2 and
  2048^2 with I/N^4 = 0.9999 at these depths).
* A 1024^2 partial view of a 16K hologram against the FP64 oracle at 1025
  sampled pixels, stored by tests/golden/make_uwa16k_crop.py (which runs the
  oracle once on the host: its 16K gridding FFT takes minutes).
* The 16 seeded 2048^2 partial views of the 16K workload at its stated depths
  (20000 points at 2-10 mm, views at 6 mm, N' = 8192 each) against the FP64
  oracle at 257 sampled pixels per view, stored by
  tests/golden/make_uwa16k_mm_views.py.
"""
import importlib.util
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-5


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


def _crop_module():
    spec = importlib.util.spec_from_file_location(
        "make_uwa16k_crop", os.path.join(HERE, "golden", "make_uwa16k_crop.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_uwa16k_full_view_point_refocus(nf):
    import synth
    from synth.configs import UWA_16K as w
    n = w.n
    lam, pitch, z = w.wavelength, w.pitch, w.z_view
    plan = nf.Plan(lam, pitch, n, n)
    view = nf.View(z=z)
    p = plan.view_plan(view)["width_m"] / n
    targets = [(8192, 8192), (12000, 3000), (2500, 13500), (14000, 11500)]
    pts = np.array([[(i - n / 2) * p, (j - n / 2) * p, z, 1.0, 0.0] for i, j in targets])
    H = synth.hologram(pts, lam, pitch, n, n)
    d_h = torch.from_numpy(H).cuda()
    del H
    out = plan.output_like(view)
    plan.load(d_h)
    plan.reconstruct(view, out)
    torch.cuda.synchronize()
    del d_h
    R = 16
    for i, j in targets:
        win = out[j - R:j + R + 1, i - R:i + R + 1].cpu().numpy()
        jj, ii = np.unravel_index(int(np.argmax(win)), win.shape)
        print("point (%d, %d): local peak at (%+d, %+d), I/N^4 = %.5f"
              % (i, j, ii - R, jj - R, float(win.max()) / float(n) ** 4))
        assert (ii, jj) == (R, R), (i, j)
    peak = float(out[8192, 8192]) / float(n) ** 4
    assert abs(peak - 1) < 1e-2, peak
    plan.close()


def test_uwa16k_partial_view_vs_oracle_samples(nf):
    import synth
    g = _crop_module()
    rows = np.loadtxt(os.path.join(HERE, "golden", "uwa16k_crop_samples.txt"))
    view_kw, pts = g.geometry()
    H = synth.hologram(pts, g.LAM, g.PITCH, g.N, g.N)
    d_h = torch.from_numpy(H).cuda()
    del H
    plan = nf.Plan(g.LAM, g.PITCH, g.N, g.N, d_h)
    f = plan.reconstruct(nf.View(kind=nf.OUT_FIELD, **view_kw))
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    plan.close()
    j = rows[:, 0].astype(np.int64)
    i = rows[:, 1].astype(np.int64)
    ref = rows[:, 2] + 1j * rows[:, 3]
    got = f[j, i].astype(np.complex128)
    e = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print("sampled rel_l2 = %.3e over %d pixels" % (e, len(ref)))
    assert e <= TOL, e
    # the oracle's brightest pixel (last row) is the GPU's brightest too
    assert np.unravel_index(int(np.argmax(np.abs(f))), f.shape) == (j[-1], i[-1])


def _mm_views_module():
    spec = importlib.util.spec_from_file_location(
        "make_uwa16k_mm_views", os.path.join(HERE, "golden", "make_uwa16k_mm_views.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def read_mm_view_samples():
    """(hologram sha256, {view: (j, i, oracle field)}) from the stored samples."""
    path = os.path.join(HERE, "golden", "uwa16k_mm_views_samples.txt")
    dig = None
    with open(path) as f:
        for line in f:
            if line.startswith("# hologram sha256"):
                dig = line.split()[-1]
    rows = np.loadtxt(path)
    out = {}
    for v in np.unique(rows[:, 0]).astype(int):
        r = rows[rows[:, 0] == v]
        out[v] = (r[:, 1].astype(np.int64), r[:, 2].astype(np.int64), r[:, 3] + 1j * r[:, 4])
    return dig, out


def test_uwa16k_mm_partial_views_vs_oracle_samples(nf):
    """The benchmark's 16 partial views (FP32 path, one plan, the views one
    after another on the loaded hologram) match the oracle within 1e-5 on
    each view's samples, and each view's brightest oracle pixel is the GPU's."""
    import synth
    g = _mm_views_module()
    W = g.W
    dig, samples = read_mm_view_samples()
    d_h = synth.gpu_hologram(W.point_cloud(), W.wavelength, W.pitch, W.n, W.n)
    assert g.digest(d_h.cpu().numpy()) == dig, "the input generator made a different hologram"
    plan = nf.Plan(W.wavelength, W.pitch, W.n, W.n, d_h)
    del d_h
    worst = 0.0
    for v, kw in enumerate(g.views()):
        view = nf.View(z=kw["z"], center_x=kw["cx"], center_y=kw["cy"], width=kw["w"],
                       height=kw["h"], out_nx=kw["ox"], out_ny=kw["oy"], kind=nf.OUT_FIELD)
        f = plan.reconstruct(view)
        torch.cuda.synchronize()
        f = f.cpu().numpy()
        j, i, ref = samples[v]
        got = f[j, i].astype(np.complex128)
        e = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        worst = max(worst, e)
        print("view %2d: sampled rel_l2 = %.3e" % (v, e))
        assert e <= TOL, (v, e)
        assert np.unravel_index(int(np.argmax(np.abs(f))), f.shape) == (j[-1], i[-1])
    plan.close()
    print("worst view: %.3e" % worst)
