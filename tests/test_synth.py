"""The seeded input generator: determinism, geometry of the point clouds, and
that the hologram is the FP64 sum of Eq. 3 rounded to complex64."""
import math

import numpy as np

import synth
from synth.configs import SMALL_512


def test_stream_is_deterministic_and_uniform():
    a = synth.uniform(123, 20000)
    assert np.array_equal(a, synth.uniform(123, 20000))
    assert not np.array_equal(a, synth.uniform(124, 20000))
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.01 and abs(a.var() - 1 / 12) < 0.005


def test_points_lie_in_the_view_pyramid():
    w = SMALL_512
    p = w.point_cloud()
    assert p.shape == (w.n_points, 5)
    z = p[:, 2]
    assert np.all((z >= w.z_range[0]) & (z <= w.z_range[1]))
    assert np.all(np.abs(p[:, 0]) <= z * w.tan_half + 1e-15)
    assert np.all(np.abs(p[:, 1]) <= z * w.tan_half + 1e-15)
    assert np.all(p[:, 3] == 1.0)
    assert np.all((p[:, 4] >= 0) & (p[:, 4] < 2 * math.pi))


def test_hologram_is_rounded_fp64_sum():
    lam, pitch, n = 532e-9, 0.4e-6, 64
    pts = synth.points(7, 5, (0.5e-3, 1e-3), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    H = synth.hologram(pts, lam, pitch, n, n)
    for ix, iy in [(0, 0), (31, 7), (63, 63), (10, 50)]:
        x, y = (ix - n / 2) * pitch, (iy - n / 2) * pitch
        ref = sum(a * np.exp(1j * (th - 2 * np.pi / lam * math.sqrt((x - px) ** 2 + (y - py) ** 2 + pz ** 2)))
                  for px, py, pz, a, th in pts)
        assert H[iy, ix] == np.complex64(ref)
        assert abs(synth.sample(pts, lam, pitch, n, n, ix, iy) - ref) < 1e-12
    rows = synth.hologram(pts, lam, pitch, n, n, row0=20, nrows=5)
    assert np.array_equal(rows, H[20:25])
