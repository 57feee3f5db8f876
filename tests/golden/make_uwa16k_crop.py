#!/usr/bin/env python
"""Writes uwa16k_crop_samples.txt: oracle values of a 1024^2 partial view of a
16384^2 ultra-wide-angle hologram, at seeded sample pixels.

The FP64 oracle needs about 25 GB of host memory and a few minutes for a 16K
hologram (its gridding FFT is 32768^2), too long to run inside the GPU test;
this script runs it once and stores the samples.  It calls only ``oracle``
and the input generator ``synth``.

  python tests/golden/make_uwa16k_crop.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "uwa16k_crop_samples.txt")

# geometry of the 16K ultra-wide-angle workload (120 deg FoV, view at 0.8 m)
LAM, PITCH, N, Z = 532e-9, 0.307e-6, 16384, 0.8
# the view: 1024^2 pixels on the full view's lattice, centred at full-view pixel (CI, CJ)
CI, CJ, OUT_N = 11000, 6000, 1024
N_SAMPLES = 1024
SEED = 20241031


def geometry():
    """The crop's view arguments and the hologram's point cloud."""
    full = oracle.plan_view(LAM, PITCH, N, N, Z)
    p = full["width"] / N
    view = dict(z=Z, center_x=(CI - N / 2) * p, center_y=(CJ - N / 2) * p, width=OUT_N * p,
                height=OUT_N * p, out_nx=OUT_N, out_ny=OUT_N)
    # object points: three in focus on crop pixels, two defocused nearby, one far outside
    def px(i):
        return (i - N / 2) * p

    pts = np.array([
        [px(CI), px(CJ), Z, 1.0, 0.0],
        [px(CI + 300), px(CJ - 200), Z, 0.8, 1.3],
        [px(CI - 410), px(CJ + 377), Z, 0.6, -2.1],
        [px(CI + 120), px(CJ + 260), 0.9 * Z, 0.7, 0.4],
        [px(CI - 200), px(CJ - 350), 1.15 * Z, 0.9, 2.7],
        [px(3000), px(12000), Z, 1.0, 0.5],
    ])
    return view, pts


def sample_pixels():
    rng = np.random.default_rng(SEED)
    return rng.integers(0, OUT_N, N_SAMPLES), rng.integers(0, OUT_N, N_SAMPLES)


def main():
    view, pts = geometry()
    t = time.time()
    H = synth.hologram(pts, LAM, PITCH, N, N)
    t_h = time.time() - t
    t = time.time()
    f, _ = oracle.reconstruct(H, LAM, PITCH, view["z"], view["center_x"], view["center_y"],
                              view["width"], view["height"], view["out_nx"], view["out_ny"])
    t_o = time.time() - t
    del H
    j, i = sample_pixels()
    jm, im = np.unravel_index(int(np.argmax(np.abs(f))), f.shape)  # the brightest pixel
    j = np.append(j, jm)
    i = np.append(i, im)
    with open(OUT, "w") as fo:
        fo.write("# Oracle (FP64) field of a 1024^2 partial view of a 16384^2 hologram, written by\n")
        fo.write("# tests/golden/make_uwa16k_crop.py (Section 4, Fig. 3 steps two to five; Eq. 17).\n")
        fo.write("# lambda %.6g m, pitch %.6g m, N %d, z %.6g m, view centre pixel (%d, %d) of the\n"
                 % (LAM, PITCH, N, Z, CI, CJ))
        fo.write("# full view; %d seeded pixels, then the brightest; oracle threads %d, %.0f s.\n"
                 % (N_SAMPLES, oracle.num_threads(), t_o))
        fo.write("# columns: row j, column i, Re, Im\n")
        for a, b in zip(j, i):
            v = f[a, b]
            fo.write("%d %d %.17g %.17g\n" % (a, b, v.real, v.imag))
    print("hologram %.1f s, oracle %.1f s, brightest (%d, %d) |O|/N^2 %.5f -> %s"
          % (t_h, t_o, jm, im, abs(f[jm, im]) / N ** 2, OUT))


if __name__ == "__main__":
    main()
