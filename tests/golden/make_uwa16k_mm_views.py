#!/usr/bin/env python
"""Writes uwa16k_mm_views_samples.txt: FP64 oracle values of the 16 seeded
2048^2 partial views of the 16384^2 ultra-wide-angle workload at its stated
depths (20000 points at z in [2, 10] mm, views at z = 6 mm, 120 deg FoV), at
seeded sample pixels of each view.

The hologram comes from the seeded input generator ``synth`` (its GPU form:
an exact FP64 sum over 2.7e8 pixels x 20000 points is out of reach on the
host), so this script needs a GPU for that one step; everything it stores is
computed by ``oracle`` on the host, one call for the 16 views (the gridded
transform of the hologram is shared; about 30 GB of host memory).  The file
records the sha256 of the hologram's bytes so that a consumer can check it
regenerates the same input.

  python tests/golden/make_uwa16k_mm_views.py
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from synth.configs import UWA_16K_MM as W  # noqa: E402

OUT = os.path.join(HERE, "uwa16k_mm_views_samples.txt")
SAMPLES_PER_VIEW = 256
SEED = 20241104


def views():
    """The 16 partial views as oracle keyword dicts (centres on the full
    view's pixel lattice, full-view pitch, partial_size^2 pixels)."""
    full = oracle.plan_view(W.wavelength, W.pitch, W.n, W.n, W.z_view)
    p = full["width"] / W.n
    s = W.partial_size
    return [dict(z=W.z_view, cx=float(dx) * p, cy=float(dy) * p, w=s * p, h=s * p, ox=s, oy=s)
            for dx, dy in W.partial_view_offsets()]


def sample_pixels(v):
    rng = np.random.default_rng(SEED + v)
    return (rng.integers(0, W.partial_size, SAMPLES_PER_VIEW),
            rng.integers(0, W.partial_size, SAMPLES_PER_VIEW))


def hologram_host():
    """The workload's hologram from the seeded generator, as host complex64."""
    import torch
    d = synth.gpu_hologram(W.point_cloud(), W.wavelength, W.pitch, W.n, W.n)
    h = d.cpu().numpy()
    del d
    torch.cuda.empty_cache()
    return h


def digest(h: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(h).view(np.uint8)).hexdigest()


def main():
    t = time.time()
    H = hologram_host()
    dig = digest(H)
    t_h = time.time() - t
    vs = views()
    t = time.time()
    outs = oracle.reconstruct_views(H, W.wavelength, W.pitch, vs)
    t_o = time.time() - t
    del H
    with open(OUT, "w") as fo:
        fo.write("# Oracle (FP64) fields of the 16 seeded %d^2 partial views of the %d^2 hologram\n"
                 % (W.partial_size, W.n))
        fo.write("# %s (Section 4, Fig. 3 steps two to five; Eq. 17), written by\n" % W.name)
        fo.write("# tests/golden/make_uwa16k_mm_views.py: %d seeded pixels per view, then its\n"
                 % SAMPLES_PER_VIEW)
        fo.write("# brightest; oracle threads %d, %.0f s for the 16 views.\n"
                 % (oracle.num_threads(), t_o))
        fo.write("# hologram sha256 %s\n" % dig)
        fo.write("# columns: view, row j, column i, Re, Im\n")
        for v, (f, _) in enumerate(outs):
            j, i = sample_pixels(v)
            jm, im = np.unravel_index(int(np.argmax(np.abs(f))), f.shape)
            for a, b in zip(np.append(j, jm), np.append(i, im)):
                z = f[a, b]
                fo.write("%d %d %d %.17g %.17g\n" % (v, a, b, z.real, z.imag))
    print("hologram %.1f s (sha256 %s), oracle %.1f s -> %s" % (t_h, dig[:16], t_o, OUT))


if __name__ == "__main__":
    main()
