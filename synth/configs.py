"""The synthetic workloads, as recipes (sizes, geometry, point-cloud statistics, seeds).

Each recipe stands in for one of the paper's workloads: seeded random point
clouds inside the square pyramid of the full field of view, holograms made by
the point-source model of Eq. 3, at the sizes and fields of view the paper
reports (up to 16K and 120 degrees).  The Neptune point clouds of Section 5
are not available; these recipes take their shape (dense random points,
random phase, wide and ultra-wide FoV) instead.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import points, hologram, tan_half_fov

LAMBDA_532 = 532e-9


@dataclass(frozen=True)
class Workload:
    name: str
    n: int                       # hologram is n x n complex64
    wavelength: float
    pitch: float
    n_points: int
    z_range: tuple               # point depths, metres
    amp_range: tuple
    z_view: float                # reconstruction distance of the full view
    seed: int
    spread: float = 1.0          # points lie within spread * full-view half width
    partial_views: int = 0       # number of seeded partial views
    partial_size: int = 0        # their size in full-view pixels
    ny: int = 0                  # rows of the hologram when not square (0: n)

    @property
    def rows(self) -> int:
        return self.ny or self.n

    @property
    def tan_half(self) -> float:
        return tan_half_fov(self.wavelength, self.pitch)

    def point_cloud(self) -> np.ndarray:
        return points(self.seed, self.n_points, self.z_range, self.tan_half, self.amp_range,
                      self.spread)

    def make_hologram(self, threads: int = 0) -> np.ndarray:
        return hologram(self.point_cloud(), self.wavelength, self.pitch, self.n, self.rows,
                        threads)

    def partial_view_offsets(self) -> np.ndarray:
        """Seeded view centres as integer full-view pixel offsets from the centre.

        Views of partial_size^2 pixels at the full-view pitch, entirely inside
        the full view.  Returns (partial_views, 2) int64 offsets (dx, dy) of the
        view centre pixel from the full-view centre pixel.
        """
        rng = np.random.default_rng(self.seed + 7)
        lim = (self.n - self.partial_size) // 2
        return rng.integers(-lim, lim + 1, size=(self.partial_views, 2)).astype(np.int64)


# Full-view reconstruction of a small CGH (8 points, unit amplitude).
SMALL_512 = Workload("pointcloud-512-532nm-0.4um-8pt", 512, LAMBDA_532, 0.4e-6, 8,
                     (0.3, 0.7), (1.0, 1.0), 0.5, seed=20241017)
# Wide-angle 4096^2 (64 deg), 2000 points in a frustum z in [0.5, 1.5] m, full
# view at 0.85 m (the depths of the 8K wide-angle tests of Section 5).
WA_4096 = Workload("pointcloud-4096-532nm-0.5um-2000pt", 4096, LAMBDA_532, 0.5e-6, 2000,
                   (0.5, 1.5), (0.5, 1.0), 0.85, seed=20241018)
# Ultra-wide-angle 16384^2 (120 deg), 20000 points in z in [0.6, 3.16] m (the
# object of the 16K test of Section 5: front at 0.6 m, 2.56 m deep), full view
# at 0.8 m (its Fig. 10a depth) plus 16 partial views of 2048^2 at the
# full-view pitch.
UWA_16K = Workload("pointcloud-16384-532nm-0.307um-20000pt", 16384, LAMBDA_532, 0.307e-6,
                   20000, (0.6, 3.16), (0.5, 1.0), 0.8, seed=20241019,
                   partial_views=16, partial_size=2048)

# A 16384 x 2048 strip of the ultra-wide-angle geometry: its full view runs
# the same 23040-point Fresnel rows along x as the 16K view, on 5760 rows
# (about 3 GB of pass traffic), a size for detailed kernel captures.
STRIP_16K = Workload("strip-16384x2048-532nm-0.307um-2000pt", 16384, LAMBDA_532, 0.307e-6,
                     2000, (0.6, 3.16), (0.5, 1.0), 0.8, seed=20241023, ny=2048)

# The same three shapes with the point depths and viewing distances stated for
# the benchmark, in millimetres: the hologram is then not small against the
# object distance (5 mm aperture at 6 mm for 16K), outside the regime where the
# method's paraxial premise holds, so these are parity and throughput cases,
# not refocus cases.
# 512^2, 0.4 um (83 deg), 8 unit-amplitude points, z in [0.5, 2] mm, view at 1 mm.
SMALL_512_MM = Workload("pointcloud-512-532nm-0.4um-8pt-z0.5-2mm", 512, LAMBDA_532, 0.4e-6, 8,
                        (0.5e-3, 2e-3), (1.0, 1.0), 1e-3, seed=20241101)
# 4096^2, 0.5 um (64 deg), 2000 points, z in [1, 5] mm, amplitudes U[0.5, 1], view at 3 mm.
WA_4096_MM = Workload("pointcloud-4096-532nm-0.5um-2000pt-z1-5mm", 4096, LAMBDA_532, 0.5e-6,
                      2000, (1e-3, 5e-3), (0.5, 1.0), 3e-3, seed=20241102)
# 16384^2, 0.307 um (120 deg), 20000 points, z in [2, 10] mm, amplitudes U[0.5, 1],
# full view at 6 mm (the middle of the depth range) plus 16 partial views of 2048^2.
UWA_16K_MM = Workload("pointcloud-16384-532nm-0.307um-20000pt-z2-10mm", 16384, LAMBDA_532,
                      0.307e-6, 20000, (2e-3, 10e-3), (0.5, 1.0), 6e-3, seed=20241103,
                      partial_views=16, partial_size=2048)

ALL = {w.name: w for w in (SMALL_512, WA_4096, UWA_16K, STRIP_16K, SMALL_512_MM, WA_4096_MM,
                           UWA_16K_MM)}


@dataclass(frozen=True)
class BatchRequest:
    holo: int          # index into the batch holograms
    size: int          # view is size x size pixels at the full-view pitch of its z
    dx: int            # view-centre offset from the full-view centre, in full-view pixels
    dy: int
    z: float


# Depths of the batched and served workloads as stated for the benchmark
# (millimetres: points and views at z in [1, 8] mm for the batch; views at z in
# [max(2 mm, N pitch^2 / lambda), 10 mm] for serving), against the paper's own
# object depths (metres) of the *_paper variants.
BATCH_Z_MM = (1e-3, 8e-3)
SERVE_Z_MM = (2e-3, 10e-3)
MAX_FFT = 49152  # the largest row the passes take (split over two CTAs above 24576)


def batch_workload(seed: int = 20241020, n_holo: int = 8, n_req: int = 64, lam: float = LAMBDA_532,
                   sizes=(2048, 4096, 8192), view_sizes=(256, 512, 1024, 2048, 4096),
                   z_range=(0.5, 3.0), max_fft: int = 24576):
    """Holograms of seeded sizes and pitches, and partial-view requests of
    uneven size, position and depth over them (the batched workload).  A
    request's z is drawn in [max(z_min, z_chirp), z_max], where z_chirp keeps
    the FFT size of the Fresnel stage within max_fft ((N pitch)^2/(lambda z)
    <= max_fft); at the paper's object depths (0.5-3 m) it does not bind, nor
    at the stated millimetre depths with max_fft = MAX_FFT.  Point depths
    follow z_range."""
    rng = np.random.default_rng(seed)
    holos = []
    for i in range(n_holo):
        n = int(rng.choice(sizes))
        pitch = float(rng.uniform(0.3e-6, 0.5e-6))
        npts = int(rng.integers(500, 5001))
        holos.append(Workload("batch-holo-%d-%d" % (i, n), n, lam, pitch, npts, z_range,
                              (0.5, 1.0), 1.0, seed=seed * 100 + i))
    reqs = []
    for _ in range(n_req):
        h = int(rng.integers(0, n_holo))
        w = holos[h]
        s = int(rng.choice([v for v in view_sizes if v <= w.n]))
        lim = (w.n - s) // 2
        dx, dy = (int(v) for v in rng.integers(-lim, lim + 1, size=2))
        zc = (w.n * w.pitch) ** 2 / (lam * max_fft) * 1.02
        z = float(rng.uniform(max(z_range[0], zc), z_range[1]))
        reqs.append(BatchRequest(h, s, dx, dy, z))
    return holos, reqs


def serve_workload(seed: int = 20241021, n_holo: int = 12, n_req: int = 10000, rate: float = 200.0,
                   lam: float = LAMBDA_532, sizes=(2048, 4096, 8192, 16384),
                   view_sizes=(256, 512, 1024, 2048, 4096), max_fft: int = 24576,
                   resident_cap_bytes: float = 72e9, z_range=(0.6, 3.2), stated=False):
    """Resident holograms and a seeded Poisson stream of view requests (the
    serving workload).  Hologram sizes are drawn from `sizes` until the
    resident set (spectrum 32 N^2 B plus tables ~30 N^2 B each) would pass
    resident_cap_bytes; then the smallest size is used.  A request's z is drawn
    in [max(z_min, z_chirp), z_max] (z_chirp keeps the Fresnel-stage FFT within
    max_fft; at the paper's object depths of 0.5-3 m it does not bind); with
    stated=True (millimetre depths) z_min is also at least N pitch^2 / lambda
    of the request's hologram, so N' stays within about N.  Points lie in
    z_range.  Returns (holograms, requests, arrival_times)."""
    rng = np.random.default_rng(seed)
    holos, resident = [], 0.0
    for i in range(n_holo):
        n = int(rng.choice(sizes))
        if resident + 62.0 * n * n > resident_cap_bytes:
            n = min(sizes)
        resident += 62.0 * n * n
        pitch = float(rng.uniform(0.307e-6, 0.5e-6))
        npts = int(rng.integers(500, 5001))
        holos.append(Workload("serve-holo-%d-%d" % (i, n), n, lam, pitch, npts, z_range,
                              (0.5, 1.0), 1.0, seed=seed * 100 + i))
    reqs = []
    for _ in range(n_req):
        h = int(rng.integers(0, n_holo))
        w = holos[h]
        s = int(rng.choice([v for v in view_sizes if v <= w.n]))
        lim = (w.n - s) // 2
        dx, dy = (int(v) for v in rng.integers(-lim, lim + 1, size=2))
        zc = (w.n * w.pitch) ** 2 / (lam * max_fft) * 1.02
        zlo = max(z_range[0], zc, w.n * w.pitch ** 2 / lam if stated else 0.0)
        z = float(rng.uniform(zlo, z_range[1]))
        reqs.append(BatchRequest(h, s, dx, dy, z))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    return holos, reqs, t
