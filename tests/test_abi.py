"""The C-ABI library without a GPU: it builds, loads, exports every function
include/nufds.h declares, and its host-only view planner makes the same
integer decisions (band, FFT sizes, band centre) as the oracle's."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2410_13474_gb300 as nf
from paper_2410_13474_gb300 import build as nfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    nfbuild.build()
    return nf.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "nufds.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nufds_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(built):
    names = _declared()
    assert set(names) == set(nf.ABI_FUNCTIONS)
    for n in names:
        assert hasattr(built, n), n
    assert nf.status_string(nf.EINVAL) == "invalid argument"
    assert nf.status_string(0) == "ok"


def test_planner_rejects_bad_geometry(built):
    with pytest.raises(nf.NufdsError) as e:
        nf.view_plan(0.6e-6, 0.3e-6, 64, 64, nf.View(z=1e-3))   # lambda >= 2 pitch
    assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError):
        nf.view_plan(0.5e-6, 0.4e-6, 64, 64, nf.View(z=0.0))
    with pytest.raises(nf.NufdsError):
        nf.view_plan(0.5e-6, 0.4e-6, 64, 64, nf.View(z=1e-3, width=1e-4, height=0.0))


CASES = [
    # (lambda, pitch, nx, ny, view kwargs)
    (532e-9, 0.4e-6, 512, 512, dict(z=1e-3)),
    (532e-9, 0.5e-6, 4096, 4096, dict(z=3e-3)),
    (532e-9, 0.307e-6, 16384, 16384, dict(z=6e-3)),
    (532e-9, 0.307e-6, 16384, 16384, dict(z=2e-3)),
    (532e-9, 0.4e-6, 256, 192, dict(z=0.7e-3)),
    (640e-9, 0.5e-6, 1024, 1024, dict(z=1.3e-3, center_x=2e-4, center_y=-1e-4, width=3e-4,
                                      height=2e-4, out_nx=96, out_ny=64)),
    (532e-9, 0.3e-6, 2048, 2048, dict(z=4e-3, center_x=-1.5e-3, center_y=1.2e-3, width=1e-3,
                                      height=1e-3, out_nx=512, out_ny=512)),
]


@pytest.mark.parametrize("case", CASES)
def test_planner_matches_oracle(built, case):
    lam, pitch, nx, ny, kw = case
    v = nf.View(**kw)
    got = nf.view_plan(lam, pitch, nx, ny, v)
    ref = oracle.plan_view(lam, pitch, nx, ny, v.z, v.center_x, v.center_y, v.width, v.height,
                           v.out_nx, v.out_ny)
    for k in ["out_nx", "out_ny", "k_lo_x", "k_hi_x", "k_lo_y", "k_hi_y", "np_x", "np_y",
              "k_c_x", "k_c_y"]:
        assert got[k] == ref[k], k
    assert abs(got["pitch_out_x_m"] / ref["pitch_out_x"] - 1) < 1e-14
    assert abs(got["width_m"] / ref["width"] - 1) < 1e-14


def test_full_view_is_on_its_own_lattice(built):
    info = nf.view_plan(532e-9, 0.4e-6, 512, 512, nf.View(z=1e-3))
    assert info["on_full_view_lattice"] == 1
    B = info["width_m"]
    p = B / 512
    sub = nf.View(z=1e-3, center_x=(300 - 256) * p, center_y=(100 - 256) * p, width=64 * p,
                  height=32 * p, out_nx=64, out_ny=32)
    assert nf.view_plan(532e-9, 0.4e-6, 512, 512, sub)["on_full_view_lattice"] == 1
    off = nf.View(z=1e-3, center_x=0.3 * p, width=64 * p, height=64 * p, out_nx=64, out_ny=64)
    assert nf.view_plan(532e-9, 0.4e-6, 512, 512, off)["on_full_view_lattice"] == 0


def test_planner_matches_oracle_random_views(built):
    """The library evaluates Eq. 17 only at the corners and at the edge pixels
    nearest the axes; the oracle scans every boundary pixel.  Same integers."""
    rng = np.random.default_rng(1)
    for it in range(150):
        n = int(rng.choice([256, 512, 1024, 2048]))
        lam, pitch = 532e-9, float(rng.uniform(0.3e-6, 0.5e-6))
        z = float(rng.uniform(0.5e-3, 5e-3))
        B = oracle.plan_view(lam, pitch, n, n, z)["width"]
        p = B / n * (float(rng.uniform(0.5, 1.5)) if it % 5 == 0 else 1.0)
        ox, oy = int(rng.integers(8, n)), int(rng.integers(8, n))
        cx = 0.0 if it % 3 == 0 else float(rng.uniform(-0.5, 0.5)) * (B - ox * p)
        cy = float(rng.uniform(-0.5, 0.5)) * (B - oy * p)
        v = nf.View(z=z, center_x=cx, center_y=cy, width=ox * p, height=oy * p, out_nx=ox,
                    out_ny=oy)
        got = nf.view_plan(lam, pitch, n, n, v)
        ref = oracle.plan_view(lam, pitch, n, n, z, cx, cy, ox * p, oy * p, ox, oy)
        for k in ["k_lo_x", "k_hi_x", "k_lo_y", "k_hi_y", "np_x", "np_y"]:
            assert got[k] == ref[k], (it, k)


def test_polynomial_planner_matches_oracle(built):
    """With the paper's polynomial surrogate (plan flag) the planner's Eq. 17
    uses the surrogate, like the oracle inside its paper_poly context."""
    rng = np.random.default_rng(2)
    for it in range(40):
        n = int(rng.choice([256, 512, 1024]))
        lam, pitch = 532e-9, float(rng.uniform(0.3e-6, 0.5e-6))
        z = float(rng.uniform(0.3, 2.0))
        B = oracle.plan_view(lam, pitch, n, n, z)["width"]
        p = B / n
        ox, oy = int(rng.integers(8, n)), int(rng.integers(8, n))
        cx = float(rng.uniform(-0.5, 0.5)) * (B - ox * p)
        cy = float(rng.uniform(-0.5, 0.5)) * (B - oy * p)
        v = nf.View(z=z, center_x=cx, center_y=cy, width=ox * p, height=oy * p, out_nx=ox,
                    out_ny=oy)
        got = nf.view_plan(lam, pitch, n, n, v, flags=nf.FLAG_PAPER_POLY_M)
        with oracle.paper_poly(lam, pitch):
            ref = oracle.plan_view(lam, pitch, n, n, z, cx, cy, ox * p, oy * p, ox, oy)
        for k in ["k_lo_x", "k_hi_x", "k_lo_y", "k_hi_y", "np_x", "np_y"]:
            assert got[k] == ref[k], (it, k)


def test_plain_frt_planner_matches_oracle(built):
    """Plain Fresnel transform views (no stretch): band from the view's own
    extent, same integers as the oracle's stretch = 0 planner."""
    rng = np.random.default_rng(2)
    for it in range(60):
        n = int(rng.choice([256, 512, 1024]))
        lam, pitch = 532e-9, float(rng.uniform(0.3e-6, 0.5e-6))
        z = float(rng.uniform(0.3, 3.0))
        B = oracle.plan_view(lam, pitch, n, n, z)["width"]
        p = B / n
        ox, oy = int(rng.integers(8, n)), int(rng.integers(8, n))
        cx = float(rng.uniform(-0.5, 0.5)) * (B - ox * p)
        cy = float(rng.uniform(-0.5, 0.5)) * (B - oy * p)
        v = nf.View(z=z, center_x=cx, center_y=cy, width=ox * p, height=oy * p, out_nx=ox,
                    out_ny=oy, mode=nf.MODE_PLAIN_FRT)
        got = nf.view_plan(lam, pitch, n, n, v)
        ref = oracle.plan_view(lam, pitch, n, n, z, cx, cy, ox * p, oy * p, ox, oy, stretch=0)
        for k in ["k_lo_x", "k_hi_x", "k_lo_y", "k_hi_y", "np_x", "np_y"]:
            assert got[k] == ref[k], (it, k)
        assert got["on_full_view_lattice"] == 0
    with pytest.raises(nf.NufdsError):
        nf.view_plan(532e-9, 0.4e-6, 64, 64, nf.View(z=0.5, mode=7))


def test_planner_limits(built):
    """Largest supported FFT: N' <= 49152 per axis (rows up to 24576 in one
    CTA's shared memory, longer ones split over a 2-CTA cluster): the
    plain-FrT full view of a 16K hologram at 120 deg needs 36864 and is
    planned; a 16K view at 0.5 mm needs ~95000 by the chirp rule and is
    refused; nx must be a positive multiple of 4."""
    lam, pitch = 532e-9, 0.307e-6
    ok = nf.view_plan(lam, pitch, 16384, 16384, nf.View(z=0.8))
    assert ok["np_x"] == 23040
    plain = nf.view_plan(lam, pitch, 16384, 16384, nf.View(z=0.8, mode=nf.MODE_PLAIN_FRT))
    assert plain["np_x"] == plain["np_y"] == 36864
    with pytest.raises(nf.NufdsError) as e:
        nf.view_plan(lam, pitch, 16384, 16384, nf.View(z=0.5e-3))
    assert e.value.code == nf.EUNSUPPORTED
    with pytest.raises(nf.NufdsError) as e:
        nf.view_plan(lam, pitch, 64, 64, nf.View(z=0.5, out_nx=70000, out_ny=8))
    assert e.value.code == nf.EUNSUPPORTED
    # a one-pixel view plans to the band around that pixel
    one = nf.view_plan(lam, pitch, 256, 256, nf.View(z=0.5, width=1e-5, height=1e-5, out_nx=1,
                                                    out_ny=1))
    assert one["out_nx"] == 1 and one["k_hi_x"] - one["k_lo_x"] <= 2


def test_product_library_has_no_bounds_checks(built):
    """The product build compiles the gathers' bounds checks out: the debug
    query answers EUNSUPPORTED (no CUDA call is made to say so)."""
    with pytest.raises(nf.NufdsError) as e:
        nf.bounds_violations()
    assert e.value.code == nf.EUNSUPPORTED
