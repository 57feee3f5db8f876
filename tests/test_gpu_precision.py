"""Storage-precision variants: the cached spectrum and the inter-pass arrays
held as FP16 (scaled by a power of two from an l1 bound) or BF16, arithmetic
in FP32.  Their error against the FP64 oracle is reported, and bounded so a
regression shows: FP16 (11-bit significand) within 3e-3 relative L2 of the
field, BF16 (8-bit) within 2e-2."""
import numpy as np
import pytest

import oracle
from synth.configs import SMALL_512

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUNDS = {"fp16": 3e-3, "bf16": 2e-2}


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def case512():
    w = SMALL_512
    H = w.make_hologram()
    ref, _ = oracle.reconstruct(H, w.wavelength, w.pitch, w.z_view)
    return w, H, ref


@pytest.mark.parametrize("name", ["fp16", "bf16"])
def test_storage_variant_error(nf, case512, name):
    w, H, ref = case512
    prec = {"fp16": nf.FP16_STORE, "bf16": nf.BF16_STORE}[name]
    h = torch.from_numpy(H).cuda()
    plan = nf.Plan(w.wavelength, w.pitch, w.n, w.n, h, precision=prec)
    f = plan.reconstruct(nf.View(z=w.z_view, kind=nf.OUT_FIELD)).cpu().numpy()
    plan.close()
    e = _rel(f, ref)
    print("%s storage: rel_l2 vs FP64 oracle = %.3e" % (name, e))
    assert np.all(np.isfinite(f))
    assert e <= BOUNDS[name]


def test_fp16_scaling_survives_large_dynamic_range(nf):
    # a bright point plus weak background: no overflow, error still bounded
    import synth
    lam, pitch, n, z = 532e-9, 0.4e-6, 256, 1e-3
    pts = synth.points(3, 12, (0.6e-3, 1.4e-3), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    pts[0, 3] = 500.0
    H = synth.hologram(pts, lam, pitch, n, n)
    ref, _ = oracle.reconstruct(H, lam, pitch, z)
    plan = nf.Plan(lam, pitch, n, n, torch.from_numpy(H).cuda(), precision=nf.FP16_STORE)
    f = plan.reconstruct(nf.View(z=z, kind=nf.OUT_FIELD)).cpu().numpy()
    plan.close()
    assert np.all(np.isfinite(f))
    assert _rel(f, ref) <= BOUNDS["fp16"]
