"""Holograms wider than one CTA's shared memory holds a row of (nx or ny
between 24577 and 32768): the spectrum's own row passes split over a cluster
of two CTAs (a radix-2 step on the way out, the halves exchanged through
distributed shared memory), and coordinate tables whose fine positions pass
+-2^15 (the pull-back table keeps its base as an offset from 2k, the output
map 32-bit bases).  Checked against the FP64 oracle on 32768 x 64 and
64 x 32768 holograms (the long axis at 83 deg FoV needs N' = 40960), full and
partial views, field within 1e-5."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
LAM, PITCH, Z = 532e-9, 0.4e-6, 10e-3


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


def _holo(ny, nx, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex64)


@pytest.mark.parametrize("shape", [(64, 32768), (32768, 64)])
def test_large_hologram_full_view(nf, shape):
    ny, nx = shape
    H = _holo(ny, nx, nx)
    info = nf.view_plan(LAM, PITCH, nx, ny, nf.View(z=Z))
    assert max(info["np_x"], info["np_y"]) == 40960
    plan = nf.Plan(LAM, PITCH, nx, ny, torch.from_numpy(H).cuda())
    f = plan.reconstruct(nf.View(z=Z, kind=nf.OUT_FIELD)).cpu().numpy()
    plan.close()
    ref, _ = oracle.reconstruct(H, LAM, PITCH, Z)
    e = float(np.linalg.norm(f - ref) / np.linalg.norm(ref))
    print("%d x %d: rel_l2 = %.3e" % (nx, ny, e))
    assert e <= TOL, e


def test_large_hologram_partial_view(nf):
    ny, nx = 64, 32768
    H = _holo(ny, nx, 3)
    B = oracle.plan_view(LAM, PITCH, nx, ny, Z)["width"]
    p = B / nx
    kw = dict(z=Z, center_x=(29000 - nx / 2) * p, center_y=(40 - ny / 2) * B / ny,
              width=1500 * p, height=20 * B / ny, out_nx=1500, out_ny=20)
    plan = nf.Plan(LAM, PITCH, nx, ny, torch.from_numpy(H).cuda())
    f = plan.reconstruct(nf.View(kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    plan.close()
    ref, _ = oracle.reconstruct(H, LAM, PITCH, Z, kw["center_x"], kw["center_y"], kw["width"],
                                kw["height"], kw["out_nx"], kw["out_ny"])
    e = float(np.linalg.norm(f - ref) / np.linalg.norm(ref))
    print("partial view near the edge of a 32768-wide hologram: rel_l2 = %.3e" % e)
    assert e <= TOL, e
