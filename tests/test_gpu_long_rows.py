"""Fresnel rows longer than one CTA's shared memory holds (N' > 24576): each
row of the view passes is split over a cluster of two CTAs (a radix-2 step
on the way in and out, the halves exchanged through distributed shared
memory).  Checked against the FP64 oracle on rectangular holograms whose
long axis forces N' of 30720 to 49152 at small distances (the chirp sampling
rule N' >= (N pitch)^2 / (lambda z)), with the short axis keeping the
oracle's grids small; both orientations, FP32 within 1e-5 and FP16 storage
within its bound; a batch that mixes a split-row view with an ordinary one
returns each view as its single-view call does.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
LAM, PITCH = 532e-9, 0.5e-6


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


def _z_for(n, chirp):
    """Distance at which the chirp rule asks for `chirp` points on an n-pixel axis."""
    return (n * PITCH) ** 2 / (LAM * chirp)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_field(nf, H, z, prec=None, **kw):
    ny, nx = H.shape
    h = torch.from_numpy(H).cuda()
    plan = nf.Plan(LAM, PITCH, nx, ny, h, precision=nf.FP32 if prec is None else prec)
    f = plan.reconstruct(nf.View(z=z, kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    plan.close()
    return f


@pytest.mark.parametrize("chirp,np_expect", [(28000, 30720), (31500, 32768), (35000, 36864),
                                             (48000, 49152)])
@pytest.mark.parametrize("long_axis", ["x", "y"])
def test_split_rows_match_oracle(nf, chirp, np_expect, long_axis):
    nlong, nshort = 2048, 64
    ny, nx = (nshort, nlong) if long_axis == "x" else (nlong, nshort)
    z = _z_for(nlong, chirp)
    info = nf.view_plan(LAM, PITCH, nx, ny, nf.View(z=z))
    got_np = info["np_x"] if long_axis == "x" else info["np_y"]
    assert got_np == np_expect > 24576
    H = _holo(ny, nx, chirp)
    f = _gpu_field(nf, H, z)
    ref, _ = oracle.reconstruct(H, LAM, PITCH, z)
    e = _rel(f, ref)
    print("N' = %d along %s: rel_l2 = %.3e" % (np_expect, long_axis, e))
    assert e <= TOL, e


def test_split_rows_partial_view_and_fp16(nf):
    nx, ny = 2048, 64
    z = _z_for(nx, 31500)
    H = _holo(ny, nx, 7)
    B = oracle.plan_view(LAM, PITCH, nx, ny, z)["width"]
    kw = dict(center_x=0.21 * B, center_y=-0.1 * B, width=0.3 * B, height=0.5 * B, out_nx=300,
              out_ny=20)
    assert nf.view_plan(LAM, PITCH, nx, ny, nf.View(z=z, **kw))["np_x"] == 32768
    ref, _ = oracle.reconstruct(H, LAM, PITCH, z, kw["center_x"], kw["center_y"], kw["width"],
                                kw["height"], kw["out_nx"], kw["out_ny"])
    assert _rel(_gpu_field(nf, H, z, **kw), ref) <= TOL
    e16 = _rel(_gpu_field(nf, H, z, prec=nf.FP16_STORE, **kw), ref)
    print("FP16 storage, split rows: rel_l2 = %.3e" % e16)
    assert e16 <= 3e-3


def test_batch_mixing_split_and_ordinary_rows(nf):
    nx, ny = 2048, 64
    H = _holo(ny, nx, 11)
    plan = nf.Plan(LAM, PITCH, nx, ny, torch.from_numpy(H).cuda())
    views = [nf.View(z=_z_for(nx, 31500), kind=nf.OUT_FIELD),
             nf.View(z=_z_for(nx, 9000), kind=nf.OUT_FIELD),
             nf.View(z=_z_for(nx, 40000), kind=nf.OUT_INTENSITY)]
    nps = [plan.view_plan(v)["np_x"] for v in views]
    assert nps[0] > 24576 and nps[1] <= 24576 and nps[2] > 24576
    outs = [plan.output_like(v) for v in views]
    st = nf.reconstruct_batch([plan] * 3, views, outs)
    assert list(st) == [0, 0, 0]
    for v, o in zip(views, outs):
        single = plan.reconstruct(v)
        torch.cuda.synchronize()
        assert torch.equal(single, o)
    plan.close()
