"""Paper-literal variant: the degree-8 polynomial surrogate for 2F1 (Section 4,
initialisation step 1; plan flag NUFDS_FLAG_PAPER_POLY_M) on the GPU against
the oracle running the same surrogate, and its distance from the exact method."""
import numpy as np
import pytest

import oracle
import synth

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


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("partial", [False, True])
def test_polynomial_variant_vs_oracle(nf, partial):
    lam, pitch, n, z = 532e-9, 0.307e-6, 384, 0.6
    pts = synth.points(55, 20, (0.4, 1.0), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    H = synth.hologram(pts, lam, pitch, n, n)
    kw = dict(z=z)
    if partial:
        B = oracle.plan_view(lam, pitch, n, n, z)["width"]
        kw = dict(z=z, center_x=0.3 * B, center_y=-0.25 * B, width=0.25 * B, height=0.2 * B,
                  out_nx=120, out_ny=96)
    h = torch.from_numpy(H).cuda()
    plan = nf.Plan(lam, pitch, n, n, h, flags=nf.FLAG_PAPER_POLY_M)
    exact = nf.Plan(lam, pitch, n, n, h)
    f = plan.reconstruct(nf.View(kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    fe = exact.reconstruct(nf.View(kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    torch.cuda.synchronize()
    args = (kw["z"], kw.get("center_x", 0.0), kw.get("center_y", 0.0), kw.get("width", 0.0),
            kw.get("height", 0.0), kw.get("out_nx", 0), kw.get("out_ny", 0))
    with oracle.paper_poly(lam, pitch):
        ref, _ = oracle.reconstruct(H, lam, pitch, *args)
    ref_exact, _ = oracle.reconstruct(H, lam, pitch, *args)
    e = _rel(f, ref)
    d_gpu, d_oracle = _rel(f, fe), _rel(ref, ref_exact)
    print("polynomial variant vs oracle: rel_l2 = %.3e; its distance from the exact method: "
          "GPU %.3e, oracle %.3e" % (e, d_gpu, d_oracle))
    assert e <= TOL
    # the variant's distance from the exact method is the oracle's, well above the tolerance
    # of either path, so the flag really changes the maps
    assert abs(d_gpu - d_oracle) <= 0.05 * d_oracle + 2 * TOL
    plan.close()
    exact.close()


@pytest.mark.parametrize("geom,partial,poly", [((532e-9, 0.307e-6, 384, 384, 0.6), False, False),
                                               ((532e-9, 0.4e-6, 256, 256, 0.5), True, False),
                                               ((640e-9, 0.5e-6, 320, 320, 0.8), False, True),
                                               ((532e-9, 0.4e-6, 320, 192, 0.6), False, False),
                                               ((532e-9, 0.307e-6, 192, 256, 0.7), True, True)])
def test_linear_variant_vs_oracle(nf, geom, partial, poly):
    """Paper-literal bilinear resampling (plan flag NUFDS_FLAG_PAPER_LINEAR) on
    the GPU against the oracle running the same variant, field and intensity;
    its distance from the ideal method is the oracle's."""
    lam, pitch, nx, ny, z = geom
    pts = synth.points(71, 16, (0.4, 1.2), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    H = synth.hologram(pts, lam, pitch, nx, ny)
    kw = dict(z=z)
    if partial:
        v = oracle.plan_view(lam, pitch, nx, ny, z)
        B, Bh = v["width"], v["height"]
        kw = dict(z=z, center_x=-0.2 * B, center_y=0.3 * Bh, width=0.3 * B, height=0.25 * Bh,
                  out_nx=100, out_ny=84)
    flags = nf.FLAG_PAPER_LINEAR | (nf.FLAG_PAPER_POLY_M if poly else 0)
    h = torch.from_numpy(H).cuda()
    plan = nf.Plan(lam, pitch, nx, ny, h, flags=flags)
    ideal = nf.Plan(lam, pitch, nx, ny, h, flags=nf.FLAG_PAPER_POLY_M if poly else 0)
    f = plan.reconstruct(nf.View(kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    i = plan.reconstruct(nf.View(**kw)).cpu().numpy()
    fi = ideal.reconstruct(nf.View(kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    torch.cuda.synchronize()
    args = (kw["z"], kw.get("center_x", 0.0), kw.get("center_y", 0.0), kw.get("width", 0.0),
            kw.get("height", 0.0), kw.get("out_nx", 0), kw.get("out_ny", 0))
    with oracle.paper_linear():
        if poly:
            with oracle.paper_poly(lam, pitch):
                ref, ref_i = oracle.reconstruct(H, lam, pitch, *args)
        else:
            ref, ref_i = oracle.reconstruct(H, lam, pitch, *args)
    if poly:
        with oracle.paper_poly(lam, pitch):
            ref_ideal, _ = oracle.reconstruct(H, lam, pitch, *args)
    else:
        ref_ideal, _ = oracle.reconstruct(H, lam, pitch, *args)
    e, ei = _rel(f, ref), _rel(i, ref_i)
    d_gpu, d_oracle = _rel(f, fi), _rel(ref, ref_ideal)
    print("linear variant vs oracle: field %.3e, intensity %.3e; distance from the ideal "
          "resampling: GPU %.3e, oracle %.3e" % (e, ei, d_gpu, d_oracle))
    assert e <= TOL and ei <= TOL
    assert abs(d_gpu - d_oracle) <= 0.05 * d_oracle + 2 * TOL
    plan.close()
    ideal.close()


def test_linear_variant_limits(nf):
    lam, pitch, n = 532e-9, 0.4e-6, 128
    with pytest.raises(nf.NufdsError) as e:
        nf.Plan(lam, pitch, n, n, precision=nf.FP16_STORE, flags=nf.FLAG_PAPER_LINEAR)
    assert e.value.code == nf.EUNSUPPORTED
    H = torch.from_numpy(synth.hologram(
        synth.points(3, 4, (0.4, 0.8), synth.tan_half_fov(lam, pitch), (0.5, 1.0)),
        lam, pitch, n, n)).cuda()
    lin = nf.Plan(lam, pitch, n, n, H, flags=nf.FLAG_PAPER_LINEAR)
    ideal = nf.Plan(lam, pitch, n, n, H)
    views = [nf.View(z=0.5), nf.View(z=0.5)]
    outs = [ideal.output_like(v) for v in views]
    st = nf.reconstruct_batch([lin, ideal], views, outs)
    torch.cuda.synchronize()
    assert st == [nf.EUNSUPPORTED, 0]
    # a sweep of the linear plan gives its single-view results
    sv = [nf.View(z=z, kind=nf.OUT_FIELD) for z in (0.5, 0.9)]
    ref = [lin.reconstruct(v).clone() for v in sv]
    got, st = lin.reconstruct_sweep(sv)
    torch.cuda.synchronize()
    assert st == [0, 0]
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    lin.close()
    ideal.close()
