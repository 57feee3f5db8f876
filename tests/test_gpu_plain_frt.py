"""Plain Fresnel transform mode (Eq. 2 alone at z, no stretch, x' = x_o; the
paper's Fig. 10b comparison) against the oracle's stretch = 0 path."""
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


def _holo(lam, pitch, n, seed):
    pts = synth.points(seed, 12, (0.3, 0.9), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    return synth.hologram(pts, lam, pitch, n, n)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("geom", [(532e-9, 0.4e-6, 256, 0.5), (532e-9, 0.307e-6, 192, 0.8)])
def test_plain_full_view_vs_oracle(nf, geom):
    lam, pitch, n, z = geom
    H = _holo(lam, pitch, n, 31)
    plan = nf.Plan(lam, pitch, n, n, torch.from_numpy(H).cuda())
    f = plan.reconstruct(nf.View(z=z, kind=nf.OUT_FIELD, mode=nf.MODE_PLAIN_FRT)).cpu().numpy()
    ref, _ = oracle.reconstruct(H, lam, pitch, z, stretch=False)
    e = _rel(f, ref)
    print("plain FrT %dx%d: rel_l2 = %.3e" % (n, n, e))
    assert f.shape == ref.shape
    assert e <= TOL
    plan.close()


def test_plain_partial_view_vs_oracle_and_batch(nf):
    lam, pitch, n, z = 532e-9, 0.4e-6, 256, 0.6
    H = _holo(lam, pitch, n, 32)
    plan = nf.Plan(lam, pitch, n, n, torch.from_numpy(H).cuda())
    B = oracle.plan_view(lam, pitch, n, n, z)["width"]
    kw = dict(z=z, center_x=0.21 * B, center_y=-0.13 * B, width=0.2 * B, height=0.15 * B,
              out_nx=90, out_ny=70, kind=nf.OUT_FIELD)
    plain = nf.View(mode=nf.MODE_PLAIN_FRT, **kw)
    f = plan.reconstruct(plain).cpu().numpy()
    ref, _ = oracle.reconstruct(H, lam, pitch, z, kw["center_x"], kw["center_y"], kw["width"],
                                kw["height"], 90, 70, stretch=False)
    e = _rel(f, ref)
    print("plain FrT partial view: rel_l2 = %.3e" % e)
    assert e <= TOL
    # plain and NU-FDS views mixed in one batch: bitwise the single-view results
    views = [plain, nf.View(**kw), nf.View(z=z, mode=nf.MODE_PLAIN_FRT), nf.View(z=z)]
    singles = [plan.reconstruct(v).clone() for v in views]
    outs = [plan.output_like(v) for v in views]
    st = nf.reconstruct_batch([plan] * len(views), views, outs)
    torch.cuda.synchronize()
    assert st == [0] * len(views)
    for a, b in zip(outs, singles):
        assert torch.equal(a, b)
    plan.close()
