"""Focal sweep: views of one hologram at several depths share the stretched
band (m is independent of z, Section 4) and give exactly the single-view
results; the band is recomputed when a view changes it."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


LAM, PITCH, N = 532e-9, 0.307e-6, 512
DEPTHS = [0.45, 0.7, 1.2, 2.5]


def _holo():
    pts = synth.points(77, 16, (0.4, 2.6), synth.tan_half_fov(LAM, PITCH), (0.5, 1.0))
    return synth.hologram(pts, LAM, PITCH, N, N)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_sweep_equals_single_views_and_stretches_once(nf, prec):
    H = torch.from_numpy(_holo()).cuda()
    p = {"fp32": nf.FP32, "fp16": nf.FP16_STORE}[prec]
    plan = nf.Plan(LAM, PITCH, N, N, H, precision=p)
    views = [nf.View(z=z, kind=nf.OUT_FIELD) for z in DEPTHS]
    bands = {tuple(plan.view_plan(v)[k] for k in ("k_lo_x", "k_hi_x", "k_lo_y", "k_hi_y",
                                                  "np_x", "np_y")) for v in views}
    assert len(bands) == 1  # full views at these depths share one band
    ref = [plan.reconstruct(v).clone() for v in views]
    plan.profile(True)
    outs, st = plan.reconstruct_sweep(views)
    torch.cuda.synchronize()
    stats = {s["name"]: s for s in plan.profile_read()}
    plan.profile(False)
    assert st == [0] * len(views)
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    assert stats["stretch"]["launches"] == 1
    assert stats["view_rows_x"]["launches"] == len(views)
    plan.close()


def test_sweep_with_a_partial_view_recomputes_the_band(nf):
    H = torch.from_numpy(_holo()).cuda()
    plan = nf.Plan(LAM, PITCH, N, N, H)
    full = plan.view_plan(nf.View(z=0.7))
    p = full["width_m"] / N
    part = nf.View(z=0.7, center_x=(400 - N / 2) * p, center_y=(130 - N / 2) * p, width=96 * p,
                   height=64 * p, out_nx=96, out_ny=64)
    views = [nf.View(z=0.7), part, nf.View(z=1.2), nf.View(z=2.5)]
    ref = [plan.reconstruct(v).clone() for v in views]
    plan.profile(True)
    outs, st = plan.reconstruct_sweep(views)
    torch.cuda.synchronize()
    stats = {s["name"]: s for s in plan.profile_read()}
    plan.profile(False)
    assert st == [0, 0, 0, 0]
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    # full, partial (new band), full again (new band), full (same band)
    assert stats["stretch"]["launches"] == 3
    plan.close()


def test_sweep_depth_against_oracle(nf):
    Hn = _holo()
    plan = nf.Plan(LAM, PITCH, N, N, torch.from_numpy(Hn).cuda())
    views = [nf.View(z=z, kind=nf.OUT_FIELD) for z in DEPTHS]
    outs, st = plan.reconstruct_sweep(views)
    torch.cuda.synchronize()
    assert st == [0] * len(views)
    for k in (1, 3):
        ref, _ = oracle.reconstruct(Hn, LAM, PITCH, DEPTHS[k])
        got = outs[k].cpu().numpy()
        e = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        print("z = %.2f m: rel_l2 = %.3e" % (DEPTHS[k], e))
        assert e <= 1e-5
    plan.close()


def test_plans_of_one_geometry_share_tables(nf):
    """The FP64 tables are shared by plans of one geometry and map function:
    results are unchanged when a sibling plan is created or destroyed, and a
    plan with the polynomial surrogate keeps its own tables."""
    H = torch.from_numpy(_holo()).cuda()
    v = nf.View(z=0.7, kind=nf.OUT_FIELD)
    a = nf.Plan(LAM, PITCH, N, N, H)
    ref = a.reconstruct(v).clone()
    b = nf.Plan(LAM, PITCH, N, N, H)
    poly = nf.Plan(LAM, PITCH, N, N, H, flags=nf.FLAG_PAPER_POLY_M)
    assert torch.equal(b.reconstruct(v), ref)
    assert not torch.equal(poly.reconstruct(v), ref)
    a.close()
    assert torch.equal(b.reconstruct(v), ref)
    b.close()
    c = nf.Plan(LAM, PITCH, N, N, H)
    assert torch.equal(c.reconstruct(v), ref)
    torch.cuda.synchronize()
    c.close()
    poly.close()
