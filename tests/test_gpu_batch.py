"""Batched reconstruction: many views of several plans (uneven sizes, both
output kinds, on- and off-lattice) in one call, run as per-stage batched
kernels inside a CUDA graph.  Each result must equal the same view computed
alone (the arithmetic per element is the same; bitwise equality is expected),
a failing view must not affect the others, and a repeated batch (graph
replay) must give the same results."""
import numpy as np
import pytest

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


def _holo(n, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy((rng.standard_normal((n, n)) +
                             1j * rng.standard_normal((n, n))).astype(np.complex64)).cuda()


def _views(nf, plan, z, seed):
    info = plan.view_plan(nf.View(z=z))
    p = info["pitch_out_x_m"]
    n = plan.nx
    rng = np.random.default_rng(seed)
    out = [nf.View(z=z), nf.View(z=z, kind=nf.OUT_FIELD)]
    for k in range(3):
        s = int(rng.integers(16, n // 2))
        cx = int(rng.integers(-(n - s) // 2, (n - s) // 2))
        out.append(nf.View(z=z, center_x=cx * p, center_y=-cx * p / 2, width=s * p, height=s * p,
                           out_nx=s, out_ny=s, kind=k % 2))
    out.append(nf.View(z=z * 1.1, center_x=0.13 * n * p, width=0.3 * n * p, height=0.2 * n * p,
                       out_nx=40, out_ny=24, kind=nf.OUT_FIELD))
    return out


def test_batch_equals_single_views(nf):
    specs = [(128, 532e-9, 0.4e-6, 0.6e-3), (256, 532e-9, 0.35e-6, 0.8e-3), (192, 640e-9, 0.5e-6, 1e-3)]
    plans, views, outs, refs = [], [], [], []
    for i, (n, lam, pitch, z) in enumerate(specs):
        pl = nf.Plan(lam, pitch, n, n, _holo(n, i))
        for v in _views(nf, pl, z, i):
            plans.append(pl)
            views.append(v)
            refs.append(pl.reconstruct(v).cpu().numpy())
            outs.append(pl.output_like(v).fill_(float("nan")) if v.kind == nf.OUT_INTENSITY
                        else pl.output_like(v))
    # an invalid view in the middle
    bad = nf.View(z=0.0)
    plans.insert(5, plans[0])
    views.insert(5, bad)
    outs.insert(5, plans[0].output_like(nf.View(z=1e-3)))
    refs.insert(5, None)
    for rep in range(2):  # second call replays the cached graph
        st = nf.reconstruct_batch(plans, views, outs)
        torch.cuda.synchronize()
        assert st[5] == nf.EINVAL
        for k, (o, r) in enumerate(zip(outs, refs)):
            if r is None:
                continue
            assert st[k] == nf.OK
            got = o.cpu().numpy()
            assert np.array_equal(got, r), (k, float(np.abs(got - r).max()))
    for p in {id(p): p for p in plans}.values():
        p.close()


def test_batch_mixed_precisions(nf):
    n, lam, pitch, z = 128, 532e-9, 0.4e-6, 0.6e-3
    h = _holo(n, 7)
    pl32 = nf.Plan(lam, pitch, n, n, h)
    pl16 = nf.Plan(lam, pitch, n, n, h, precision=nf.FP16_STORE)
    v = nf.View(z=z, kind=nf.OUT_FIELD)
    r32 = pl32.reconstruct(v).cpu().numpy()
    r16 = pl16.reconstruct(v).cpu().numpy()
    o32, o16 = pl32.output_like(v), pl16.output_like(v)
    st = nf.reconstruct_batch([pl32, pl16], [v, v], [o32, o16])
    torch.cuda.synchronize()
    assert st == [nf.OK, nf.OK]
    assert np.array_equal(o32.cpu().numpy(), r32)
    assert np.array_equal(o16.cpu().numpy(), r16)
    pl32.close()
    pl16.close()


def test_batch_views_match_oracle(nf):
    """A mixed batch (three holograms, full and partial views, on and off the
    full view's lattice, field and intensity) against the FP64 oracle view by
    view: field within 1e-5, intensity within 3e-5 (relative L2)."""
    import oracle
    specs = [(128, 532e-9, 0.4e-6, 0.6e-3), (256, 532e-9, 0.35e-6, 0.8e-3), (192, 640e-9, 0.5e-6, 1e-3)]
    plans, views, outs, cases = [], [], [], []
    for i, (n, lam, pitch, z) in enumerate(specs):
        rng = np.random.default_rng(40 + i)
        H = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
        pl = nf.Plan(lam, pitch, n, n, torch.from_numpy(H).cuda())
        for v in _views(nf, pl, z, 40 + i)[1:5]:
            plans.append(pl)
            views.append(v)
            outs.append(pl.output_like(v))
            cases.append((H, lam, pitch, v))
    st = nf.reconstruct_batch(plans, views, outs)
    torch.cuda.synchronize()
    assert all(s == 0 for s in st), st
    worst = 0.0
    for o, (H, lam, pitch, v) in zip(outs, cases):
        f, I = oracle.reconstruct(H, lam, pitch, v.z, v.center_x, v.center_y, v.width, v.height,
                                  v.out_nx, v.out_ny)
        got = o.cpu().numpy()
        ref = f if v.kind == nf.OUT_FIELD else I
        e = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        worst = max(worst, e)
        assert e <= (1e-5 if v.kind == nf.OUT_FIELD else 3e-5), (v, e)
    print("batch vs oracle: worst rel_l2 %.3e over %d views" % (worst, len(outs)))
    for p in {id(p): p for p in plans}.values():
        p.close()


def test_batches_on_many_streams_keep_a_bounded_workspace(nf):
    """Batches on ten successive new streams: the results stay bitwise equal,
    and the device memory held afterwards is bounded by the library's four
    retained batch workspaces per device, not one per stream ever used."""
    n, lam, pitch, z = 256, 532e-9, 0.35e-6, 0.8e-3
    pl = nf.Plan(lam, pitch, n, n, _holo(n, 11))
    views = _views(nf, pl, z, 11)
    outs = [pl.output_like(v) for v in views]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s0 = torch.cuda.Stream()
    assert all(c == nf.OK for c in nf.reconstruct_batch([pl] * len(views), views, outs, stream=s0))
    torch.cuda.synchronize()
    ref = [o.cpu().numpy() for o in outs]
    per = free0 - torch.cuda.mem_get_info()[0]     # one stream's batch workspace
    streams = [s0]
    for _ in range(10):
        s = torch.cuda.Stream()
        streams.append(s)
        for o in outs:
            o.zero_()
        torch.cuda.synchronize()
        assert all(c == nf.OK for c in nf.reconstruct_batch([pl] * len(views), views, outs, stream=s))
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    held = free0 - torch.cuda.mem_get_info()[0]
    print("one workspace %.1f MB, held after 11 streams %.1f MB" % (per / 2**20, held / 2**20))
    assert per > 0 and held <= 4 * per + (64 << 20), (per, held)
    pl.close()
