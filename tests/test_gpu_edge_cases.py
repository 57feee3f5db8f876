"""Edge cases and error paths of the C ABI on the GPU: the smallest hologram,
one-pixel views, empty batches and sweeps, per-view statuses in a batch, and
the EINVAL / ENOMEM / EUNSUPPORTED returns."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM, PITCH = 532e-9, 0.4e-6


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
    return (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_smallest_hologram_and_one_pixel_view(nf):
    with pytest.raises(nf.NufdsError) as e:            # below the smallest row FFT
        nf.Plan(LAM, PITCH, 60, 60)
    assert e.value.code == nf.EUNSUPPORTED
    n, z = 64, 0.3
    H = _holo(n, 1)
    plan = nf.Plan(LAM, PITCH, n, n, torch.from_numpy(H).cuda())
    f = plan.reconstruct(nf.View(z=z, kind=nf.OUT_FIELD)).cpu().numpy()
    ref, _ = oracle.reconstruct(H, LAM, PITCH, z)
    assert _rel(f, ref) <= 1e-5
    B = oracle.plan_view(LAM, PITCH, n, n, z)["width"]
    kw = dict(z=z, center_x=0.11 * B, center_y=-0.2 * B, width=B / n, height=B / n, out_nx=1,
              out_ny=1)
    f1 = plan.reconstruct(nf.View(kind=nf.OUT_FIELD, **kw)).cpu().numpy()
    r1, _ = oracle.reconstruct(H, LAM, PITCH, kw["z"], kw["center_x"], kw["center_y"],
                               kw["width"], kw["height"], 1, 1)
    assert f1.shape == (1, 1) and _rel(f1, r1) <= 1e-5
    plan.close()


def test_error_returns(nf):
    n = 64
    h = torch.from_numpy(_holo(n, 2)).cuda()
    with pytest.raises(nf.NufdsError) as e:
        nf.Plan(LAM, PITCH, 62, 64)                    # not a multiple of 4
    assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError) as e:
        nf.Plan(LAM, PITCH, n, n, h, budget=1 << 16)   # tables alone exceed the budget
    assert e.value.code == nf.ENOMEM
    with pytest.raises(nf.NufdsError) as e:
        nf.Plan(0.9e-6, PITCH, n, n)                   # lambda >= 2 pitch (Eq. 1)
    assert e.value.code == nf.EINVAL
    plan = nf.Plan(LAM, PITCH, n, n)                   # no hologram yet
    with pytest.raises(nf.NufdsError) as e:
        plan.reconstruct(nf.View(z=0.3))
    assert e.value.code == nf.EINVAL
    plan.load(h)
    B = oracle.plan_view(LAM, PITCH, n, n, 0.3)["width"]
    with pytest.raises(nf.NufdsError) as e:             # band beyond the full view's
        plan.reconstruct(nf.View(z=0.3, center_x=3 * B, width=B / 4, height=B / 4, out_nx=16,
                                 out_ny=16))
    assert e.value.code == nf.EUNSUPPORTED
    plan.close()


def test_batch_statuses_and_empty_calls(nf):
    n, z = 64, 0.3
    h = torch.from_numpy(_holo(n, 3)).cuda()
    good = nf.Plan(LAM, PITCH, n, n, h)
    empty = nf.Plan(LAM, PITCH, n, n)                  # not loaded
    B = oracle.plan_view(LAM, PITCH, n, n, z)["width"]
    views = [nf.View(z=z), nf.View(z=z), nf.View(z=-1.0),
             nf.View(z=z, center_x=3 * B, width=B / 4, height=B / 4, out_nx=16, out_ny=16),
             nf.View(z=1.5 * z)]
    plans = [good, empty, good, good, good]
    outs = [torch.zeros((n, n), dtype=torch.float32, device="cuda") for _ in views[:2]]
    outs += [torch.zeros((16, 16), dtype=torch.float32, device="cuda") for _ in views[2:4]]
    outs += [torch.zeros((n, n), dtype=torch.float32, device="cuda")]
    st = nf.reconstruct_batch(plans, views, outs)
    torch.cuda.synchronize()
    assert st == [0, nf.EINVAL, nf.EINVAL, nf.EUNSUPPORTED, 0]
    assert torch.equal(outs[0], good.reconstruct(views[0]))
    assert torch.equal(outs[4], good.reconstruct(views[4]))
    assert nf.reconstruct_batch([], [], []) == []
    o, s = good.reconstruct_sweep([])
    assert o == [] and s == []
    good.close()
    empty.close()
