"""HostPipeline: host-resident holograms through one plan with the copies
overlapped gives, step for step, exactly the views of direct calls."""
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


@pytest.mark.parametrize("kind", ["intensity", "field"])
def test_pipeline_matches_direct_calls(nf, kind):
    import synth
    from paper_2410_13474_gb300.pipeline import HostPipeline
    from synth.configs import SMALL_512 as w
    n = w.n
    holos = []
    for s in range(3):
        pts = synth.points(100 + s, 12, w.z_range, w.tan_half)
        holos.append(torch.from_numpy(synth.hologram(pts, w.wavelength, w.pitch, n, n)).pin_memory())
    view = nf.View(z=w.z_view, kind=nf.OUT_INTENSITY if kind == "intensity" else nf.OUT_FIELD)
    plan = nf.Plan(w.wavelength, w.pitch, n, n)
    ref = []
    for h in holos:
        plan.load(h.cuda())
        ref.append(plan.reconstruct(view).cpu())
    order = [0, 1, 2, 1, 0, 2, 2]
    outs = [torch.empty(ref[0].shape, dtype=ref[0].dtype).pin_memory() for _ in order]
    pipe = HostPipeline(plan, view)
    pipe.begin()
    for i, k in enumerate(order):
        pipe.submit(holos[k], outs[i])
    pipe.drain()
    torch.cuda.synchronize()
    for i, k in enumerate(order):
        assert torch.equal(outs[i], ref[k]), (i, k)
    plan.close()
