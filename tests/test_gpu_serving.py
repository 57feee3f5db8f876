"""Serving on the GPU: requests arriving while others run are batched and
overlap on two streams; every result must equal the same view reconstructed
alone (bitwise: batching does not change the per-element arithmetic), and a
subset of the served results matches the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as nf
    from paper_2410_13474_gb300.serving import GpuExecutor, Request, Scheduler

    specs = [(128, 0.4e-6, 0.6e-3), (256, 0.35e-6, 0.9e-3), (192, 0.45e-6, 1.2e-3)]
    plans, holos = [], []
    rng = np.random.default_rng(5)
    for n, pitch, _ in specs:
        h = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
        holos.append(h)
        plans.append(nf.Plan(532e-9, pitch, n, n, torch.from_numpy(h).cuda()))
    reqs = []
    for i in range(48):
        k = int(rng.integers(0, 3))
        n, _, z = specs[k]
        p = plans[k].view_plan(nf.View(z=z))["pitch_out_x_m"]
        s = int(rng.integers(8, n))
        cx = int(rng.integers(-(n - s) // 2, (n - s) // 2 + 1))
        v = nf.View(z=z, center_x=cx * p, width=s * p, height=s * p, out_nx=s, out_ny=s,
                    kind=i % 2)
        reqs.append(Request(i, k, v, 0.002 * i))
    ex = GpuExecutor(plans, slots=2, keep_outputs=True)
    for r in reqs:
        r.ws_bytes = ex.workspace_bytes(r.holo, r.view)
    st = Scheduler(ex, budget_bytes=8 << 30, slots=2, max_batch=8).run(reqs)
    torch.cuda.synchronize()
    assert st.completed == 48 and st.rejected == 0
    for r in reqs:
        assert r.status == 0
        alone = plans[r.holo].reconstruct(r.view)
        assert torch.equal(alone, r.out), r.rid
    # and a subset against the FP64 oracle
    import oracle
    for r in reqs[::6]:
        n, pitch, _ = specs[r.holo]
        v = r.view
        f, I = oracle.reconstruct(holos[r.holo], 532e-9, pitch, v.z, v.center_x, v.center_y,
                                  v.width, v.height, v.out_nx, v.out_ny)
        ref = f if v.kind == nf.OUT_FIELD else I
        got = r.out.cpu().numpy()
        e = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert e <= (1e-5 if v.kind == nf.OUT_FIELD else 3e-5), (r.rid, e)
    for p in plans:
        p.close()
