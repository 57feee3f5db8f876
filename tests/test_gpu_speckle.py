"""Speckle averaging (Section 5): the mean intensity over CGHs of one point
cloud with independent random phases, accumulated in place on the GPU."""
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


def test_accumulated_mean_intensity(nf):
    lam, pitch, n, z, K = 532e-9, 0.4e-6, 256, 0.5, 4
    pts = synth.points(91, 24, (0.4, 0.6), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    phases = synth.uniform(92, K * len(pts)).reshape(K, len(pts)) * 2 * np.pi
    holos = []
    for k in range(K):
        p = pts.copy()
        p[:, 4] = phases[k]
        holos.append(synth.hologram(p, lam, pitch, n, n))
    plan = nf.Plan(lam, pitch, n, n)
    acc = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    singles = []
    for H in holos:
        plan.load(torch.from_numpy(H).cuda())
        plan.reconstruct(nf.View(z=z, kind=nf.OUT_INTENSITY_ACCUM), acc)
        singles.append(plan.reconstruct(nf.View(z=z)).clone())
    torch.cuda.synchronize()
    # in place accumulation = the same float32 sum in the same order
    s = singles[0]
    for t in singles[1:]:
        s = s + t
    assert torch.equal(acc, s)
    mean = (acc / K).cpu().numpy().astype(np.float64)
    ref = np.mean([oracle.reconstruct(H, lam, pitch, z)[1] for H in holos], axis=0)
    e = float(np.linalg.norm(mean - ref) / np.linalg.norm(ref))
    print("mean intensity over %d CGHs: rel_l2 = %.3e" % (K, e))
    assert e <= 3e-5
    plan.close()
