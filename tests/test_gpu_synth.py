"""The GPU point-cloud generator (input making for large workloads) against
the exact FP64 host sum of Eq. 3 on sampled pixels."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_gpu_generator_matches_fp64_sum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lam, pitch, n = 532e-9, 0.307e-6, 1024
    pts = synth.points(99, 300, (2e-3, 10e-3), synth.tan_half_fov(lam, pitch), (0.5, 1.0))
    g = synth.gpu_hologram(pts, lam, pitch, n, n).cpu().numpy()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, size=(200, 2))
    idx[:4] = [[0, 0], [n - 1, n - 1], [0, n - 1], [511, 512]]
    ref = np.array([synth.sample(pts, lam, pitch, n, n, int(i), int(j)) for i, j in idx])
    got = g[idx[:, 1], idx[:, 0]]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 2e-5, err
