"""The allocation-free entry point, checked against the allocating one.

nufds_reconstruct_noalloc serves callers that must not allocate device
memory (their memory is reserved by another allocator, or they cannot take
cudaFree's device-wide synchronisation); it keeps all working memory in a
static device array.  Called through the C ABI twice in a row, it must give
the same field as nufds_plan_create + nufds_reconstruct, within the tolerance
of the other parity tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

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
    L = m.lib()
    L.nufds_reconstruct_noalloc.argtypes = [ctypes.POINTER(m._Params), ctypes.POINTER(m._View),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.nufds_reconstruct_noalloc.restype = ctypes.c_int
    return m


def _noalloc(m, H, lam, pitch, view):
    ny, nx = H.shape
    prm = m._Params(lam, pitch, nx, ny, m.FP32, 0, 0)
    v = view._c()
    dt = torch.float32 if view.kind == m.OUT_INTENSITY else torch.complex64
    info = m.view_plan(lam, pitch, nx, ny, view)
    out = torch.full((info["out_ny"], info["out_nx"]), float("nan"), dtype=dt, device="cuda")
    st = torch.cuda.current_stream()
    rc = m.lib().nufds_reconstruct_noalloc(ctypes.byref(prm), ctypes.byref(v),
                                           ctypes.c_void_p(H.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(st.cuda_stream))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


CASES = [
    (128, 128, 532e-9, 0.4e-6, dict(z=0.6e-3)),
    (96, 64, 532e-9, 0.307e-6, dict(z=0.3e-3)),
    (128, 128, 532e-9, 0.4e-6, dict(z=0.6e-3, center_x=1.1e-5, center_y=-2.3e-5, width=6e-5,
                                     height=4e-5, out_nx=50, out_ny=30)),
]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_plan_path_twice(nf, case):
    ny, nx, lam, pitch, kw = case
    rng = np.random.default_rng(nx + ny)
    H = torch.from_numpy((rng.standard_normal((ny, nx)) +
                          1j * rng.standard_normal((ny, nx))).astype(np.complex64)).cuda()
    for kind in (nf.OUT_FIELD, nf.OUT_INTENSITY):
        view = nf.View(kind=kind, **kw)
        plan = nf.Plan(lam, pitch, nx, ny, H)
        ref = plan.reconstruct(view).cpu().numpy()
        plan.close()
        for _ in range(2):
            rc, got = _noalloc(nf, H, lam, pitch, view)
            assert rc == nf.OK, nf.status_string(rc)
            assert _rel(got, ref) <= TOL


def test_noalloc_rejects_sizes_beyond_its_maximum(nf):
    H = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
    rc, _ = _noalloc(nf, H, 532e-9, 0.4e-6, nf.View(z=1e-3))
    assert rc == nf.EUNSUPPORTED


def test_noalloc_allocates_no_device_memory(nf):
    """Repeated calls leave the device's free memory unchanged (cudaMemGetInfo):
    the library allocates nothing on this path.  Outputs are allocated up
    front, and one warm-up round loads the kernels' code first (lazy module
    loading takes device memory on a kernel's first launch)."""
    jobs = []
    for k, (ny, nx, lam, pitch, kw) in enumerate(CASES):
        rng = np.random.default_rng(100 + k)
        H = torch.from_numpy((rng.standard_normal((ny, nx)) +
                              1j * rng.standard_normal((ny, nx))).astype(np.complex64)).cuda()
        for kind in (nf.OUT_FIELD, nf.OUT_INTENSITY):
            view = nf.View(kind=kind, **kw)
            info = nf.view_plan(lam, pitch, nx, ny, view)
            dt = torch.float32 if kind == nf.OUT_INTENSITY else torch.complex64
            out = torch.empty((info["out_ny"], info["out_nx"]), dtype=dt, device="cuda")
            jobs.append((nf._Params(lam, pitch, nx, ny, nf.FP32, 0, 0), view._c(), H, out))
    st = torch.cuda.current_stream()

    def run_all():
        for prm, v, H, out in jobs:
            rc = nf.lib().nufds_reconstruct_noalloc(ctypes.byref(prm), ctypes.byref(v),
                                                    ctypes.c_void_p(H.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    ctypes.c_void_p(st.cuda_stream))
            assert rc == nf.OK, nf.status_string(rc)
        torch.cuda.synchronize()

    run_all()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        run_all()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
