"""The debug library (libnufds_bc.so: both gathers compiled with
NUFDS_BOUNDS_CHECK) on a set of small reconstructions that reach every
gather form: full and partial views on and off the lattice, views whose
windows wrap around the periodic spectrum, FP32/FP16/BF16 storage, the
paper-literal bilinear variant, the plain Fresnel transform, a batch and a
sweep.  None may record a read outside its row or table, and each result
must equal the product library's (the checks skip nothing when every read
is inside, so the arithmetic is the same).

The debug library runs in a child process (NUFDS_BOUNDS_CHECK=1 selects it
at import); the product library's results come from this process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import json, sys
import numpy as np
import torch
import paper_2410_13474_gb300 as nf


def holo(n, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy((rng.standard_normal((n, n)) +
                             1j * rng.standard_normal((n, n))).astype(np.complex64)).cuda()


def run():
    """name -> output array for every case (same list in both processes)."""
    res = {}
    lam, pitch, n, z = 532e-9, 0.4e-6, 128, 0.5e-3
    for prec, pname in ((nf.FP32, "fp32"), (nf.FP16_STORE, "fp16"), (nf.BF16_STORE, "bf16")):
        pl = nf.Plan(lam, pitch, n, n, holo(n, 1), precision=prec)
        p = pl.view_plan(nf.View(z=z))["pitch_out_x_m"]
        views = {
            "full": nf.View(z=z, kind=nf.OUT_FIELD),
            "lattice": nf.View(z=z, center_x=20 * p, center_y=-12 * p, width=40 * p, height=24 * p,
                               out_nx=40, out_ny=24, kind=nf.OUT_FIELD),
            "offlattice": nf.View(z=1.3 * z, center_x=0.21 * n * p, center_y=0.3 * n * p,
                                  width=0.5 * n * p, height=0.3 * n * p, out_nx=48, out_ny=20,
                                  kind=nf.OUT_FIELD),
            # a view at the edge of the full window: its band reaches the
            # spectrum's Nyquist edge, where gather windows wrap
            "edge": nf.View(z=z, center_x=(n / 2 - 8) * p, center_y=-(n / 2 - 8) * p,
                            width=16 * p, height=16 * p, out_nx=16, out_ny=16, kind=nf.OUT_FIELD),
            "plain": nf.View(z=z, mode=nf.MODE_PLAIN_FRT, kind=nf.OUT_FIELD),
        }
        for k, v in views.items():
            res["%s_%s" % (pname, k)] = pl.reconstruct(v)
        vs = [nf.View(z=z * (1 + 0.1 * i), kind=nf.OUT_FIELD) for i in range(3)]
        souts, sst = pl.reconstruct_sweep(vs)
        assert all(s == 0 for s in sst), sst
        for i, o in enumerate(souts):
            res["%s_sweep%d" % (pname, i)] = o
        pl2 = nf.Plan(640e-9, 0.5e-6, 96, 96, holo(96, 2), precision=prec)
        bv = [views["offlattice"], nf.View(z=0.8e-3, kind=nf.OUT_FIELD), views["edge"]]
        bp = [pl, pl2, pl]
        outs = [q.output_like(v) for q, v in zip(bp, bv)]
        st = nf.reconstruct_batch(bp, bv, outs)
        assert all(s == 0 for s in st), st
        for i, o in enumerate(outs):
            res["%s_batch%d" % (pname, i)] = o
    pl = nf.Plan(lam, pitch, n, n, holo(n, 3), flags=nf.FLAG_PAPER_LINEAR | nf.FLAG_PAPER_POLY_M)
    p = pl.view_plan(nf.View(z=z))["pitch_out_x_m"]
    res["linear_full"] = pl.reconstruct(nf.View(z=z, kind=nf.OUT_FIELD))
    res["linear_off"] = pl.reconstruct(nf.View(z=z, center_x=0.3 * n * p, width=0.4 * n * p,
                                               height=0.4 * n * p, out_nx=30, out_ny=30,
                                               kind=nf.OUT_FIELD))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in res.items()}


if __name__ == "__main__":
    out = run()
    n, first = nf.bounds_violations(reset=True)
    np.savez(sys.argv[1], **out)
    print(json.dumps({"violations": n, "first": first}))
'''


@pytest.fixture(scope="module")
def nf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_13474_gb300 import build
    build.build()
    build.build(bounds_check=True)
    import paper_2410_13474_gb300 as m
    return m


def test_product_library_reports_no_checks(nf):
    with pytest.raises(nf.NufdsError) as e:
        nf.bounds_violations()
    assert e.value.code == -3


def test_bounds_checked_gathers_read_inside(nf, tmp_path):
    script = tmp_path / "cases.py"
    script.write_text(CASES)
    npz = tmp_path / "bc.npz"
    env = dict(os.environ, NUFDS_BOUNDS_CHECK="1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, str(script), str(npz)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    print("debug library:", rep)
    assert rep["violations"] == 0, rep
    got = np.load(npz)
    ns = {"__name__": "cases"}
    exec(compile(CASES, "cases", "exec"), ns)
    ref = ns["run"]()
    assert set(ref) == set(got.files)
    worst, equal = 0.0, 0
    for k, v in ref.items():
        g = got[k]
        e = float(np.linalg.norm(g - v) / max(np.linalg.norm(v), 1e-30))
        worst = max(worst, e)
        equal += int(np.array_equal(g, v))
        assert e <= 1e-6, (k, e)
    print("%d of %d outputs bitwise equal, worst rel_l2 %.2e" % (equal, len(ref), worst))
