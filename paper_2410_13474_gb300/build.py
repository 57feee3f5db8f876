"""Build libnufds.so (CUDA, sm_103a) in-tree with nvcc.

Each translation unit compiles in parallel to an object under _build/, then
nvcc links them into paper_2410_13474_gb300/libnufds.so.  The debug library
libnufds_bc.so (bounds-checked gathers: gather.cu compiled with
NUFDS_BOUNDS_CHECK, the other objects shared) is built on request.  Usage:
    python -m paper_2410_13474_gb300.build [--verbose-ptxas] [--bounds-check]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnufds.so")
LIB_BC = os.path.join(HERE, "libnufds_bc.so")
BC_SOURCES = ["gather.cu"]   # the translation units whose reads the debug build checks
SOURCES = ["api.cu", "fft_rows.cu", "maps.cu", "gather.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA extension cannot be built")
    return p


def _flags(ptxas_verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True,
          bounds_check: bool = False) -> str:
    """Build libnufds.so (or, with bounds_check, libnufds_bc.so) and return its path."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "nufds.h"))
    nv = nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        checked = bounds_check and s in BC_SOURCES
        obj = os.path.join(BUILD, s.replace(".cu", "_bc.o" if checked else ".o"))
        objs.append(obj)
        if force or ptxas_verbose or _stale(obj, [src] + headers):
            jobs.append([nv, "-c", src, "-o", obj] + _flags(ptxas_verbose)
                        + (["-DNUFDS_BOUNDS_CHECK"] if checked else []))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for cmd, r in ex.map(run, jobs):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stdout + r.stderr))
            if not quiet or ptxas_verbose:
                sys.stdout.write(r.stdout + r.stderr)
    lib = LIB_BC if bounds_check else LIB
    if force or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nv, "-shared"] + ARCH + ["-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s" % (r.stdout + r.stderr))
        os.replace(tmp, lib)
    return lib



def sources_digest(files=None) -> str:
    """sha256 over CUDA sources and headers (all, or the named files of csrc/):
    ties a profile to the code it measured."""
    import hashlib
    h = hashlib.sha256()
    if files is None:
        files = [f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    for f in sorted(files):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


if __name__ == "__main__":
    print(build(force=True, ptxas_verbose="--verbose-ptxas" in sys.argv, quiet=False,
                bounds_check="--bounds-check" in sys.argv))
