"""FP64 CPU oracle for the NU-FDS reconstruction path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never loads it.
``build()`` compiles ``nufds_oracle.c`` (plain C11 + OpenMP, FP64) with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)
_d = ctypes.c_double
_i = ctypes.c_int


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "nufds_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.or_fft.argtypes = [_dp, _i, _i]
            L.or_centred_dft2.argtypes = [_dp, _i, _i, _i]
            L.or_hyp2f1.argtypes = [_d]
            L.or_hyp2f1.restype = _d
            L.or_mag.argtypes = [_d, _d, _d, _dp, _dp]
            L.or_forward.argtypes = [_d, _d, _d, _dp, _dp]
            L.or_pullback.argtypes = [_d, _d, _d, _d, _dp, _dp]
            L.or_pullback.restype = _i
            L.or_output_map.argtypes = [_d, _d, _d, _d, _dp, _dp]
            L.or_output_map_iterative_inverse.argtypes = [_d, _d, _d, _d, _i, _dp, _dp]
            L.or_ps_tools.argtypes = [_d, _d, _d, _d, _dp, _dp]
            L.or_lerp2.argtypes = [_dp, _i, _i, _dp, _dp, ctypes.c_int64, _dp]
            L.or_set_paper_linear.argtypes = [_i]
            L.or_wavefront_error.argtypes = [_d, _d, _i, _d, _d, _d, _i, _d, _i, _dp, _dp]
            L.or_wavefront_error.restype = _d
            L.or_nice.argtypes = [ctypes.c_int64]
            L.or_nice.restype = ctypes.c_int64
            L.or_plan_view_ex.argtypes = [_d, _d, _i, _i, _d, _d, _d, _d, _d, _i, _i, _i, _i64p,
                                          _dp]
            L.or_plan_view_ex.restype = _i
            L.or_dtft2_direct.argtypes = [_dp, _i, _i, _dp, _dp, ctypes.c_int64, _dp]
            L.or_nufft2.argtypes = [_dp, _i, _i, _dp, _dp, ctypes.c_int64, _dp]
            L.or_reconstruct.argtypes = [_d, _d, _i, _i, _fp, _d, _d, _d, _d, _d, _i, _i, _i, _i,
                                         _dp, _dp]
            L.or_reconstruct.restype = _i
            L.or_reconstruct_views.argtypes = [_d, _d, _i, _i, _fp, _i, _dp, _dp, _dp, _dp, _dp,
                                               ctypes.POINTER(_i), ctypes.POINTER(_i), _i, _i,
                                               ctypes.POINTER(_dp), ctypes.POINTER(_dp)]
            L.or_reconstruct_views.restype = _i
            L.or_num_threads.restype = _i
            L.or_set_paper_poly.argtypes = [_i, _d, _d, _dp]
            L.or_set_paper_poly.restype = None
            _lib = L
    return _lib


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, np.complex128).copy()
    lib().or_fft(_ptr(a), a.size, sign)
    return a


def centred_dft2(a: np.ndarray, sign: int = -1) -> np.ndarray:
    b = np.ascontiguousarray(a, np.complex128).copy()
    ny, nx = b.shape
    lib().or_centred_dft2(_ptr(b), nx, ny, sign)
    return b


def hyp2f1(w: float) -> float:
    return lib().or_hyp2f1(float(w))


def _pair(fn, *args):
    a, b = _d(), _d()
    r = fn(*[float(x) for x in args], ctypes.byref(a), ctypes.byref(b))
    return r, a.value, b.value


def mag(lam, fx, fy):
    return _pair(lib().or_mag, lam, fx, fy)[1:]


def forward(lam, fx, fy):
    return _pair(lib().or_forward, lam, fx, fy)[1:]


def pullback(lam, pitch, fpx, fpy):
    ok, fx, fy = _pair(lib().or_pullback, lam, pitch, fpx, fpy)
    return (fx, fy) if ok else None


def output_map(lam, z, xo, yo):
    return _pair(lib().or_output_map, lam, z, xo, yo)[1:]


def output_map_iterative_inverse(lam, z, xop, yop, steps):
    a, b = _d(), _d()
    lib().or_output_map_iterative_inverse(lam, z, xop, yop, int(steps), ctypes.byref(a),
                                          ctypes.byref(b))
    return a.value, b.value


def ps_tools(lam, xo, yo, zo):
    return _pair(lib().or_ps_tools, lam, xo, yo, zo)[1:]


def wavefront_error(lam, pitch, n, xo, yo, zo, method="nufds", z_r=0.0, samples=1025):
    """Wavefront error (waves) along the hologram's central row: returns
    (x, W, max|W|); method "nufds" (Eq. 17 focus at z_o) or "frt" (plain
    Fresnel transform at z_r, z_o when z_r <= 0)."""
    x = np.zeros(samples)
    w = np.zeros(samples)
    m = {"nufds": 0, "frt": 1}[method]
    mx = lib().or_wavefront_error(lam, pitch, int(n), xo, yo, zo, m, z_r, int(samples),
                                  x.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    return x, w, mx


def nice(n: int) -> int:
    return int(lib().or_nice(int(n)))


def plan_view(lam, pitch, nx, ny, z, cx=0.0, cy=0.0, w=0.0, h=0.0, ox=0, oy=0, stretch=1):
    iv = np.zeros(8, np.int64)
    dv = np.zeros(4, np.float64)
    r = lib().or_plan_view_ex(lam, pitch, nx, ny, z, cx, cy, w, h, ox, oy, stretch,
                              _ptr(iv, _i64p), _ptr(dv))
    if r:
        raise ValueError("invalid view")
    keys = ["out_nx", "out_ny", "k_lo_x", "k_hi_x", "k_lo_y", "k_hi_y", "np_x", "np_y"]
    d = {k: int(v) for k, v in zip(keys, iv)}
    d.update(pitch_out_x=dv[0], pitch_out_y=dv[1], width=dv[2], height=dv[3])
    d["k_c_x"] = (d["k_lo_x"] + d["k_hi_x"]) // 2
    d["k_c_y"] = (d["k_lo_y"] + d["k_hi_y"]) // 2
    return d


def _targets(tx, ty):
    tx = np.ascontiguousarray(tx, np.float64).ravel()
    ty = np.ascontiguousarray(ty, np.float64).ravel()
    assert tx.size == ty.size
    return tx, ty


def dtft2_direct(c: np.ndarray, tx, ty) -> np.ndarray:
    c = np.ascontiguousarray(c, np.complex128)
    tx, ty = _targets(tx, ty)
    out = np.empty(tx.size, np.complex128)
    ny, nx = c.shape
    lib().or_dtft2_direct(_ptr(c), nx, ny, _ptr(tx), _ptr(ty), tx.size, _ptr(out))
    return out


def nufft2(c: np.ndarray, tx, ty) -> np.ndarray:
    c = np.ascontiguousarray(c, np.complex128)
    tx, ty = _targets(tx, ty)
    out = np.empty(tx.size, np.complex128)
    ny, nx = c.shape
    lib().or_nufft2(_ptr(c), nx, ny, _ptr(tx), _ptr(ty), tx.size, _ptr(out))
    return out


def lerp2(c: np.ndarray, tx, ty) -> np.ndarray:
    """Bilinear interpolation of the grid values of the trigonometric polynomial
    of nufft2 (its centred DFT), periodic: the paper-literal resampling."""
    c = np.ascontiguousarray(c, np.complex128)
    tx, ty = _targets(tx, ty)
    out = np.empty(tx.size, np.complex128)
    ny, nx = c.shape
    lib().or_lerp2(_ptr(c), nx, ny, _ptr(tx), _ptr(ty), tx.size, _ptr(out))
    return out


def reconstruct(holo: np.ndarray, wavelength: float, pitch: float, z: float, cx=0.0, cy=0.0,
                w=0.0, h=0.0, ox=0, oy=0, stretch=True, threads=0):
    """FP64 NU-FDS reconstruction of a complex64 hologram; returns (field, intensity)."""
    holo = np.ascontiguousarray(holo, np.complex64)
    ny, nx = holo.shape
    plan = plan_view(wavelength, pitch, nx, ny, z, cx, cy, w, h, ox, oy, int(stretch))
    field = np.empty((plan["out_ny"], plan["out_nx"]), np.complex128)
    inten = np.empty((plan["out_ny"], plan["out_nx"]), np.float64)
    r = lib().or_reconstruct(wavelength, pitch, nx, ny, _ptr(holo, _fp), z, cx, cy, w, h, ox, oy,
                             int(stretch), int(threads), _ptr(field), _ptr(inten))
    if r:
        raise ValueError("invalid view")
    return field, inten


def reconstruct_views(holo: np.ndarray, wavelength: float, pitch: float, views, stretch=True,
                      threads=0):
    """Several views of one hologram, each a dict(z, cx, cy, w, h, ox, oy) as the
    arguments of reconstruct; returns a list of (field, intensity).  Same
    results as one reconstruct call per view; step two's gridded transform of
    the hologram is shared."""
    holo = np.ascontiguousarray(holo, np.complex64)
    ny, nx = holo.shape
    nv = len(views)
    cols = {k: np.array([float(v.get(k, 0.0)) for v in views]) for k in ("z", "cx", "cy", "w", "h")}
    oxs = (_i * nv)(*[int(v.get("ox", 0)) for v in views])
    oys = (_i * nv)(*[int(v.get("oy", 0)) for v in views])
    outs = []
    for v in views:
        p = plan_view(wavelength, pitch, nx, ny, v["z"], v.get("cx", 0.0), v.get("cy", 0.0),
                      v.get("w", 0.0), v.get("h", 0.0), v.get("ox", 0), v.get("oy", 0),
                      int(stretch))
        outs.append((np.empty((p["out_ny"], p["out_nx"]), np.complex128),
                     np.empty((p["out_ny"], p["out_nx"]), np.float64)))
    fp = (_dp * nv)(*[_ptr(f) for f, _ in outs])
    ip = (_dp * nv)(*[_ptr(i) for _, i in outs])
    r = lib().or_reconstruct_views(wavelength, pitch, nx, ny, _ptr(holo, _fp), nv,
                                   _ptr(cols["z"]), _ptr(cols["cx"]), _ptr(cols["cy"]),
                                   _ptr(cols["w"]), _ptr(cols["h"]), oxs, oys, int(stretch),
                                   int(threads), fp, ip)
    if r:
        raise ValueError("invalid view")
    return outs


class paper_poly:
    """Context: inside it, Eq. 16 uses the paper's degree-8 polynomial surrogate
    for 2F1 fitted to 51 frequencies across the band of (lam, pitch) (Section 4)
    instead of the exact function.  .coef holds its 9 coefficients (in s = lambda f)."""

    def __init__(self, lam, pitch):
        self.lam, self.pitch = lam, pitch
        self.coef = np.zeros(9)

    def __enter__(self):
        lib().or_set_paper_poly(1, self.lam, self.pitch, _ptr(self.coef))
        return self

    def __exit__(self, *exc):
        lib().or_set_paper_poly(0, 0.0, 0.0, None)
        return False


class paper_linear:
    """Context: inside it, steps two and five resample by bilinear interpolation
    on the unpadded grids (the paper-literal variant) instead of ideally."""

    def __enter__(self):
        lib().or_set_paper_linear(1)
        return self

    def __exit__(self, *exc):
        lib().or_set_paper_linear(0)
        return False


def num_threads() -> int:
    return int(lib().or_num_threads())
