"""Seeded synthetic point-cloud holograms (inputs only).

This package makes the inputs that both the FP64 oracle and the CUDA path
consume.  It contains no arithmetic of the reconstruction method: only the
point-source model of Eq. 3 (a spherical wave e^{-ikR} per object point) and a
splitmix64 random stream.  ``build()`` compiles ``pointcloud.c`` with gcc.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "pointcloud.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, dp]
            lib.synth_points.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, dp]
            lib.synth_hologram_rows.argtypes = [dp, ctypes.c_int32, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, fp]
            lib.synth_sample.argtypes = [dp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, dp]
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def uniform(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().synth_uniform(seed, n, _dptr(out))
    return out


def points(seed: int, n_points: int, z_range, tan_half_fov: float, amp_range=(1.0, 1.0),
           spread: float = 1.0) -> np.ndarray:
    """Point cloud (n_points x 5: x, y, z, amplitude, phase), all in metres/radians."""
    out = np.empty((n_points, 5), np.float64)
    _load().synth_points(seed, n_points, float(z_range[0]), float(z_range[1]),
                         float(tan_half_fov), float(spread), float(amp_range[0]),
                         float(amp_range[1]), _dptr(out))
    return out


def hologram(pts: np.ndarray, wavelength: float, pitch: float, nx: int, ny: int,
             threads: int = 0, row0: int = 0, nrows: int | None = None) -> np.ndarray:
    """complex64 hologram rows [row0, row0+nrows) of shape (nrows, nx), FP64 sum."""
    pts = np.ascontiguousarray(pts, np.float64)
    nrows = ny - row0 if nrows is None else nrows
    out = np.empty((nrows, nx), np.complex64)
    _load().synth_hologram_rows(_dptr(pts), pts.shape[0], wavelength, pitch, nx, ny, row0,
                                nrows, threads,
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


def sample(pts: np.ndarray, wavelength: float, pitch: float, nx: int, ny: int, ix: int,
           iy: int) -> complex:
    pts = np.ascontiguousarray(pts, np.float64)
    out = np.empty(2, np.float64)
    _load().synth_sample(_dptr(pts), pts.shape[0], wavelength, pitch, nx, ny, ix, iy,
                         _dptr(out))
    return complex(out[0], out[1])


def tan_half_fov(wavelength: float, pitch: float) -> float:
    """tan(asin(lambda / (2 pitch))): half-angle of the grating-equation FoV (Eq. 1)."""
    s = wavelength / (2.0 * pitch)
    return s / math.sqrt(1.0 - s * s)
