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


# --------------------------------------------------------------------------
# GPU generator (large inputs): same model, FP64 tile-centre phases + FP32
# in-tile offsets (~3e-5 rad per term); see pointcloud_gpu.cu.
# --------------------------------------------------------------------------
_SO_GPU = os.path.join(_HERE, "libsynth_gpu.so")
_lib_gpu = None


def build_gpu(force: bool = False) -> str:
    src = os.path.join(_HERE, "pointcloud_gpu.cu")
    if force or not os.path.exists(_SO_GPU) or os.path.getmtime(_SO_GPU) < os.path.getmtime(src):
        import shutil
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _SO_GPU + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, "-shared", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-Xcompiler", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO_GPU)
    return _SO_GPU


def gpu_hologram(pts: np.ndarray, wavelength: float, pitch: float, nx: int, ny: int, out=None):
    """complex64 cuda tensor (ny, nx) of the point-source hologram, made on the GPU."""
    import torch
    global _lib_gpu
    with _lock:
        if _lib_gpu is None:
            build_gpu()
            L = ctypes.CDLL(_SO_GPU)
            L.synth_gpu_hologram.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_void_p]
            _lib_gpu = L
    d_pts = torch.from_numpy(np.ascontiguousarray(pts, np.float64)).cuda()
    if out is None:
        out = torch.empty((ny, nx), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = _lib_gpu.synth_gpu_hologram(ctypes.c_void_p(d_pts.data_ptr()), pts.shape[0], wavelength,
                                     pitch, nx, ny, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(st))
    if rc:
        raise RuntimeError("synth_gpu_hologram failed (%d)" % rc)
    torch.cuda.synchronize()
    return out
