"""GB300 NU-FDS reconstruction of wide-angle holograms: thin Python binding.

The work runs in libnufds.so (hand-written sm_103a CUDA behind the C ABI of
include/nufds.h).  This module only marshals arguments: torch provides device
memory and streams.  There is no CPU fallback: if the library is not built,
``lib()`` raises.

    import torch, paper_2410_13474_gb300 as nf
    plan = nf.Plan(wavelength=532e-9, pitch=0.4e-6, nx=512, ny=512, hologram=h)  # h: cuda complex64
    out = plan.reconstruct(nf.View(z=1e-3))                                     # float32 intensity
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
# NUFDS_BOUNDS_CHECK=1 in the environment loads the debug library instead
# (bounds-checked gathers; build.build(bounds_check=True) makes it)
LIB_PATH = os.path.join(_HERE, "libnufds_bc.so" if os.environ.get("NUFDS_BOUNDS_CHECK") == "1"
                        else "libnufds.so")

OK, EINVAL, ENOMEM, EUNSUPPORTED, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4, -5
FP32, FP16_STORE, BF16_STORE = 0, 1, 2
OUT_INTENSITY, OUT_FIELD, OUT_INTENSITY_ACCUM = 0, 1, 2
MODE_NUFDS, MODE_PLAIN_FRT = 0, 1
FLAG_PAPER_POLY_M = 1   # the paper's degree-8 polynomial for 2F1 (Section 4)
FLAG_PAPER_LINEAR = 2   # bilinear resampling on the unpadded grids (Section 4, steps 2 and 5)

# every function include/nufds.h declares
ABI_FUNCTIONS = ("nufds_plan_create", "nufds_plan_load", "nufds_view_plan", "nufds_reconstruct",
                 "nufds_reconstruct_batch", "nufds_reconstruct_sweep", "nufds_destroy", "nufds_plan_device_bytes",
                 "nufds_status_string", "nufds_launch_count", "nufds_profile",
                 "nufds_profile_read", "nufds_reconstruct_noalloc", "nufds_wavefront_error",
                 "nufds_output_map", "nufds_output_map_inverse", "nufds_debug_bounds_violations")


class NufdsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, status_string(code), code))


class _Params(ctypes.Structure):
    _fields_ = [("wavelength_m", ctypes.c_double), ("pitch_m", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64)]


class _View(ctypes.Structure):
    _fields_ = [("z_m", ctypes.c_double), ("center_x_m", ctypes.c_double),
                ("center_y_m", ctypes.c_double), ("width_m", ctypes.c_double),
                ("height_m", ctypes.c_double), ("out_nx", ctypes.c_int32),
                ("out_ny", ctypes.c_int32), ("out_kind", ctypes.c_int32),
                ("mode", ctypes.c_int32)]


class _ViewInfo(ctypes.Structure):
    _fields_ = [("out_nx", ctypes.c_int64), ("out_ny", ctypes.c_int64),
                ("k_lo_x", ctypes.c_int64), ("k_hi_x", ctypes.c_int64),
                ("k_lo_y", ctypes.c_int64), ("k_hi_y", ctypes.c_int64),
                ("np_x", ctypes.c_int64), ("np_y", ctypes.c_int64),
                ("k_c_x", ctypes.c_int64), ("k_c_y", ctypes.c_int64),
                ("pitch_out_x_m", ctypes.c_double), ("pitch_out_y_m", ctypes.c_double),
                ("width_m", ctypes.c_double), ("height_m", ctypes.c_double),
                ("on_full_view_lattice", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_uint64)]


class _StageStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libnufds.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built (run paper_2410_13474_gb300.build.build());"
                               " there is no CPU fallback" % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.nufds_plan_create.argtypes = [ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(vp)]
        L.nufds_plan_load.argtypes = [vp, vp, vp]
        L.nufds_view_plan.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_View),
                                      ctypes.POINTER(_ViewInfo)]
        L.nufds_reconstruct.argtypes = [vp, ctypes.POINTER(_View), vp, vp]
        L.nufds_reconstruct_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_View),
                                              ctypes.POINTER(vp), ctypes.c_int32, vp,
                                              ctypes.POINTER(ctypes.c_int32)]
        L.nufds_reconstruct_sweep.argtypes = [vp, ctypes.POINTER(_View), ctypes.POINTER(vp),
                                              ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_int32)]
        L.nufds_destroy.argtypes = [vp]
        L.nufds_destroy.restype = None
        L.nufds_plan_device_bytes.argtypes = [vp]
        L.nufds_plan_device_bytes.restype = ctypes.c_uint64
        L.nufds_status_string.argtypes = [ctypes.c_int]
        L.nufds_status_string.restype = ctypes.c_char_p
        L.nufds_profile.argtypes = [vp, ctypes.c_int32]
        L.nufds_profile_read.argtypes = [vp, ctypes.POINTER(_StageStat), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)]
        L.nufds_launch_count.argtypes = [ctypes.c_int32]
        dp = ctypes.POINTER(ctypes.c_double)
        L.nufds_output_map.argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, dp, dp]
        L.nufds_output_map_inverse.argtypes = [ctypes.POINTER(_Params), ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                               dp, dp]
        L.nufds_wavefront_error.argtypes = [ctypes.POINTER(_Params), ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                            ctypes.c_double, ctypes.c_int32, dp, dp, dp]
        L.nufds_launch_count.restype = ctypes.c_int64
        L.nufds_debug_bounds_violations.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().nufds_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != OK:
        raise NufdsError(code, what)


def bounds_violations(reset: bool = False):
    """(count, first element offset or -1) of the gather reads the debug
    library found outside their arrays (nufds_debug_bounds_violations);
    raises NufdsError(EUNSUPPORTED) on the product library."""
    first = ctypes.c_int64(-1)
    n = lib().nufds_debug_bounds_violations(1 if reset else 0, ctypes.byref(first))
    if n < 0:
        raise NufdsError(n, "nufds_debug_bounds_violations")
    return int(n), int(first.value)


def launch_count(reset: bool = False) -> int:
    """Kernel launches this library issued on the calling thread (see nufds_launch_count)."""
    return int(lib().nufds_launch_count(1 if reset else 0))


@dataclass
class View:
    """One requested view: distance z, centre and size in the object plane
    (0,0 = full view of Eq. 1), output pixels (0,0 = hologram size)."""
    z: float
    center_x: float = 0.0
    center_y: float = 0.0
    width: float = 0.0
    height: float = 0.0
    out_nx: int = 0
    out_ny: int = 0
    kind: int = OUT_INTENSITY
    mode: int = MODE_NUFDS          # MODE_PLAIN_FRT: Eq. 2 alone (no stretch, x' = x_o)

    def _c(self) -> _View:
        return _View(self.z, self.center_x, self.center_y, self.width, self.height,
                     self.out_nx, self.out_ny, self.kind, self.mode)


def _params(wavelength, pitch, nx, ny, precision=FP32, budget=0, flags=0) -> _Params:
    return _Params(wavelength, pitch, nx, ny, precision, flags, budget)


def view_plan(wavelength: float, pitch: float, nx: int, ny: int, view: View,
              flags: int = 0) -> dict:
    """Host-only planner result for one view (band, FFT sizes N', output grid)."""
    info = _ViewInfo()
    p = _params(wavelength, pitch, nx, ny, flags=flags)
    v = view._c()
    _check(lib().nufds_view_plan(ctypes.byref(p), ctypes.byref(v), ctypes.byref(info)),
           "nufds_view_plan")
    return {name: getattr(info, name) for name, _ in _ViewInfo._fields_ if name != "reserved"}


def output_map(wavelength: float, pitch: float, n: int, z: float, xo: float, yo: float,
               flags: int = 0):
    """Eq. 17 on the host: (x_o', y_o') for the object point (x_o, y_o) at z."""
    a, b = ctypes.c_double(), ctypes.c_double()
    p = _params(wavelength, pitch, n, n, flags=flags)
    _check(lib().nufds_output_map(ctypes.byref(p), z, xo, yo, ctypes.byref(a), ctypes.byref(b)),
           "nufds_output_map")
    return a.value, b.value


def output_map_inverse(wavelength: float, pitch: float, n: int, z: float, xp: float, yp: float,
                       steps: int = 4, flags: int = 0):
    """The paper's fixed-point inverse of Eq. 17 (second Eq. 18), on the host."""
    a, b = ctypes.c_double(), ctypes.c_double()
    p = _params(wavelength, pitch, n, n, flags=flags)
    _check(lib().nufds_output_map_inverse(ctypes.byref(p), z, xp, yp, steps, ctypes.byref(a),
                                          ctypes.byref(b)), "nufds_output_map_inverse")
    return a.value, b.value


def wavefront_error(wavelength: float, pitch: float, n: int, xo: float, yo: float, zo: float,
                    mode: int = MODE_NUFDS, z_r: float = 0.0, samples: int = 1025,
                    flags: int = 0):
    """Wavefront error (waves) of the point (xo, yo, zo) along the hologram's
    central row, host only: returns (x, W, max|W|) as numpy arrays and a float;
    W is NaN where the point's local frequency leaves the band."""
    import numpy as np
    x = np.zeros(samples)
    w = np.zeros(samples)
    mx = ctypes.c_double()
    p = _params(wavelength, pitch, n, n, flags=flags)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().nufds_wavefront_error(ctypes.byref(p), xo, yo, zo, mode, z_r, samples,
                                       x.ctypes.data_as(dp), w.ctypes.data_as(dp),
                                       ctypes.byref(mx)), "nufds_wavefront_error")
    return x, w, mx.value


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A hologram geometry with its FP64-derived tables and (once loaded) the
    cached oversampled spectrum of one hologram, on the current CUDA device."""

    def __init__(self, wavelength: float, pitch: float, nx: int, ny: int, hologram=None,
                 stream=None, precision: int = FP32, budget: int = 0, flags: int = 0):
        self.wavelength, self.pitch, self.nx, self.ny = wavelength, pitch, nx, ny
        self.flags = flags
        self._p = ctypes.c_void_p()
        prm = _params(wavelength, pitch, nx, ny, precision, budget, flags)
        holo = None if hologram is None else self._holo_ptr(hologram)
        _check(lib().nufds_plan_create(ctypes.byref(prm), holo, _stream_handle(stream),
                                       ctypes.byref(self._p)), "nufds_plan_create")

    def _holo_ptr(self, h):
        import torch
        if not (h.is_cuda and h.dtype == torch.complex64 and h.is_contiguous()
                and tuple(h.shape) == (self.ny, self.nx)):
            raise ValueError("hologram must be a contiguous cuda complex64 tensor of shape (ny, nx)")
        return ctypes.c_void_p(h.data_ptr())

    def load(self, hologram, stream=None):
        _check(lib().nufds_plan_load(self._p, self._holo_ptr(hologram), _stream_handle(stream)),
               "nufds_plan_load")

    def view_plan(self, view: View) -> dict:
        return view_plan(self.wavelength, self.pitch, self.nx, self.ny, view, self.flags)

    def output_like(self, view: View):
        import torch
        info = self.view_plan(view)
        dt = torch.complex64 if view.kind == OUT_FIELD else torch.float32
        return torch.empty((info["out_ny"], info["out_nx"]), dtype=dt, device="cuda")

    def reconstruct(self, view: View, out=None, stream=None):
        import torch
        if out is None:
            out = self.output_like(view)
        want = torch.complex64 if view.kind == OUT_FIELD else torch.float32
        if not (out.is_cuda and out.dtype == want and out.is_contiguous()):
            raise ValueError("out must be a contiguous cuda %s tensor" % want)
        v = view._c()
        _check(lib().nufds_reconstruct(self._p, ctypes.byref(v), ctypes.c_void_p(out.data_ptr()),
                                       _stream_handle(stream)), "nufds_reconstruct")
        return out

    def reconstruct_sweep(self, views, outs=None, stream=None):
        """Views of the loaded hologram in order (e.g. a focal sweep over z); a view
        with the band and N' of the previous one reuses its stretched spectrum.
        Returns (outs, per-view status codes)."""
        if outs is None:
            outs = [self.output_like(v) for v in views]
        n = len(views)
        va = (_View * n)(*[v._c() for v in views])
        oa = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        st = (ctypes.c_int32 * n)()
        lib().nufds_reconstruct_sweep(self._p, va, oa, n, _stream_handle(stream), st)
        return outs, list(st)

    def profile(self, enable: bool = True):
        """Start (clearing) or stop recording CUDA events around every launch."""
        _check(lib().nufds_profile(self._p, 1 if enable else 0), "nufds_profile")

    def profile_read(self) -> list:
        """Per-stage [{name, launches, total_ms, bytes}] of what was recorded."""
        arr = (_StageStat * 16)()
        n = ctypes.c_int32()
        _check(lib().nufds_profile_read(self._p, arr, 16, ctypes.byref(n)), "nufds_profile_read")
        return [dict(name=arr[i].name.decode(), launches=int(arr[i].launches),
                     total_ms=float(arr[i].total_ms), bytes=float(arr[i].bytes))
                for i in range(min(n.value, 16))]

    def device_bytes(self) -> int:
        return int(lib().nufds_plan_device_bytes(self._p))

    def close(self):
        if self._p:
            lib().nufds_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct_batch(plans, views, outs, stream=None):
    """Reconstruct views[i] of plans[i] into outs[i] in order; returns per-view status codes."""
    n = len(views)
    pa = (ctypes.c_void_p * n)(*[p._p.value for p in plans])
    va = (_View * n)(*[v._c() for v in views])
    oa = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    st = (ctypes.c_int32 * n)()
    lib().nufds_reconstruct_batch(pa, va, oa, n, _stream_handle(stream), st)
    return list(st)
