"""The pins catch plausible mistakes: each test plants one mistake (a
transposed operand, a dropped term, a wrong sign or index) in a copy of the
oracle's C source, builds it, and checks that the pin meant to catch that
kind of mistake passes on the real oracle and fails on the mutant.  CPU only;
the mutants are built in a temporary directory and never used elsewhere."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "nufds_oracle.c")
_d, _i = ctypes.c_double, ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)


def _build(tmp_path, name, old=None, new=None):
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, "mutation site not unique: %r" % old
        src = src.replace(old, new)
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", str(so), str(c),
                           "-lm"])
    L = ctypes.CDLL(str(so))
    L.or_forward.argtypes = [_d, _d, _d, _dp, _dp]
    L.or_output_map.argtypes = [_d, _d, _d, _d, _dp, _dp]
    L.or_lerp2.argtypes = [_dp, _i, _i, _dp, _dp, ctypes.c_int64, _dp]
    L.or_centred_dft2.argtypes = [_dp, _i, _i, _i]
    L.or_wavefront_error.argtypes = [_d, _d, _i, _d, _d, _d, _i, _d, _i, _dp, _dp]
    L.or_wavefront_error.restype = _d
    L.or_nufft2.argtypes = [_dp, _i, _i, _dp, _dp, ctypes.c_int64, _dp]
    L.or_dtft2_direct.argtypes = [_dp, _i, _i, _dp, _dp, ctypes.c_int64, _dp]
    L.or_reconstruct.argtypes = [_d, _d, _i, _i, ctypes.POINTER(ctypes.c_float), _d, _d, _d, _d,
                                 _d, _i, _i, _i, _i, _dp, _dp]
    L.or_reconstruct.restype = _i
    L.or_hyp2f1.argtypes = [_d]
    L.or_hyp2f1.restype = _d
    L.or_output_map_iterative_inverse.argtypes = [_d, _d, _d, _d, _i, _dp, _dp]
    L.or_nice.argtypes = [ctypes.c_int64]
    L.or_nice.restype = ctypes.c_int64
    return L


def _pair(fn, *args):
    a, b = _d(), _d()
    fn(*[float(x) for x in args], ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


# --- the pins, each written against a library handle ---------------------

def pin_eq15(L):
    """Eq. 15 by finite differences, both axes (test_oracle_pins)."""
    lam = 0.532e-6
    for u, v in [(0.5, -0.3), (-0.7, 0.4)]:
        fx, fy = u / lam, v / lam
        h = 1e-5 / lam
        d = (_pair(L.or_forward, lam, fx + h, fy)[0] - _pair(L.or_forward, lam, fx - h, fy)[0]) / (2 * h)
        eq = math.sqrt(1 - v * v) * (1 - v * v - u * u) ** -0.75
        if abs(d - eq) >= 1e-7 * eq:
            return False
        d = (_pair(L.or_forward, lam, fx, fy + h)[1] - _pair(L.or_forward, lam, fx, fy - h)[1]) / (2 * h)
        eq = math.sqrt(1 - u * u) * (1 - v * v - u * u) ** -0.75
        if abs(d - eq) >= 1e-7 * eq:
            return False
    return True


def pin_printed_output_map(L, golden):
    g = golden["output_map_example"]
    for lam in g["wavelengths"]:
        xop, yop = _pair(L.or_output_map, lam, g["z"], g["xo"], 0.0)
        if not (abs(xop - g["xop"]) < g["tol"] and yop == 0.0):
            return False
    return True


def pin_centred_dft(L):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((6, 10)) + 1j * rng.standard_normal((6, 10))
    b = np.ascontiguousarray(a, np.complex128).copy()
    L.or_centred_dft2(b.ctypes.data_as(_dp), 10, 6, -1)
    want = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(a)))
    return np.abs(b - want).max() < 1e-9


def pin_lerp_affine(L):
    ny, nx = 12, 16
    KX, KY = np.meshgrid(np.arange(nx) - nx // 2, np.arange(ny) - ny // 2)
    g = (0.3 - 1.1j) + (0.7 + 0.2j) * KX - (0.4 - 0.9j) * KY
    c = np.ascontiguousarray(np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g))), np.complex128)
    rng = np.random.default_rng(4)
    tx = rng.uniform(-nx // 2, nx // 2 - 1, 30)
    ty = rng.uniform(-ny // 2, ny // 2 - 1, 30)
    out = np.empty(30, np.complex128)
    L.or_lerp2(c.ctypes.data_as(_dp), nx, ny, tx.ctypes.data_as(_dp), ty.ctypes.data_as(_dp), 30,
               out.ctypes.data_as(_dp))
    want = (0.3 - 1.1j) + (0.7 + 0.2j) * tx - (0.4 - 0.9j) * ty
    return np.abs(out - want).max() < 1e-10


def pin_wavefront_two_ffts(L):
    """The brute-force W of test_wavefront on its first near-field case."""
    from test_wavefront import _brute_force_spectra, _phase_at
    lam, pitch, n, xo, zo = 0.5e-6, 0.5e-6, 8192, 2e-3, 0.008
    f, Hh, Hp, f0 = _brute_force_spectra(lam, pitch, n, xo, zo, "frt", pad=8)
    xs = np.zeros(257)
    w = np.zeros(257)
    L.or_wavefront_error(lam, pitch, n, xo, 0.0, zo, 1, 0.0, 257, xs.ctypes.data_as(_dp),
                         w.ctypes.data_as(_dp))
    R = np.sqrt((xs - xo) ** 2 + zo ** 2)
    fl = -(xs - xo) / (lam * R)
    inner = np.abs(xs) <= 0.3 * n * pitch
    fq = np.append(fl[inner], f0)
    ph_h, ph_p = _phase_at(f, Hh, fq), _phase_at(f, Hp, fq)
    w_bf = (ph_h[:-1] - ph_h[-1]) - (ph_p[:-1] - ph_p[-1])
    return bool(np.all(np.isfinite(w[inner]))) and np.abs(w[inner] - w_bf).max() < 0.02


def pin_nufft(L):
    """NUFFT against the direct DTFT on a rectangular grid (test_oracle_pins)."""
    rng = np.random.default_rng(4)
    ny, nx = 24, 40
    c = np.ascontiguousarray(rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx)))
    tx = rng.uniform(-nx / 2, nx / 2, 200)
    ty = rng.uniform(-ny / 2, ny / 2, 200)
    got = np.empty(200, np.complex128)
    ref = np.empty(200, np.complex128)
    args = (c.ctypes.data_as(_dp), nx, ny, tx.ctypes.data_as(_dp), ty.ctypes.data_as(_dp), 200)
    L.or_nufft2(*args, got.ctypes.data_as(_dp))
    L.or_dtft2_direct(*args, ref.ctypes.data_as(_dp))
    return np.abs(got - ref).max() < 1e-10 * np.abs(c).sum() / math.sqrt(c.size)


def pin_refocus(L):
    """A point source refocuses on its own pixel, and a centred one with peak
    N^4 (test_oracle_pins, whole method against Eq. 3)."""
    import oracle
    import synth
    lam, pitch, n, z = 532e-9, 0.4e-6, 256, 1.0e-3
    B = oracle.plan_view(lam, pitch, n, n, z)["width"]
    p = B / n
    for ix, iy in [(128, 128), (200, 60)]:
        pts = np.array([[(ix - n / 2) * p, (iy - n / 2) * p, z, 1.0, 0.3]])
        H = np.ascontiguousarray(synth.hologram(pts, lam, pitch, n, n), np.complex64)
        field = np.empty((n, n), np.complex128)
        inten = np.empty((n, n), np.float64)
        r = L.or_reconstruct(lam, pitch, n, n, H.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             z, 0.0, 0.0, 0.0, 0.0, 0, 0, 1, 0, field.ctypes.data_as(_dp),
                             inten.ctypes.data_as(_dp))
        if r:
            return False
        j, i = np.unravel_index(np.argmax(inten), inten.shape)
        if (i, j) != (ix, iy):
            return False
        if (ix, iy) == (128, 128) and abs(inten.max() / n ** 4 - 1) >= 5e-3:
            return False
    return True


def pin_hyp2f1(L):
    """2F1(1/2, 3/4; 3/2; w) against scipy on both sides of w = 1/2."""
    from scipy.special import hyp2f1
    for w in (0.1, 0.45, 0.7, 0.95):
        ref = hyp2f1(0.5, 0.75, 1.5, w)
        if abs(L.or_hyp2f1(w) - ref) > 1e-13 * ref:
            return False
    return True


def pin_inverse_iteration(L):
    """Many steps of the paper's iteration invert Eq. 17 (test_oracle_pins)."""
    lam, z = 0.5e-6, 1.0
    for xo, yo in [(0.31, 0.0), (0.2, -0.15)]:
        xp, yp = _pair(L.or_output_map, lam, z, xo, yo)
        a, b = _d(), _d()
        L.or_output_map_iterative_inverse(lam, z, xp, yp, 200, ctypes.byref(a), ctypes.byref(b))
        if abs(a.value - xo) > 1e-9 or abs(b.value - yo) > 1e-9:
            return False
    return True


def pin_nice(L):
    """N' = the smallest 64 * 2^a * {1, 3, 5, 9, 15, 45} >= n (test_oracle_pins)."""
    def ok(c):
        if c % 64:
            return False
        c //= 64
        while c % 2 == 0:
            c //= 2
        return c in (1, 3, 5, 9, 15, 45)
    for n in [1, 63, 65, 587, 4439, 7926, 22112, 30000]:
        m = L.or_nice(n)
        if m < n or not ok(m) or any(ok(c) for c in range(n, m)):
            return False
    return True


def pin_fresnel(L):
    """Plain Fresnel-transform field against the closed-form Fresnel integral of
    a Gaussian beam, no fitted constant (test_oracle_pins)."""
    from test_oracle_pins import FRESNEL_CASES, gaussian_beam_case
    for case in FRESNEL_CASES:
        H, a, ref = gaussian_beam_case(case)
        H = np.ascontiguousarray(H, np.complex64)
        field = np.empty(ref.shape, np.complex128)
        inten = np.empty(ref.shape, np.float64)
        r = L.or_reconstruct(a["lam"], a["pitch"], H.shape[1], H.shape[0],
                             H.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a["z"], a["cx"],
                             a["cy"], a["w"], a["h"], a["ox"], a["oy"], 0, 0,
                             field.ctypes.data_as(_dp), inten.ctypes.data_as(_dp))
        if r or not np.linalg.norm(field - ref) < 1e-6 * np.linalg.norm(ref):
            return False
    return True


# --- mutants ----------------------------------------------------------------

MUTANTS = [
    # transposed operand: x stretch with the y magnification (Eqs. 9-10)
    ("stretch_other_axis", "*fpx = fx * mx;", "*fpx = fx * my;", "eq15"),
    # dropped term: the a_y^2 division in the argument of 2F1 (Eq. 16)
    ("eq16_argument", "F_of(lam * lam * fx * fx / ay,", "F_of(lam * lam * fx * fx,", "eq15"),
    # wrong index: the output map takes the y frequency (Eq. 17)
    ("output_map_axis", "*xop = z * lam * fpx;", "*xop = z * lam * fpy;", "output_map"),
    # dropped centring shift of the centred DFT
    ("dft_centring",
     "t[(size_t)((r + ny / 2) % ny) * nx + (c + nx / 2) % nx] = a[(size_t)r * nx + c];",
     "t[(size_t)r * nx + c] = a[(size_t)r * nx + c];", "centred_dft"),
    # swapped interpolation weights (the linear variant)
    ("lerp_weights", "(1 - ax) * v[0][0] + ax * v[0][1]", "ax * v[0][0] + (1 - ax) * v[0][1]",
     "lerp"),
    # wrong sign: the z term of the point's spectrum phase (wavefront error)
    ("spectrum_phase_sign", "return -(fx * xo + fy * yo + zo * sqrt(",
     "return -(fx * xo + fy * yo - zo * sqrt(", "wavefront"),
    # transposed operand: the y deconvolution of the NUFFT with the x grid length
    ("nufft_deconv_axis", "dy[n] = 1.0 / gauss_ft(p->a2, n - ny / 2, p->my);",
     "dy[n] = 1.0 / gauss_ft(p->a2, n - ny / 2, p->mx);", "nufft"),
    # wrong sign: the input chirp of Eq. 2 conjugated
    ("input_chirp_sign", "S[(size_t)m * npx + n] *= inv * (cos(ph) + I * sin(ph));",
     "S[(size_t)m * npx + n] *= inv * (cos(ph) - I * sin(ph));", "refocus"),
    # wrong term: a Pochhammer factor of the series (2F1)
    ("series_pochhammer", "term *= (a + n) * (b + n) / ((c + n) * (n + 1.0)) * w;",
     "term *= (a + n) * (b + n) / ((c + n + 1.0) * (n + 1.0)) * w;", "hyp2f1"),
    # wrong sign in the connection formula A&S 15.3.6 (w > 1/2)
    ("connection_sign", "return t1 + t2;", "return t1 - t2;", "hyp2f1"),
    # transposed operand: the inverse iteration divides by m_y
    ("inverse_iteration_axis", "double xn = xop * R / (z * mx), yn = yop * R / (z * my);",
     "double xn = xop * R / (z * my), yn = yop * R / (z * mx);", "inverse"),
    # dropped case: the factor 5 of the FFT sizes (planner)
    ("nice_no_factor5", "for (int c = 0; c <= 1; ++c) {", "for (int c = 0; c <= 0; ++c) {",
     "nice"),
    # dropped term: one axis of the inverse transform's 1 / (N'_x N'_y)
    ("idft_normalisation", "const double inv = 1.0 / ((double)npx * npy);",
     "const double inv = 1.0 / (double)npx;", "refocus"),
    # wrong sign: the output chirp of Eq. 2 conjugated (step O9)
    ("output_chirp_sign", "cplx O = (cos(ph) + I * sin(ph)) * P[o];",
     "cplx O = (cos(ph) - I * sin(ph)) * P[o];", "fresnel"),
    # dropped term: no output chirp at all (step O9)
    ("output_chirp_dropped", "cplx O = (cos(ph) + I * sin(ph)) * P[o];", "cplx O = P[o];",
     "fresnel"),
]


@pytest.fixture(scope="module")
def real(tmp_path_factory):
    return _build(tmp_path_factory.mktemp("oracle_real"), "real")


def _run_pin(kind, L, golden):
    return {"eq15": lambda: pin_eq15(L),
            "output_map": lambda: pin_printed_output_map(L, golden),
            "centred_dft": lambda: pin_centred_dft(L),
            "lerp": lambda: pin_lerp_affine(L),
            "wavefront": lambda: pin_wavefront_two_ffts(L),
            "nufft": lambda: pin_nufft(L),
            "refocus": lambda: pin_refocus(L),
            "hyp2f1": lambda: pin_hyp2f1(L),
            "inverse": lambda: pin_inverse_iteration(L),
            "nice": lambda: pin_nice(L),
            "fresnel": lambda: pin_fresnel(L)}[kind]()


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, real, golden, name, old, new, pin):
    assert _run_pin(pin, real, golden), "the pin fails on the real oracle"
    mutant = _build(tmp_path, name, old, new)
    assert not _run_pin(pin, mutant, golden), "the pin misses mutant %s" % name
