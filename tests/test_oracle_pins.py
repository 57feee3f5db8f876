"""Pins of the FP64 oracle against things other than itself.

Each check is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong normalisation)
fails at least one of them:

* the FFT against the direct O(N^2) definition and Parseval;
* 2F1 against scipy, mpmath and Gauss's closed form at w = 1;
* Eq. 15 by finite differences of the stretch of Eqs. 9, 10 and 16;
* the pull-back against the forward map (round trip, symmetry);
* the paper's printed values (tests/golden/paper_pins.json);
* the off-grid evaluation against the direct DTFT;
* the whole method against the physics of Eq. 3: a point source must refocus
  at the pixel of its true position, with peak intensity N^4, while the plain
  Fresnel transform lands it where Eq. 4 predicts;
* the field of the plain Fresnel transform, output chirp included, against
  the closed-form Fresnel diffraction integral of a Gaussian beam.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _dft_direct(x, sign=-1):
    n = x.size
    k = np.arange(n)
    ang = 2.0 * np.pi * ((np.outer(k, k)) % n) / n
    return (np.cos(ang) + sign * 1j * np.sin(ang)) @ x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 12, 15, 30, 45, 64, 90, 7, 49])
def test_fft_matches_direct_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        ref = _dft_direct(x, sign)
        got = oracle.fft(x, sign)
        assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def test_fft_inverse_round_trip_and_parseval():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(360) + 1j * rng.standard_normal(360)
    X = oracle.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) - x.size * np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(X) ** 2)
    assert np.abs(oracle.fft(X, +1) / x.size - x).max() < 1e-14


def test_centred_dft2_definition():
    rng = np.random.default_rng(2)
    ny, nx = 12, 20
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    got = oracle.centred_dft2(a)
    cx = np.arange(nx) - nx // 2
    cy = np.arange(ny) - ny // 2
    Ex = np.exp(-2j * np.pi * np.outer(cx, cx) / nx)
    Ey = np.exp(-2j * np.pi * np.outer(cy, cy) / ny)
    ref = Ey @ a @ Ex.T
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_hyp2f1_against_scipy_and_closed_form(golden):
    from scipy.special import hyp2f1
    for w in np.concatenate([np.linspace(0, 0.999, 60), [0.5, 0.9999, 1 - 1e-9]]):
        ref = hyp2f1(0.5, 0.75, 1.5, w)
        assert abs(oracle.hyp2f1(w) - ref) <= 3e-14 * ref
    g = golden["hyp2f1_at_one"]
    closed = math.gamma(1.5) * math.gamma(0.25) / math.gamma(0.75)
    assert abs(closed - g["value"]) < g["tol"]
    assert abs(oracle.hyp2f1(1.0) - closed) < 1e-14
    assert math.isnan(oracle.hyp2f1(1.0 + 1e-12))


def test_hyp2f1_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for w in [0.01, 0.37, 0.5, 0.61, 0.83, 0.97, 0.99999]:
        ref = float(mpmath.hyp2f1(0.5, 0.75, 1.5, w))
        assert abs(oracle.hyp2f1(w) - ref) <= 2e-15 * ref


@pytest.mark.parametrize("u,v", [(0.1, 0.05), (0.5, -0.3), (-0.7, 0.4), (0.6, 0.6), (0.05, 0.9)])
def test_eq15_by_finite_differences(u, v):
    """d f'_x / d f_x = sqrt(1 - l^2 fy^2) (1 - l^2 fy^2 - l^2 fx^2)^(-3/4)  (Eq. 15)."""
    lam = 0.532e-6
    fx, fy = u / lam, v / lam
    h = 1e-5 / lam
    d = (oracle.forward(lam, fx + h, fy)[0] - oracle.forward(lam, fx - h, fy)[0]) / (2 * h)
    eq15 = math.sqrt(1 - v * v) * (1 - v * v - u * u) ** -0.75
    assert abs(d - eq15) < 1e-7 * eq15
    # the same law for the y axis (variables exchanged)
    d = (oracle.forward(lam, fx, fy + h)[1] - oracle.forward(lam, fx, fy - h)[1]) / (2 * h)
    eq15y = math.sqrt(1 - u * u) * (1 - v * v - u * u) ** -0.75
    assert abs(d - eq15y) < 1e-7 * eq15y


def test_magnification_basic_properties():
    lam = 0.532e-6
    assert oracle.mag(lam, 0.0, 0.0) == (1.0, 1.0)
    # paraxial limit m -> 1 + O(f^2); m > 1 elsewhere (Fig. 4a: magnification greater than one)
    mx, my = oracle.mag(lam, 1e3, 2e3)
    assert abs(mx - 1) < 1e-5 and abs(my - 1) < 1e-5
    for u, v in [(0.3, 0.1), (0.6, 0.5), (0.1, 0.8)]:
        mx, my = oracle.mag(lam, u / lam, v / lam)
        assert mx > 1 and my > 1
    # m_x(fx, fy) = m_y(fy, fx)
    a = oracle.mag(lam, 0.4 / lam, 0.2 / lam)
    b = oracle.mag(lam, 0.2 / lam, 0.4 / lam)
    assert a[0] == b[1] and a[1] == b[0]


def test_pullback_round_trip_and_symmetry():
    lam, pitch = 0.532e-6, 0.3e-6
    rng = np.random.default_rng(3)
    for _ in range(200):
        r = 0.97 * math.sqrt(rng.random())
        a = 2 * math.pi * rng.random()
        fx, fy = r * math.cos(a) / lam, r * math.sin(a) / lam
        fpx, fpy = oracle.forward(lam, fx, fy)
        back = oracle.pullback(lam, pitch, fpx, fpy)
        assert back is not None
        assert abs(back[0] - fx) <= 1e-13 / pitch and abs(back[1] - fy) <= 1e-13 / pitch
        nb = oracle.pullback(lam, pitch, -fpx, fpy)
        assert abs(nb[0] + fx) <= 1e-13 / pitch and abs(nb[1] - fy) <= 1e-13 / pitch
    # beyond the image of the propagating disc there is no pre-image
    assert oracle.pullback(lam, pitch, 3.0 / lam, 0.0) is None
    assert oracle.pullback(lam, pitch, 2.3 / lam, 2.3 / lam) is None   # diagonal max ~2.205


def test_printed_geometry_pins(golden):
    g = golden["image_size_eq1"]
    p = oracle.plan_view(g["wavelength"], g["pitch"], 64, 64, g["z"])
    assert abs(p["width"] - g["B"]) < g["B_tol"]
    assert abs(2 * math.degrees(math.atan(p["width"] / (2 * g["z"]))) - g["fov_deg"]) < g["fov_tol"]
    g = golden["fov_vs_pitch"]
    for pitch, fov in zip(g["pitches"], g["fov_deg"]):
        w = oracle.plan_view(g["wavelength"], pitch, 64, 64, 1.0)["width"]
        assert abs(2 * math.degrees(math.atan(w / 2)) - fov) < g["fov_tol"]
    g = golden["fov_cgh3"]
    w = oracle.plan_view(g["wavelength"], g["pitch_100"], 64, 64, 1.0)["width"]
    assert abs(2 * math.degrees(math.atan(w / 2)) - g["fov_deg_100"]) < g["fov_tol_100"]
    w = oracle.plan_view(g["wavelength"], g["pitch_60"], 64, 64, g["z_60"])["width"]
    assert abs(w - g["B_60"]) < g["B_tol"]
    g = golden["fov_neptune_8k"]
    w = oracle.plan_view(g["wavelength"], g["pitch"], 64, 64, 1.0)["width"]
    assert abs(2 * math.degrees(math.atan(w / 2)) - g["fov_deg"]) < g["fov_tol"]


def test_printed_phase_space_pins(golden):
    g = golden["frt_wrong_coordinate"]
    x, y, z = g["point"]
    fxl, cxl = oracle.ps_tools(g["wavelength"], x, y, z)
    assert abs(z * g["wavelength"] * fxl - g["x_ro"]) < g["tol"]
    g = golden["frt_corrected_distance"]
    fxl, cxl = oracle.ps_tools(g["wavelength"], x, y, z)
    assert abs(-1.0 / cxl - g["z_ro"]) < g["tol"]
    assert abs(g["wavelength"] * fxl / (-cxl) - g["x_ro"]) < g["tol"]
    g = golden["frt_corrected_distances_three_points"]
    for z, zro in zip(g["z"], g["z_ro"]):
        B = oracle.plan_view(g["wavelength"], g["pitch"], 64, 64, z)["width"]
        fxl, cxl = oracle.ps_tools(g["wavelength"], 0.45 * B, 0.0, z)
        assert abs(-1.0 / cxl - zro) < g["tol"]


def test_printed_stretch_and_output_map_pins(golden):
    g = golden["frequency_stretch_example"]
    assert abs(oracle.forward(g["wavelength"], g["fx"], 0.0)[0] - g["fpx"]) < g["tol"]
    g = golden["output_map_example"]
    for lam in g["wavelengths"]:
        xop, yop = oracle.output_map(lam, g["z"], g["xo"], 0.0)
        assert abs(xop - g["xop"]) < g["tol"] and yop == 0.0
    # Fig. 4b: x_o' is always smaller than x_o
    for xo in [0.05, 0.3, 0.9]:
        assert oracle.output_map(0.64e-6, 1.0, xo, 0.2)[0] < xo


def test_iterative_inverse_converges_within_half_pixel(golden):
    from scipy.optimize import brentq
    g = golden["iterative_inverse_convergence"]
    lam, z = g["wavelength"], g["z"]
    B = oracle.plan_view(lam, g["pitch"], g["n"], g["n"], z)["width"]
    pix = B / g["n"]
    lim = g["window_fraction"] * B
    worst = 0.0
    for xo in np.linspace(-lim, lim, 21):
        for yo in np.linspace(-lim, lim, 21):
            xop, yop = oracle.output_map(lam, z, xo, yo)
            x4, y4 = oracle.output_map_iterative_inverse(lam, z, xop, yop, g["steps"])
            x5, y5 = oracle.output_map_iterative_inverse(lam, z, xop, yop, g["steps"] + 1)
            worst = max(worst, abs(x4 - x5) / pix, abs(y4 - y5) / pix)
    assert worst < g["max_err_pixels"]
    # the iteration contracts everywhere in the window, towards the exact inverse of Eq. 17
    for xo, yo in [(0.8, 0.0), (0.6, -0.7), (-0.3, 0.2)]:
        xop, yop = oracle.output_map(lam, z, xo, yo)
        steps = [oracle.output_map_iterative_inverse(lam, z, xop, yop, k) for k in range(1, 12)]
        d = [abs(a[0] - xo) + abs(a[1] - yo) for a in steps]
        assert all(d[k + 1] < d[k] for k in range(len(d) - 1) if d[k] > 1e-12)
        far = oracle.output_map_iterative_inverse(lam, z, xop, yop, 200)
        assert abs(far[0] - xo) < 1e-9 and abs(far[1] - yo) < 1e-9
    xop, _ = oracle.output_map(lam, z, 0.6, 0.0)
    root = brentq(lambda x: oracle.output_map(lam, z, x, 0.0)[0] - xop, 0.0, 1.0, xtol=1e-15)
    assert abs(root - 0.6) < 1e-12


def test_nice_sizes():
    for n in [1, 63, 64, 65, 587, 640, 4439, 4608, 7926, 22112, 30000]:
        m = oracle.nice(n)
        assert m >= n and m % 64 == 0
        r = m // 64
        while r % 2 == 0:
            r //= 2
        assert r in (1, 3, 5, 9, 15, 45)
        # nothing smaller of that form
        for cand in range(n, m):
            c = cand
            if c % 64:
                continue
            c //= 64
            while c % 2 == 0:
                c //= 2
            assert c not in (1, 3, 5, 9, 15, 45)


def test_view_plan_sizes_of_the_workloads():
    from synth.configs import SMALL_512, WA_4096, UWA_16K, SMALL_512_MM, WA_4096_MM, UWA_16K_MM
    expect = {SMALL_512.name: 640, WA_4096.name: 4608, UWA_16K.name: 23040,
              SMALL_512_MM.name: 640, WA_4096_MM.name: 4608, UWA_16K_MM.name: 23040}
    for w in (SMALL_512, WA_4096, UWA_16K, SMALL_512_MM, WA_4096_MM, UWA_16K_MM):
        p = oracle.plan_view(w.wavelength, w.pitch, w.n, w.n, w.z_view)
        assert p["np_x"] == p["np_y"] == expect[w.name]
        assert p["k_lo_x"] == -p["k_hi_x"] - 1 or p["k_lo_x"] == -p["k_hi_x"]


def test_nufft_matches_direct_dtft():
    rng = np.random.default_rng(4)
    ny, nx = 24, 40
    c = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    tx = rng.uniform(-nx / 2, nx / 2, 300)
    ty = rng.uniform(-ny / 2, ny / 2, 300)
    tx[:5] = [0, -nx / 2, nx / 2 - 1e-9, 3.0, -7.5]
    ty[:5] = [0, -ny / 2, 1.0, ny / 2, 2.25]
    ref = oracle.dtft2_direct(c, tx, ty)
    got = oracle.nufft2(c, tx, ty)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(c).sum() / math.sqrt(c.size)
    # on the integer lattice the DTFT is the centred DFT
    kx, ky = np.meshgrid(np.arange(nx) - nx // 2, np.arange(ny) - ny // 2)
    lat = oracle.dtft2_direct(c, kx, ky).reshape(ny, nx)
    assert np.abs(lat - oracle.centred_dft2(c)).max() < 1e-11 * np.abs(lat).max()


def fresnel_gaussian_1d(xp, c, w, f0, lam, z):
    """The Fresnel diffraction integral of a 1-D Gaussian beam in closed form:
    int exp(-(x - c)^2 / (2 w^2) + 2 pi i f0 x) exp(i pi (xp - x)^2 / (lambda z)) dx.
    The exponent is -A x^2 + B x + C with Re A > 0, whose integral over the
    real line is sqrt(pi / A) exp(B^2 / (4 A) + C) (principal square root)."""
    A = 1.0 / (2 * w * w) - 1j * np.pi / (lam * z)
    B = c / (w * w) + 2j * np.pi * f0 - 2j * np.pi * xp / (lam * z)
    C = -c * c / (2 * w * w) + 1j * np.pi * xp * xp / (lam * z)
    return np.sqrt(np.pi / A) * np.exp(B * B / (4 * A) + C)


# (z, beam centre, carrier frequency in units of 1/pitch, view): full views and an
# off-centre partial view that the beam is steered into
FRESNEL_CASES = [
    (0.1e-3, (2e-6, -1e-6), (0.15, -0.1), None),
    (0.3e-3, (-3e-6, 2e-6), (-0.2, 0.05), None),
    (0.1e-3, (2e-6, -1e-6), (0.3, 0.2), (0.3, 0.25, 40, 32)),
]


def gaussian_beam_case(case, lam=532e-9, pitch=0.4e-6, n=128, w=3e-6):
    """A sampled Gaussian beam H (complex64, n x n), the view arguments of the
    plain transform, and the expected field on the view's pixels: the Fresnel
    integral of the beam divided by pitch^2 (a sum over samples is the integral
    over the cells, and Eq. 2 carries no prefactor)."""
    z, (cx, cy), (ax, ay), view = case
    fx0, fy0 = ax / pitch, ay / pitch
    x = (np.arange(n) - n / 2) * pitch
    gx = np.exp(-(x - cx) ** 2 / (2 * w * w) + 2j * np.pi * fx0 * x)
    gy = np.exp(-(x - cy) ** 2 / (2 * w * w) + 2j * np.pi * fy0 * x)
    H = (gy[:, None] * gx[None, :]).astype(np.complex64)
    B = oracle.plan_view(lam, pitch, n, n, z, stretch=0)["width"]
    if view is None:
        kw = dict(cx=0.0, cy=0.0, w=0.0, h=0.0, ox=0, oy=0)
    else:
        # the beam lands near x' = c + lambda z f0 (stationary phase)
        kw = dict(cx=cx + lam * z * fx0, cy=cy + lam * z * fy0, w=view[0] * B, h=view[1] * B,
                  ox=view[2], oy=view[3])
    pv = oracle.plan_view(lam, pitch, n, n, z, kw["cx"], kw["cy"], kw["w"], kw["h"], kw["ox"],
                          kw["oy"], stretch=0)
    xo = kw["cx"] + (np.arange(pv["out_nx"]) - 0.5 * pv["out_nx"]) * pv["pitch_out_x"]
    yo = kw["cy"] + (np.arange(pv["out_ny"]) - 0.5 * pv["out_ny"]) * pv["pitch_out_y"]
    ref = (fresnel_gaussian_1d(yo, cy, w, fy0, lam, z)[:, None] *
           fresnel_gaussian_1d(xo, cx, w, fx0, lam, z)[None, :]) / pitch ** 2
    return H, dict(lam=lam, pitch=pitch, z=z, **kw), ref


@pytest.mark.parametrize("case", FRESNEL_CASES)
def test_plain_fresnel_field_is_the_fresnel_integral(case):
    """Eq. 2 including its output factor e^{i pi |x'|^2/(lambda z)} (step O9):
    the plain transform (no stretch, x' = x_o) of a sampled Gaussian beam is
    the Fresnel diffraction integral int H(x) e^{i pi |x' - x|^2/(lambda z)} dx
    (the same kernel with the square not expanded), known in closed form for a
    Gaussian.  The field is compared element by element with no fitted
    constant; a conjugated or missing output chirp leaves an O(1) residual."""
    H, a, ref = gaussian_beam_case(case)
    f, _ = oracle.reconstruct(H, a["lam"], a["pitch"], a["z"], a["cx"], a["cy"], a["w"], a["h"],
                              a["ox"], a["oy"], stretch=False)
    assert f.shape == ref.shape
    e = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert e < 1e-6, e   # complex64 rounding of H is ~3e-8
    # the beam lands inside the view, away from its border
    j, i = np.unravel_index(np.argmax(np.abs(ref)), ref.shape)
    assert 2 <= i < ref.shape[1] - 2 and 2 <= j < ref.shape[0] - 2


GEOM = dict(lam=532e-9, pitch=0.4e-6, n=256, z=1.0e-3)


def _point_hologram(ix, iy, n=GEOM["n"], z=GEOM["z"], lam=GEOM["lam"], pitch=GEOM["pitch"]):
    B = oracle.plan_view(lam, pitch, n, n, z)["width"]
    p = B / n
    xo, yo = (ix - n / 2) * p, (iy - n / 2) * p
    H = synth.hologram(np.array([[xo, yo, z, 1.0, 0.3]]), lam, pitch, n, n)
    return H, xo, yo, p


@pytest.mark.parametrize("ix,iy", [(128, 128), (200, 128), (240, 30), (60, 210), (20, 236)])
def test_point_source_refocuses_at_its_position(ix, iy):
    """Whole method vs the physics of Eq. 3 (the exact spherical wave from a
    point converges at the point): the NU-FDS intensity peak is the pixel of
    the generating point; the plain FrT (Eq. 2, no stretch) puts it where the
    local frequency of Eq. 4 says, x_ro = z lambda f_xl(0,0)."""
    lam, n, z = GEOM["lam"], GEOM["n"], GEOM["z"]
    H, xo, yo, p = _point_hologram(ix, iy)
    _, I = oracle.reconstruct(H, lam, GEOM["pitch"], z)
    j, i = np.unravel_index(np.argmax(I), I.shape)
    assert (i, j) == (ix, iy)
    if (ix, iy) == (128, 128):
        # normalisation: unnormalised forward DFT, IDFT / N'^2, FrT sum => |O|^2 = N^4
        assert abs(I.max() / n ** 4 - 1) < 5e-3
    _, I0 = oracle.reconstruct(H, lam, GEOM["pitch"], z, stretch=False)
    j0, i0 = np.unravel_index(np.argmax(I0), I0.shape)
    fxl, _ = oracle.ps_tools(lam, xo, yo, z)
    fyl, _ = oracle.ps_tools(lam, yo, xo, z)
    # the plain FrT image is blurred (Fig. 2b): its peak is within a few pixels of x_ro
    assert abs(i0 - (n / 2 + z * lam * fxl / p)) <= 3
    assert abs(j0 - (n / 2 + z * lam * fyl / p)) <= 3
    if (ix, iy) != (128, 128):
        assert I0.max() < 0.5 * I.max()      # the plain FrT blurs a wide-angle point


def test_two_points_focus_at_their_own_depths():
    """Fig. 7b-e style: two points at different depths near the FoV edge each
    focus sharply at their own distance and are defocused at the other's."""
    lam, pitch, n = GEOM["lam"], GEOM["pitch"], 256
    z1, z2 = 0.8e-3, 1.6e-3
    B1 = oracle.plan_view(lam, pitch, n, n, z1)["width"]
    B2 = oracle.plan_view(lam, pitch, n, n, z2)["width"]
    p1, p2 = B1 / n, B2 / n
    x1, x2 = (220 - n / 2) * p1, (30 - n / 2) * p2
    pts = np.array([[x1, 0.0, z1, 1.0, 0.1], [x2, 0.0, z2, 1.0, 2.0]])
    H = synth.hologram(pts, lam, pitch, n, n)
    _, I1 = oracle.reconstruct(H, lam, pitch, z1)
    _, I2 = oracle.reconstruct(H, lam, pitch, z2)
    assert np.unravel_index(np.argmax(I1), I1.shape) == (128, 220)
    assert np.unravel_index(np.argmax(I2), I2.shape) == (128, 30)
    assert I1[128, 220] > 20 * I2[128, int(round(n / 2 + x1 / p2))]


def test_reconstruct_views_equals_single_views():
    """The multi-view entry point (one gridded transform of the hologram shared
    by the views) returns exactly what one call per view returns."""
    rng = np.random.default_rng(8)
    H = (rng.standard_normal((96, 128)) + 1j * rng.standard_normal((96, 128))).astype(np.complex64)
    lam, pitch = 532e-9, 0.4e-6
    vs = [dict(z=0.4e-3), dict(z=0.5e-3, cx=2e-5, cy=-1e-5, w=3e-5, h=2e-5, ox=30, oy=21)]
    for v, (f, i) in zip(vs, oracle.reconstruct_views(H, lam, pitch, vs)):
        f1, i1 = oracle.reconstruct(H, lam, pitch, v["z"], v.get("cx", 0.0), v.get("cy", 0.0),
                                    v.get("w", 0.0), v.get("h", 0.0), v.get("ox", 0),
                                    v.get("oy", 0))
        assert np.array_equal(f, f1) and np.array_equal(i, i1)


def test_partial_view_covering_the_window_equals_full_view():
    lam, pitch, n, z = GEOM["lam"], GEOM["pitch"], 128, 1.0e-3
    rng = np.random.default_rng(5)
    H = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    B = oracle.plan_view(lam, pitch, n, n, z)["width"]
    f_full, _ = oracle.reconstruct(H, lam, pitch, z)
    f_part, _ = oracle.reconstruct(H, lam, pitch, z, 0.0, 0.0, B, B, n, n)
    assert np.array_equal(f_full, f_part)


def test_partial_view_refocuses_in_focus_points_like_the_full_view():
    """Reading of the partial view as a spectral sub-band (Section 4): for an
    in-focus point inside the view, the peak pixel and value match the full
    view cropped to the same window."""
    lam, pitch, n, z = GEOM["lam"], GEOM["pitch"], 256, 1.0e-3
    H, xo, yo, p = _point_hologram(190, 70)
    _, I_full = oracle.reconstruct(H, lam, pitch, z)
    # 64 x 64 view whose pixel lattice is a window of the full view's
    cx, cy = (180 - n / 2) * p, (80 - n / 2) * p
    _, I_part = oracle.reconstruct(H, lam, pitch, z, cx, cy, 64 * p, 64 * p, 64, 64)
    j, i = np.unravel_index(np.argmax(I_part), I_part.shape)
    assert (i + 180 - 32, j + 80 - 32) == (190, 70)
    assert abs(I_part.max() / I_full.max() - 1) < 0.02
    plan = oracle.plan_view(lam, pitch, n, n, z, cx, cy, 64 * p, 64 * p, 64, 64)
    assert plan["np_x"] < oracle.plan_view(lam, pitch, n, n, z)["np_x"] or \
        plan["k_hi_x"] - plan["k_lo_x"] < 0.5 * n


# --- the paper's polynomial surrogate for 2F1 (Section 4, initialisation step 1) ---
@pytest.mark.parametrize("lam,pitch,max_err", [(0.64e-6, 0.5e-6, 1e-5), (532e-9, 0.307e-6, 1e-3)])
def test_paper_polynomial_surrogate_fit(lam, pitch, max_err):
    """Degree 8, 51 frequencies uniform over |f| <= 1/(2 pitch) at f_y = 0:
    the oracle's Householder fit equals numpy's least squares on the same
    samples (an independent solver); the samples are symmetric, so the odd
    coefficients vanish; and its distance from the exact 2F1 over the band
    (largest at 120 deg FoV, where 2F1 steepens at the band edge) is stated."""
    from scipy.special import hyp2f1
    with oracle.paper_poly(lam, pitch) as pp:
        c = pp.coef.copy()
    s = lam * (-0.5 + np.arange(51) / 50.0) / pitch
    y = hyp2f1(0.5, 0.75, 1.5, s * s)
    ref = np.linalg.lstsq(np.vander(s, 9, increasing=True), y, rcond=None)[0]
    assert np.allclose(c, ref, rtol=1e-8, atol=1e-10)
    assert np.all(np.abs(c[1::2]) < 1e-11)
    ss = np.linspace(s[0], s[-1], 2001)
    err = np.abs(np.polynomial.polynomial.polyval(ss, c) - hyp2f1(0.5, 0.75, 1.5, ss * ss))
    print("max |P - 2F1| over the band: %.3e" % err.max())
    assert err.max() < max_err


def test_paper_polynomial_reproduces_printed_stretch(golden):
    """The paper computed Fig. 4a with its polynomial: f_x = 0.75 um^-1 still
    lands at 0.8 um^-1 (8K hologram of 0.64 um, pitch 0.5 um)."""
    g = golden["frequency_stretch_example"]
    with oracle.paper_poly(g["wavelength"], 0.5e-6):
        fpx = oracle.forward(g["wavelength"], g["fx"], 0.0)[0]
    assert abs(fpx - g["fpx"]) < g["tol"]


def test_paper_polynomial_variant_distance_from_exact():
    """The variant against the exact method on a wide-angle point source
    (120 deg FoV, z = 0.5 m): same peak pixel; the intensity difference is
    reported."""
    lam, pitch, n, z = 532e-9, 0.307e-6, 256, 0.5
    H, xo, yo, p = _point_hologram(200, 60, n=n, z=z, lam=lam, pitch=pitch)
    _, I = oracle.reconstruct(H, lam, pitch, z)
    with oracle.paper_poly(lam, pitch):
        _, Ip = oracle.reconstruct(H, lam, pitch, z)
    e = float(np.linalg.norm(Ip - I) / np.linalg.norm(I))
    print("polynomial m vs exact 2F1: intensity rel_l2 = %.3e, peak ratio %.5f"
          % (e, Ip.max() / I.max()))
    assert np.unravel_index(np.argmax(Ip), Ip.shape) == np.unravel_index(np.argmax(I), I.shape)
    assert e < 0.1


# ---------------------------------------------------------------------------
# Paper-literal linear resampling (Section 4, steps two and five)
# ---------------------------------------------------------------------------

def test_lerp2_is_the_dft_on_the_grid_and_linear_between():
    """or_lerp2 at integer positions is the centred DFT (numpy's FFT); between
    them it reproduces affine grid data exactly, and across the periodic edge
    it averages the last and the first grid values."""
    rng = np.random.default_rng(5)
    ny, nx = 12, 16
    c = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    grid = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(c)))  # [ky + ny/2][kx + nx/2]
    kx = rng.integers(-nx // 2, nx // 2, 20)
    ky = rng.integers(-ny // 2, ny // 2, 20)
    got = oracle.lerp2(c, kx.astype(float), ky.astype(float))
    assert np.abs(got - grid[ky + ny // 2, kx + nx // 2]).max() < 1e-10
    # affine data: grid values a + b kx + d ky -> c by the inverse centred DFT
    KX, KY = np.meshgrid(np.arange(nx) - nx // 2, np.arange(ny) - ny // 2)
    g = (0.3 - 1.1j) + (0.7 + 0.2j) * KX - (0.4 - 0.9j) * KY
    c_aff = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g)))
    tx = rng.uniform(-nx // 2, nx // 2 - 1, 50)
    ty = rng.uniform(-ny // 2, ny // 2 - 1, 50)
    want = (0.3 - 1.1j) + (0.7 + 0.2j) * tx - (0.4 - 0.9j) * ty
    assert np.abs(oracle.lerp2(c_aff, tx, ty) - want).max() < 1e-10
    # periodic edge: halfway between kx = nx/2 - 1 and kx = -nx/2
    e = oracle.lerp2(c, [nx / 2 - 0.5], [0.0])[0]
    assert abs(e - 0.5 * (grid[ny // 2, -1] + grid[ny // 2, 0])) < 1e-10


def test_paper_linear_variant_refocuses_and_its_distance_from_ideal():
    """The bilinear variant still focuses a wide-angle point at its own pixel
    (the maps are the same), with the loss of the linear interpolant; its
    distance from the ideal method is reported."""
    lam, pitch, n, z = 532e-9, 0.307e-6, 256, 0.5
    H, xo, yo, p = _point_hologram(200, 60, n=n, z=z, lam=lam, pitch=pitch)
    F, I = oracle.reconstruct(H, lam, pitch, z)
    with oracle.paper_linear():
        Fl, Il = oracle.reconstruct(H, lam, pitch, z)
    e = float(np.linalg.norm(Il - I) / np.linalg.norm(I))
    print("bilinear vs ideal resampling: intensity rel_l2 = %.3e, peak ratio %.4f"
          % (e, Il.max() / I.max()))
    assert np.unravel_index(np.argmax(Il), Il.shape) == np.unravel_index(np.argmax(I), I.shape)
    assert 1e-4 < e < 1.0
    assert 0.1 < Il.max() / I.max() < 1.0  # a phasor turning ~1.8 rad per bin loses amplitude
