"""Wavefront-error diagnostic (Section 2, Figs. 2c/2f; Section 4, Fig. 5).

The oracle's W is pinned against brute force: the FFT of a sampled point
hologram gives the exact spectrum phase, the FFT of a sampled paraxial
(Fresnel) point wave gives the phase the Fresnel transform focuses, and their
difference at the point's local frequencies (Eq. 4) must be the oracle's W.
Then the paper's statements about W (FrT at z_o vs at 1/|c_xl|, NU-FDS below
the Rayleigh bound, growth with the pitch), and the library's host entry
point against the oracle.
"""
import numpy as np
import pytest

import oracle


def _spectrum(h, pitch):
    """Centred DFT of a row of samples at x_n = (n - N/2) pitch (kernel
    e^{-2 pi i f x}); returns the frequencies and the spectrum."""
    n = len(h)
    H = np.fft.fftshift(np.fft.fft(np.fft.ifftshift(h)))
    f = (np.arange(n) - n // 2) / (n * pitch)
    return f, H


def _brute_force_spectra(lam, pitch, n, xo, zo, method, z_r=0.0, pad=16):
    """Spectra of the sampled point hologram e^{-ikR_o} and of the paraxial
    point wave the transform focuses, over an aperture of n pixels zero-padded
    to pad * n samples (so the spectrum phase moves < pi / pad per bin)."""
    m = n * pad
    x = (np.arange(m) - m // 2) * pitch
    inside = np.abs(x) <= n * pitch / 2
    k = 2 * np.pi / lam
    h = np.where(inside, np.exp(-1j * k * np.sqrt((x - xo) ** 2 + zo ** 2)), 0)
    f, Hh = _spectrum(h, pitch)
    f0 = xo / (lam * np.hypot(xo, zo))
    if method == "nufds":
        zf = zo
        xf = zo * lam * oracle.forward(lam, f0, 0.0)[0]
    else:
        zf = z_r if z_r > 0 else zo
        xf = zf * lam * f0
    hp = np.where(inside, np.exp(-1j * k * (zf + (x - xf) ** 2 / (2 * zf))), 0)
    _, Hp = _spectrum(hp, pitch)
    return f, Hh, Hp, f0


def _phase_at(f, H, fr):
    """Unwrapped spectrum phase (cycles) interpolated at the frequencies fr."""
    lo, hi = fr.min(), fr.max()
    df = f[1] - f[0]
    b = (f >= lo - 2 * df) & (f <= hi + 2 * df)
    ph = np.unwrap(np.angle(H[b]))
    return np.interp(fr, f[b], ph) / (2 * np.pi)


# near-field points (a few mm), where W is waves large, so a dropped term, a
# wrong sign or a wrong focus shows far above the brute force's own ripple
# (the aperture edges, < 0.01 waves on the inner 60 % of the hologram)
BF_CASES = [(0.5e-6, 8192, 2e-3, 0.008), (0.5e-6, 8192, -1.5e-3, 0.012),
            (0.4e-6, 8192, 1e-3, 0.004), (0.75e-6, 4096, 1e-3, 0.01)]


@pytest.mark.parametrize("method", ["frt", "nufds"])
@pytest.mark.parametrize("pitch,n,xo,zo", BF_CASES)
def test_oracle_w_against_two_ffts(method, pitch, n, xo, zo):
    lam = 0.5e-6
    f, Hh, Hp, f0 = _brute_force_spectra(lam, pitch, n, xo, zo, method, pad=8)
    xs, w, _ = oracle.wavefront_error(lam, pitch, n, xo, 0.0, zo, method, 0.0, 257)
    # local frequency of each hologram sample (Eq. 4), interior of the footprint
    R = np.sqrt((xs - xo) ** 2 + zo ** 2)
    fl = -(xs - xo) / (lam * R)
    inner = np.abs(xs) <= 0.3 * n * pitch
    fq = np.append(fl[inner], f0)
    if method == "nufds":
        fpq = np.array([oracle.forward(lam, v, 0.0)[0] for v in fq])
    else:
        fpq = fq
    ph_h = _phase_at(f, Hh, fq)
    ph_p = _phase_at(f, Hp, fpq)
    w_bf = (ph_h[:-1] - ph_h[-1]) - (ph_p[:-1] - ph_p[-1])
    diff = w[inner] - w_bf
    print("%s: max|W| %.3f waves, max deviation from the two-FFT W %.4f" %
          (method, np.abs(w[inner]).max(), np.abs(diff).max()))
    assert np.abs(w[inner]).max() > 0.5
    assert np.abs(diff).max() < 0.02


def test_frt_wavefront_fig2(golden):
    p = golden["wavefront_frt_fig2"]
    lam, pitch, n = p["wavelength"], p["pitch"], p["n"]
    for z in p["z"]:
        B = 2 * z * np.tan(np.arcsin(lam / (2 * pitch)))
        xo = p["x_over_B"] * B
        _, _, w_zo = oracle.wavefront_error(lam, pitch, n, xo, 0.0, z, "frt")
        _, c = oracle.ps_tools(lam, xo, 0.0, z)
        _, _, w_zr = oracle.wavefront_error(lam, pitch, n, xo, 0.0, z, "frt", 1.0 / abs(c))
        print("z = %.1f m: FrT at z_o %.3f waves, at 1/|c| = %.3f m %.4f waves" %
              (z, w_zo, 1 / abs(c), w_zr))
        assert w_zo > p["large_above_waves"]
        assert w_zr < p["negligible_below_waves"]


def test_nufds_wavefront_fig5(golden):
    p = golden["wavefront_nufds_fig5"]
    lam, n = p["wavelength"], p["n"]
    worst = []
    for pitch in sorted(p["pitches"] + [p["pitch_1um"]]):
        th = np.arcsin(lam / (2 * pitch))
        ws = []
        for z in p["z"]:
            xo = p["x_over_B"] * 2 * z * np.tan(th)
            _, w, mx = oracle.wavefront_error(lam, pitch, n, xo, 0.0, z, "nufds")
            _, _, frt = oracle.wavefront_error(lam, pitch, n, xo, 0.0, z, "frt")
            assert np.all(np.isfinite(w))
            assert mx < 0.1 * frt  # the stretch removes most of the FrT error
            ws.append(mx)
        print("pitch %.2f um: max|W| = %s waves" % (pitch * 1e6, ["%.4f" % v for v in ws]))
        if pitch in p["pitches"]:
            assert max(ws) <= p["printed_max_waves"]
        if pitch == p["pitch_1um"]:
            assert ws[p["z"].index(p["z_1um"])] < p["rayleigh_waves"]
        # closer points are harder (Fig. 5: the 0.5 m point has the largest error)
        assert ws[0] > ws[1] > ws[2]
        worst.append(max(ws))
    assert all(a < b for a, b in zip(worst, worst[1:]))  # grows with the pitch


def test_w_is_flat_at_the_hologram_centre():
    """The focus of each method (Eq. 17 for NU-FDS, z_r lambda f_xl for the
    FrT) is the point where W has zero slope at the hologram centre."""
    lam, pitch, n = 0.5e-6, 0.4e-6, 8192
    for method, zr in (("nufds", 0.0), ("frt", 0.0), ("frt", 1.7)):
        x, w, _ = oracle.wavefront_error(lam, pitch, n, 0.3, 0.1, 0.9, method, zr, 1025)
        c = len(x) // 2
        slope = (w[c + 1] - w[c - 1]) / (x[c + 1] - x[c - 1])
        curv = (w[c + 1] - 2 * w[c] + w[c - 1]) / (x[c + 1] - x[c]) ** 2
        span = x[-1] - x[0]
        assert abs(slope) * span < 1e-6 + 1e-3 * abs(curv) * span ** 2


def test_band_edge_points_are_masked():
    lam, pitch, n, z = 0.5e-6, 0.5e-6, 8192, 0.001
    B = 2 * z * np.tan(np.arcsin(lam / (2 * pitch)))
    x, w, mx = oracle.wavefront_error(lam, pitch, n, 0.5 * B, 0.0, z, "nufds")
    bad = ~np.isfinite(w)
    assert 0 < bad.sum() < len(w)
    assert mx == np.nanmax(np.abs(w))
    R = np.sqrt((x - 0.5 * B) ** 2 + z ** 2)
    fl = -(x - 0.5 * B) / (lam * R)
    assert np.array_equal(bad, np.abs(fl) >= 0.5 / pitch)


def _nf():
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


@pytest.mark.parametrize("poly", [False, True])
def test_library_wavefront_error_matches_oracle(poly):
    nf = _nf()
    lam = 0.5e-6
    cases = [(0.75e-6, 0.45, 0.0, 0.5), (0.5e-6, 0.45, 0.2, 1.0), (0.3e-6, 0.3, -0.25, 2.0),
             (0.5e-6, 0.5, 0.0, 0.001)]
    for pitch, fx, fy, z in cases:
        B = 2 * z * np.tan(np.arcsin(lam / (2 * pitch)))
        for mode, name, zr in ((nf.MODE_NUFDS, "nufds", 0.0), (nf.MODE_PLAIN_FRT, "frt", 0.0),
                               (nf.MODE_PLAIN_FRT, "frt", 1.3 * z)):
            args = (lam, pitch, 8192, fx * B, fy * B, z)
            if poly:
                with oracle.paper_poly(lam, pitch):
                    xa, wa, ma = oracle.wavefront_error(*args, name, zr, 513)
            else:
                xa, wa, ma = oracle.wavefront_error(*args, name, zr, 513)
            xb, wb, mb = nf.wavefront_error(*args, mode, zr, 513,
                                            nf.FLAG_PAPER_POLY_M if poly else 0)
            assert np.array_equal(xa, xb)
            assert np.array_equal(np.isfinite(wa), np.isfinite(wb))
            ok = np.isfinite(wa)
            assert np.all(np.abs(wa[ok] - wb[ok]) < 1e-7)
            assert abs(ma - mb) < 1e-7


def test_library_wavefront_error_arguments():
    nf = _nf()
    with pytest.raises(nf.NufdsError) as e:
        nf.wavefront_error(0.5e-6, 0.5e-6, 1024, 0.1, 0.0, -1.0)
    assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError) as e:
        nf.wavefront_error(1.1e-6, 0.5e-6, 1024, 0.1, 0.0, 1.0)        # lambda >= 2 pitch
    assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError) as e:
        nf.wavefront_error(0.5e-6, 0.5e-6, 1024, 0.1, 0.0, 1.0, mode=7)
    assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError) as e:
        nf.wavefront_error(0.5e-6, 0.5e-6, 1024, 0.1, 0.0, 1.0, samples=0)
    assert e.value.code == nf.EINVAL
