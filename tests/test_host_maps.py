"""Host-only ABI functions of the output coordinate map: Eq. 17 and the
paper's fixed-point inverse (Section 4, the second Eq. 18), against the
oracle's pinned implementations, exact and with the polynomial surrogate."""
import numpy as np
import pytest

import oracle


def _nf():
    from paper_2410_13474_gb300 import build
    build.build()
    import paper_2410_13474_gb300 as m
    return m


CASES = [(532e-9, 0.307e-6, 0.8), (500e-9, 0.5e-6, 1.0), (640e-9, 0.5e-6, 0.5)]


@pytest.mark.parametrize("poly", [False, True])
@pytest.mark.parametrize("lam,pitch,z", CASES)
def test_output_map_and_inverse_match_oracle(lam, pitch, z, poly):
    nf = _nf()
    B = 2 * z * np.tan(np.arcsin(lam / (2 * pitch)))
    rng = np.random.default_rng(11)
    pts = rng.uniform(-0.5 * B, 0.5 * B, (40, 2))
    pts[0] = (0.0, 0.0)
    pts[1] = (0.3 * B, 0.0)
    flags = nf.FLAG_PAPER_POLY_M if poly else 0
    for xo, yo in pts:
        got = nf.output_map(lam, pitch, 1024, z, xo, yo, flags)
        gi = nf.output_map_inverse(lam, pitch, 1024, z, got[0], got[1], 4, flags)
        if poly:
            with oracle.paper_poly(lam, pitch):
                ref = oracle.output_map(lam, z, xo, yo)
                ri = oracle.output_map_iterative_inverse(lam, z, ref[0], ref[1], 4)
        else:
            ref = oracle.output_map(lam, z, xo, yo)
            ri = oracle.output_map_iterative_inverse(lam, z, ref[0], ref[1], 4)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15 * B)
        assert np.allclose(gi, ri, rtol=1e-11, atol=1e-14 * B)


def test_inverse_converges_to_the_forward_map():
    """Many steps of the iteration invert Eq. 17 (where it converges), and
    one step is the identity x_o(1) = x_o'."""
    nf = _nf()
    lam, pitch, z = 500e-9, 0.5e-6, 1.0
    xo, yo = 0.31, -0.12
    xp, yp = nf.output_map(lam, pitch, 1024, z, xo, yo)
    assert nf.output_map_inverse(lam, pitch, 1024, z, xp, yp, 1) == (xp, yp)
    x, y = nf.output_map_inverse(lam, pitch, 1024, z, xp, yp, 200)
    assert abs(x - xo) < 1e-9 and abs(y - yo) < 1e-9


def test_output_map_arguments():
    nf = _nf()
    for bad in [dict(z=0.0), dict(z=-1.0)]:
        with pytest.raises(nf.NufdsError) as e:
            nf.output_map(500e-9, 0.5e-6, 1024, bad["z"], 0.1, 0.1)
        assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError) as e:
        nf.output_map_inverse(500e-9, 0.5e-6, 1024, 1.0, 0.1, 0.1, 0)
    assert e.value.code == nf.EINVAL
    with pytest.raises(nf.NufdsError) as e:
        nf.output_map(1.2e-6, 0.5e-6, 1024, 1.0, 0.1, 0.1)
    assert e.value.code == nf.EINVAL
