"""Pins of the oracle's HEALPix RING geometry (and of the input generator's
copy of it) against facts fixed by the pixelisation's definition."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "healpix_pixel_centres.txt")


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64, 512])
def test_ring_counts_and_equal_area(nside):
    """4 Nside - 1 rings whose lengths add up to Npix; the spherical cap above
    each ring's centre latitude holds exactly (pixels above + half the ring)
    pixels of area Omega -- the equal-area, iso-latitude property that fixes
    the ring latitudes."""
    npix = 12 * nside * nside
    omega = 4 * math.pi / npix
    total = 0
    prev_off = 0
    for r in range(4 * nside - 1):
        z, nphi, phi0, off = O.ring_info(nside, r)
        assert off == prev_off
        prev_off = off + nphi
        total += nphi
        cap = 2 * math.pi * (1.0 - z)
        assert cap == pytest.approx((off + nphi / 2) * omega, rel=1e-13, abs=1e-13)
        # the ring lengths: 4i in the caps, 4 Nside in the belt
        i = r + 1
        ip = min(i, 4 * nside - i)
        assert nphi == 4 * min(ip, nside)
    assert total == npix
    with pytest.raises(RuntimeError):
        O.ring_info(nside, 4 * nside - 1)


def test_golden_pixel_centres():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for ns, p, th, ph in rows:
        ns, p, th, ph = int(ns), int(p), float(th), float(ph)
        z, phi = O.pixel_angles(ns)
        digits = 1e-12 if len(str(th)) > 12 else 1e-8
        assert math.acos(z[p]) == pytest.approx(th, abs=digits)
        assert phi[p] == pytest.approx(ph, abs=digits)


@pytest.mark.parametrize("nside", [1, 2, 8, 32])
def test_symmetries(nside):
    """North/south mirror symmetry, uniform azimuth spacing, and the half-pixel
    shift rule (cap rings and every other belt ring are shifted)."""
    z, phi = O.pixel_angles(nside)
    npix = z.size
    # RING order of the south hemisphere mirrors the north ring by ring
    for r in range(2 * nside - 1):
        zn, nn, pn, on = O.ring_info(nside, r)
        zs, ns_, ps, os_ = O.ring_info(nside, 4 * nside - 2 - r)
        assert zs == pytest.approx(-zn, abs=1e-15) and nn == ns_ and pn == ps
    for r in range(4 * nside - 1):
        zr, n, p0, off = O.ring_info(nside, r)
        d = np.diff(phi[off:off + n])
        assert np.allclose(d, 2 * math.pi / n, rtol=0, atol=1e-13)
        i = min(r + 1, 4 * nside - r - 1)
        if i < nside:
            assert p0 == pytest.approx(math.pi / n)
        else:
            shifted = ((r + 1 - nside) % 2 == 0)
            assert p0 == pytest.approx(math.pi / n if shifted else 0.0)
    assert z.size == npix


@pytest.mark.parametrize("nside", [1, 4, 16])
def test_generator_geometry_matches(nside):
    """The input generator's own pixel centres agree with the oracle's."""
    z1, p1 = O.pixel_angles(nside)
    z2, p2 = I.pixel_centres(nside)
    assert np.array_equal(z1, z2)
    assert np.allclose(p1, p2, rtol=0, atol=1e-13)
