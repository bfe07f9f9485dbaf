"""Pins of the oracle's alm2map / map2alm against a dense synthesis matrix
built from scipy's spherical harmonics (independent of wf_oracle.c)."""
import math

import numpy as np
import pytest

from oracle import dense as D
from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I


@pytest.mark.parametrize("nside,lmax", [(1, 2), (2, 6), (4, 8), (4, 13), (8, 16)])
def test_alm2map_vs_dense(nside, lmax):
    """Includes lmax >= nphi/2 on the polar rings, where m aliases."""
    rng = np.random.default_rng(nside * 100 + lmax)
    z, phi = I.pixel_centres(nside)
    Y = D.synthesis_matrix(z, phi, lmax)
    alm = I.draw_alm(np.ones(lmax + 1), rng)
    f = O.alm2map(nside, lmax, alm)
    ref = Y @ D.pack(alm, lmax)
    assert np.allclose(f, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("nside,lmax", [(1, 2), (2, 6), (4, 8), (4, 13), (8, 16)])
def test_map2alm_vs_dense(nside, lmax):
    rng = np.random.default_rng(nside * 7 + lmax)
    z, phi = I.pixel_centres(nside)
    Y = D.synthesis_matrix(z, phi, lmax)
    Yd = D.adjoint_matrix(Y, lmax, z.size)
    f = rng.standard_normal(z.size)
    a = O.map2alm(nside, lmax, f)
    ref = D.unpack(Yd @ f, lmax)
    assert np.allclose(a, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("nside,lmax", [(8, 24), (16, 32)])
def test_adjointness(nside, lmax):
    """Omega <Y a, f> = <a, Y^dagger f> with the real-field inner product."""
    rng = np.random.default_rng(3)
    a = I.draw_alm(np.ones(lmax + 1), rng)
    f = rng.standard_normal(12 * nside * nside)
    omega = 4 * math.pi / f.size
    lhs = omega * np.dot(O.alm2map(nside, lmax, a), f)
    b = O.map2alm(nside, lmax, f)
    rhs = np.sum(O.alm_weight(lmax) * (a.conj() * b).real)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_monopole_exact():
    """A constant map integrates exactly: a_00 = sqrt(4 pi) c, all other l = 0
    a_l0 from the equal-area quadrature of the monopole vanish for odd l."""
    nside, lmax = 8, 16
    a = O.map2alm(nside, lmax, np.full(12 * nside * nside, 2.5))
    assert a[0].real == pytest.approx(2.5 * math.sqrt(4 * math.pi), rel=1e-14)
    for l in range(1, lmax + 1, 2):
        assert abs(a[O.alm_index(lmax, l, 0)]) < 1e-13


def test_quadrature_is_nearly_orthogonal():
    """Y^dagger Y is close to (but not exactly) the identity at low l: the
    reason the discrete messenger fixed point differs slightly from Eq. 2."""
    nside, lmax = 16, 16
    rng = np.random.default_rng(5)
    a = I.draw_alm(np.ones(lmax + 1), rng)
    back = O.map2alm(nside, lmax, O.alm2map(nside, lmax, a))
    err = O.rel_l2(back, a, lmax)
    assert 1e-8 < err < 5e-2


@pytest.mark.parametrize("nside,lmax", [(4, 8), (16, 40)])
def test_partial_evaluations(nside, lmax):
    """The pixel-wise synthesis and the mode-wise analysis used for sampled
    checks at large sizes agree with the full transforms."""
    rng = np.random.default_rng(11)
    a = I.draw_alm(np.ones(lmax + 1), rng)
    f = O.alm2map(nside, lmax, a)
    pix = rng.integers(0, f.size, 50)
    assert np.allclose(O.alm2map_pixels(nside, lmax, a, pix), f[pix], rtol=0, atol=1e-12)
    g = rng.standard_normal(f.size)
    b = O.map2alm(nside, lmax, g)
    idx = rng.integers(0, b.size, 40)
    ls, ms = O.l_of_index(lmax)[idx], O.m_of_index(lmax)[idx]
    assert np.allclose(O.map2alm_modes(nside, lmax, g, ls, ms), b[idx], rtol=0, atol=1e-13)
