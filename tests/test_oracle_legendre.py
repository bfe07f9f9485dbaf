"""Pins of the oracle's orthonormal associated Legendre functions."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre, sph_harm_y

from oracle import oracle as O


def closed_forms(theta):
    """Textbook Y_lm(theta, 0) for l <= 2 with the Condon-Shortley phase."""
    c, s = math.cos(theta), math.sin(theta)
    pi = math.pi
    return {
        (0, 0): 1 / math.sqrt(4 * pi),
        (1, 0): math.sqrt(3 / (4 * pi)) * c,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s,
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * c * c - 1),
        (2, 1): -math.sqrt(15 / (8 * pi)) * s * c,
        (2, 2): 0.25 * math.sqrt(15 / (2 * pi)) * s * s,
    }


@pytest.mark.parametrize("theta", [0.0, 0.1, 0.7, 1.3, math.pi / 2, 2.2, 3.0, math.pi])
def test_closed_forms(theta):
    x = math.cos(theta)
    for (l, m), v in closed_forms(theta).items():
        assert O.legendre(2, m, x)[l] == pytest.approx(v, rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("x", [0.999999, 0.95, 0.5, 0.0, -0.3, -0.99])
def test_against_scipy(x):
    theta = math.acos(x)
    lmax = 80
    for m in range(0, lmax + 1, 7):
        lam = O.legendre(lmax, m, x)
        ref = np.array([sph_harm_y(l, m, theta, 0.0).real if l >= m else 0.0 for l in range(lmax + 1)])
        assert np.allclose(lam, ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("x", [0.9999999, 0.8, 0.1, -0.6])
def test_m0_is_legendre_polynomial(x):
    """lambda_l0 = sqrt((2l+1)/(4 pi)) P_l at high l (scipy's P_l)."""
    lmax = 4096
    lam = O.legendre(lmax, 0, x)
    ls = np.arange(0, lmax + 1, 97)
    ref = np.sqrt((2 * ls + 1) / (4 * math.pi)) * eval_legendre(ls, x)
    assert np.allclose(lam[ls], ref, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("x", [0.99999997, 0.9999, 0.9, 0.3, 0.0, -0.75])
def test_addition_theorem_high_l(x):
    """sum_m (2 - delta_m0) lambda_lm(x)^2 = (2l+1)/(4 pi) for every l <= 4096.
    Near the pole this exercises the rescaled start value: sin^m(theta)
    underflows a double long before m = 4096."""
    lmax = 4096
    acc = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        lam = O.legendre(lmax, m, x)
        acc += (1.0 if m == 0 else 2.0) * lam * lam
    l = np.arange(lmax + 1)
    assert np.allclose(acc, (2 * l + 1) / (4 * math.pi), rtol=1e-10, atol=0)


def test_orthonormality_gauss_legendre():
    """2 pi int_{-1}^{1} lambda_lm lambda_l'm dx = delta_ll' (Gauss-Legendre nodes)."""
    lmax = 64
    xs, ws = np.polynomial.legendre.leggauss(lmax + 2)
    for m in (0, 1, 5, 31, 64):
        P = np.array([O.legendre(lmax, m, x) for x in xs])  # [node, l]
        G = 2 * math.pi * (P * ws[:, None]).T @ P
        sub = G[m:, m:]
        assert np.allclose(sub, np.eye(lmax + 1 - m), atol=1e-12)


@pytest.mark.parametrize("x", [0.9, 0.35])
def test_parity(x):
    """lambda_lm(-x) = (-1)^(l+m) lambda_lm(x)."""
    lmax = 200
    for m in (0, 3, 100, 200):
        a, b = O.legendre(lmax, m, x), O.legendre(lmax, m, -x)
        sign = np.array([(-1.0) ** (l + m) for l in range(lmax + 1)])
        assert np.allclose(b, sign * a, rtol=1e-13, atol=1e-300)


def test_pole_and_bad_args():
    lam = O.legendre(10, 3, 1.0)
    assert np.all(lam == 0.0)
    lam0 = O.legendre(10, 0, 1.0)
    assert np.allclose(lam0, np.sqrt((2 * np.arange(11) + 1) / (4 * math.pi)))
    with pytest.raises(RuntimeError):
        O.legendre(10, 11, 0.5)
    with pytest.raises(RuntimeError):
        O.legendre(10, 2, 1.5)
