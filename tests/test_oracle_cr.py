"""Pins of the oracle's constrained realisations (Sect. 3, WMAP analysis, and
the power-spectra figure: a Wiener-filter map plus a fluctuation map is a
constrained realisation with the correct signal variance) and of its
counter-based random numbers."""
import math

import numpy as np
import pytest

from oracle import cr as CR
from oracle import dense as D
from oracle import oracle as O

from test_oracle_messenger import dense_setup, tiny_problem


@pytest.mark.parametrize("key,ctr", [((5, 7), (1, 0, 0, 0)), ((2 ** 64 - 3, 12345), (99, 1, 3, 0)),
                                     ((0, 0), (7, 0, 63, 0))])
def test_philox_matches_numpy_bit_generator(key, ctr):
    """Philox4x64-10 from its published definition against numpy's own
    implementation of the same generator (numpy advances its 256-bit counter
    before each block, so it is started one below)."""
    start = np.array([ctr[0] - 1, ctr[1], ctr[2], ctr[3]], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    ref = bg.random_raw(12).reshape(3, 4)
    ctrs = np.array([[ctr[0] + j, ctr[1], ctr[2], ctr[3]] for j in range(3)], dtype=np.uint64)
    got = CR.philox4x64(ctrs, key)
    assert np.array_equal(got, ref)


def test_normals_are_standard():
    """Box-Muller normals of one stream: mean 0, variance 1, Gaussian
    (Kolmogorov-Smirnov), and independent streams for other kinds/realisations."""
    from scipy import stats
    z = CR.normals(11, 0, 0, 400000)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    other = CR.normals(11, 1, 0, 1000), CR.normals(11, 0, 1, 1000), CR.normals(12, 0, 0, 1000)
    for o in other:
        assert abs(np.corrcoef(z[:1000], o)[0, 1]) < 0.2


def test_signal_draws_have_prior_power():
    """xi ~ N(0, S): averaged over realisations, |a_lm|^2 = C_l for every l
    (m > 0 counted twice, the imaginary part of m = 0 zero)."""
    lmax, nreal = 12, 400
    cl = np.zeros(lmax + 1)
    cl[2:] = 1.0 / np.arange(2, lmax + 1) ** 2
    ls, ms = O.l_of_index(lmax), O.m_of_index(lmax)
    wgt = np.where(ms == 0, 1.0, 2.0)
    acc = np.zeros(lmax + 1)
    for i in range(nreal):
        xi = CR.draw_signal(3, i, lmax, cl)
        assert np.all(xi[ms == 0].imag == 0.0)
        acc += np.bincount(ls, weights=wgt * np.abs(xi) ** 2, minlength=lmax + 1)
    power = acc / (nreal * (2 * np.arange(lmax + 1) + 1))
    for l in range(2, lmax + 1):
        assert abs(power[l] / cl[l] - 1) < 5 * math.sqrt(2.0 / (nreal * (2 * l + 1)))
    assert np.all(power[:2] == 0)


def test_noise_draws_follow_pixel_variance():
    var = np.linspace(0.5, 3.0, 200)
    mask = np.ones(200, np.uint8)
    mask[:20] = 0
    acc = np.zeros(200)
    for i in range(300):
        n = CR.draw_noise(5, i, var, mask)
        assert np.all(n[:20] == 0)
        acc += n * n
    ratio = acc[20:] / (300 * var[20:])
    assert abs(ratio.mean() - 1.0) < 5 * math.sqrt(2.0 / (300 * 180))


def test_zero_draws_give_the_wiener_filter():
    """With xi = 0 and n' = 0 the constrained realisation is s_WF(d) itself."""
    nside, lmax = 4, 8
    cl, var, mask, d, z, phi = tiny_problem(nside, lmax, 51, noise=1e-2)
    opts = O.Options(tol=1e-12, max_iter=20000, cooling=False)
    wf = O.solve(nside, lmax, cl, var, mask, d, opts).alm
    got = CR.constrained_realisation(nside, lmax, cl, var, mask, d, np.zeros_like(wf), np.zeros(d.size), opts)
    assert np.array_equal(got, wf)


def test_fluctuation_is_dense_posterior_fluctuation_with_prior_covariance():
    """The oracle's realisation minus the Wiener filter is xi - W (Y xi + n')
    with W the dense Eq. 2 solution operator; and with that W, the
    realisation's covariance over data drawn from the model,
        W Y S Y^T W^T + W N W^T + (1 - W Y) S (1 - W Y)^T + W N W^T,
    is the prior S on the modes with C_l > 0 (the correct signal variance)."""
    nside, lmax = 4, 8
    cl, var, mask, d, z, phi = tiny_problem(nside, lmax, 52, noise=1e-2)
    Y, Yd, f_dof, a_pix, w, tau, omega = dense_setup(nside, lmax, cl, var, mask, z, phi, 1.0)
    cl_dof, wgt = cl[D.dof_l(lmax)], D.dof_weight(lmax)
    good = cl_dof > 0
    Yg = Y[:, good]
    A = np.diag(wgt[good] / cl_dof[good]) + Yg.T @ (w[:, None] * Yg)
    Wg = np.linalg.solve(A, Yg.T * w[None, :])         # dense WF operator on the modes with C_l > 0
    opts = O.Options(tol=1e-13, max_iter=50000, cooling=False)
    xi = CR.draw_signal(9, 0, lmax, cl)
    n_prime = CR.draw_noise(9, 0, var, mask)
    wf = O.solve(nside, lmax, cl, var, mask, d, opts).alm
    got = CR.constrained_realisation(nside, lmax, cl, var, mask, d, xi, n_prime, opts, wf=wf) - wf
    x_xi = D.pack(xi, lmax)
    expect = x_xi.copy()
    expect[good] -= Wg @ (Y @ x_xi + n_prime)
    assert np.allclose(D.pack(got, lmax), expect, rtol=0, atol=1e-9 * np.abs(expect).max())
    # covariance identity (real degrees of freedom: Re / Im of m > 0 carry C_l / 2 each)
    Sg = np.diag(cl_dof[good] / wgt[good])
    Nd = np.diag(np.where(mask != 0, var, 0.0))
    WY = Wg @ Yg
    I = np.eye(WY.shape[0])
    cov = WY @ Sg @ WY.T + 2 * Wg @ Nd @ Wg.T + (I - WY) @ Sg @ (I - WY).T
    assert np.allclose(cov, Sg, rtol=0, atol=1e-10 * Sg.max())


def test_constrained_realisations_have_prior_power_in_masked_data():
    """Monte Carlo over data drawn from the model: the realisations' power per
    l matches C_l within sampling error, while the Wiener filter's alone falls
    short where the data are noise-dominated (its power is suppressed there)."""
    nside, lmax, ndraw = 4, 8, 100
    cl = np.zeros(lmax + 1)
    cl[2:] = 1.0 / (np.arange(2, lmax + 1) * np.arange(3, lmax + 2))
    rng = np.random.default_rng(61)
    z, phi = np.array(O.pixel_angles(nside)[0]), None
    npix = 12 * nside * nside
    var = np.full(npix, 0.05)
    mask = (np.abs(z) > 0.35).astype(np.uint8)
    opts = O.Options(tol=1e-7, max_iter=20000)
    ls, ms = O.l_of_index(lmax), O.m_of_index(lmax)
    wgt = np.where(ms == 0, 1.0, 2.0)
    p_cr, p_wf = np.zeros(lmax + 1), np.zeros(lmax + 1)
    from paper_1211_0585_gb300 import inputs as I
    for k in range(ndraw):
        a = I.draw_alm(cl, rng)
        d = O.alm2map(nside, lmax, a) + rng.standard_normal(npix) * np.sqrt(var)
        wf = O.solve(nside, lmax, cl, var, mask, d, opts).alm
        s = CR.constrained_realisation(nside, lmax, cl, var, mask, d, CR.draw_signal(1, k, lmax, cl),
                                       CR.draw_noise(1, k, var, mask), opts, wf=wf)
        p_cr += np.bincount(ls, weights=wgt * np.abs(s) ** 2, minlength=lmax + 1)
        p_wf += np.bincount(ls, weights=wgt * np.abs(wf) ** 2, minlength=lmax + 1)
    nmode = ndraw * (2 * np.arange(lmax + 1) + 1)
    ratio_cr = p_cr[2:] / nmode[2:] / cl[2:]
    ratio_wf = p_wf[2:] / nmode[2:] / cl[2:]
    err = np.sqrt(2.0 / nmode[2:])
    assert np.all(np.abs(ratio_cr - 1) < 5 * err), ratio_cr
    assert ratio_wf[-1] < 0.8, ratio_wf        # the Wiener filter alone loses power at high l
