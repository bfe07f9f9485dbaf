"""Pins of the oracle's temperature-polarisation filter (Sect. 4: the method
on T and P maps together): the spin-2 functions against the spin-raising
operator's definition and their orthonormality and addition theorem, the
transform pair's adjointness and E/B rotation structure, and the iteration
against the dense joint (T, E, B) Wiener filter and the temperature-only
iteration."""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import dense as D
from oracle import oracle as O
from oracle import pol as PO
from paper_1211_0585_gb300 import inputs as I


def test_spin2_functions_match_eth_definition():
    """_+-2 lambda from eth^2 / eth-bar^2 of Y_lm (finite differences of
    scipy's spherical harmonics in theta): F+ + F- and F+ - F-."""
    h = 1e-3
    for l, m in [(2, 0), (3, 1), (5, 2), (6, 5), (8, 3), (9, 9)]:
        nl = 1.0 / math.sqrt((l - 1.0) * l * (l + 1.0) * (l + 2.0))
        for th in (0.4, 1.1, 2.2):
            f = lambda t: sph_harm_y(l, m, t, 0.0).real
            v = [f(th + k * h) for k in (-2, -1, 0, 1, 2)]
            d1 = (v[0] - 8 * v[1] + 8 * v[3] - v[4]) / (12 * h)
            d2 = (-v[0] + 16 * v[1] - 30 * v[2] + 16 * v[3] - v[4]) / (12 * h * h)
            x, s = math.cos(th), math.sin(th)
            eth2 = d2 - (2 * m + x) * d1 / s + (2 * m * x + m * m) * v[2] / (s * s)
            ethb2 = d2 + (2 * m - x) * d1 / s + (m * m - 2 * m * x) * v[2] / (s * s)
            fp, fm = PO.spin2_functions(l, m, x)
            assert fp[l] + fm[l] == pytest.approx(nl * eth2, abs=1e-6)
            assert fp[l] - fm[l] == pytest.approx(nl * ethb2, abs=1e-6)


@pytest.mark.parametrize("x", [0.95, 0.3, -0.7])
def test_spin2_addition_theorem(x):
    """sum over m = -l .. l of |_2 Y_lm|^2 = (2 l + 1) / 4 pi (negative m carry _-2 lambda)."""
    lmax = 60
    acc = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        fp, fm = PO.spin2_functions(lmax, m, x)
        acc += fp ** 2 if m == 0 else 2.0 * (fp ** 2 + fm ** 2)
    l = np.arange(2, lmax + 1)
    assert np.allclose(acc[2:], (2 * l + 1) / (4 * math.pi), rtol=1e-12, atol=0)


def test_spin2_orthonormal():
    """2 pi int _2 lambda_lm _2 lambda_l'm dx = delta_ll' (Gauss-Legendre quadrature, exact here)."""
    lmax = 24
    xs, ws = np.polynomial.legendre.leggauss(64)
    for m in (0, 1, 4, 11):
        F = np.array([PO.spin2_functions(lmax, m, x) for x in xs])       # [node][+-][l]
        sp = F[:, 0, :] + F[:, 1, :]
        G = 2 * math.pi * (sp * ws[:, None]).T @ sp
        l0 = max(2, m)
        assert np.allclose(G[l0:, l0:], np.eye(lmax + 1 - l0), atol=1e-12)


def rand_alm3(lmax, rng):
    a = np.array([I.draw_alm(np.ones(lmax + 1), rng) for _ in range(3)])
    a[1:, O.l_of_index(lmax) < 2] = 0.0
    return a


@pytest.mark.parametrize("nside,lmax", [(4, 8), (8, 12)])
def test_transforms_adjoint(nside, lmax):
    """<Y a, f> Omega = <a, Y^dagger f> over (T, Q, U) and (T, E, B), m > 0 counted twice."""
    rng = np.random.default_rng(nside + lmax)
    a = rand_alm3(lmax, rng)
    f = rng.standard_normal((3, 12 * nside * nside))
    omega = 4 * math.pi / f.shape[1]
    lhs = float(np.sum(PO.pol_alm2map(nside, lmax, a) * f)) * omega
    b = PO.pol_map2alm(nside, lmax, f)
    wgt = O.alm_weight(lmax)
    rhs = float(sum(np.sum(wgt * (np.conj(a[i]) * b[i]).real) for i in range(3)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_rotating_q_u_swaps_e_and_b():
    """(Q, U) -> (U, -Q) (a 45 degree rotation of the polarisation basis) maps (E, B) -> (B, -E)."""
    nside, lmax = 8, 16
    rng = np.random.default_rng(3)
    f = rng.standard_normal((3, 12 * nside * nside))
    a = PO.pol_map2alm(nside, lmax, f)
    g = np.array([f[0], f[2], -f[1]])
    b = PO.pol_map2alm(nside, lmax, g)
    assert np.allclose(b[1], a[2], atol=1e-14) and np.allclose(b[2], -a[1], atol=1e-14)
    x = PO.pol_alm2map(nside, lmax, np.array([a[0], a[2], -a[1]]))
    y = PO.pol_alm2map(nside, lmax, a)
    assert np.allclose(x[1], y[2], atol=1e-13) and np.allclose(x[2], -y[1], atol=1e-13)


def pol_problem(nside, lmax, seed, noise=2e-3):
    rng = np.random.default_rng(seed)
    z, phi = I.pixel_centres(nside)
    npix = z.size
    l = np.arange(lmax + 1, dtype=float)
    tt = np.where(l >= 2, 1.0 / np.maximum(l * (l + 1), 1.0), 0.0)
    ee = 0.1 * tt
    bb = 0.02 * tt
    te = 0.5 * np.sqrt(tt * ee)
    nz = np.zeros((npix, 4))
    nz[:, 0] = noise * (1 + rng.random(npix))
    nz[:, 1] = 2 * noise * (1 + rng.random(npix))
    nz[:, 3] = 2 * noise * (1 + rng.random(npix))
    nz[:, 2] = 0.3 * np.sqrt(nz[:, 1] * nz[:, 3]) * rng.uniform(-1, 1, npix)
    mt = (np.abs(z) > 0.25).astype(np.uint8)
    mp = (np.abs(z) > 0.4).astype(np.uint8)
    # signal with the TE correlation: a_T = sqrt(TT) g1, a_E = TE / sqrt(TT) g1 + sqrt(EE - TE^2 / TT) g2
    g1, g2, g3 = (I.draw_alm(np.ones(lmax + 1), rng) for _ in range(3))
    ls = O.l_of_index(lmax)
    sq = lambda v: np.sqrt(np.maximum(v, 0.0))
    aT = sq(tt[ls]) * g1
    aE = np.where(tt[ls] > 0, te[ls] / sq(np.where(tt[ls] > 0, tt[ls], 1.0)), 0.0) * g1 + \
        sq(ee[ls] - np.where(tt[ls] > 0, te[ls] ** 2 / np.where(tt[ls] > 0, tt[ls], 1.0), 0.0)) * g2
    aB = sq(bb[ls]) * g3
    d = PO.pol_alm2map(nside, lmax, np.array([aT, aE, aB]))
    # noise with the per-pixel covariance
    d[0] += rng.standard_normal(npix) * np.sqrt(nz[:, 0])
    L11 = np.sqrt(nz[:, 1])
    L21 = nz[:, 2] / L11
    L22 = np.sqrt(nz[:, 3] - L21 ** 2)
    e1, e2 = rng.standard_normal(npix), rng.standard_normal(npix)
    d[1] += L11 * e1
    d[2] += L21 * e1 + L22 * e2
    return (tt, ee, bb, te), nz, mt, mp, d


def dense_pol_wf(nside, lmax, cls, nz, mt, mp, d, lam=1.0):
    """(S^-1 + Y^T W_lam Y) x = Y^T W_lam d on the real degrees of freedom, Y the oracle's
    (T, E, B) -> (T, Q, U) synthesis applied to unit vectors, W_lam = (N + (lambda - 1) tau)^-1."""
    npix = 12 * nside * nside
    dof = D.dof_lm(lmax)
    nd = len(dof)
    cols = []
    for f in range(3):
        for j in range(nd):
            x = np.zeros(nd)
            x[j] = 1.0
            a = np.zeros((3, O.nalm_of(lmax)), dtype=np.complex128)
            a[f] = D.unpack(x, lmax)
            cols.append(PO.pol_alm2map(nside, lmax, a).reshape(-1))
    Y = np.array(cols).T                                     # [3 npix][3 nd]
    tau = PO.messenger_tau_pol(nz, mt, mp)
    c = (lam - 1.0) * tau
    W = np.zeros((3 * npix, 3 * npix))
    w = PO.inverse_noise_pol(nz, mt, mp)
    for p in range(npix):
        Wp = np.array([[w[p, 0], 0, 0], [0, w[p, 1], w[p, 2]], [0, w[p, 2], w[p, 3]]])
        Gp = Wp @ np.linalg.inv(np.eye(3) + c * Wp)
        idx = [p, npix + p, 2 * npix + p]
        W[np.ix_(idx, idx)] = Gp
    tt, ee, bb, te = cls
    ld = np.array([l for (l, _, _) in dof])
    wgt = D.dof_weight(lmax)
    Sinv = np.zeros((3 * nd, 3 * nd))
    for j in range(nd):
        l = ld[j]
        blk = np.array([[tt[l], te[l]], [te[l], ee[l]]])
        if tt[l] > 0 and ee[l] > 0:
            iv = np.linalg.inv(blk) * wgt[j]
            Sinv[np.ix_([j, nd + j], [j, nd + j])] = iv
        elif tt[l] > 0:
            Sinv[j, j] = wgt[j] / tt[l]
        if bb[l] > 0:
            Sinv[2 * nd + j, 2 * nd + j] = wgt[j] / bb[l]
    good = np.diag(Sinv) > 0
    A = Sinv[np.ix_(good, good)] + Y[:, good].T @ W @ Y[:, good]
    x = np.zeros(3 * nd)
    x[good] = np.linalg.solve(A, Y[:, good].T @ W @ d.reshape(-1))
    return np.array([D.unpack(x[f * nd:(f + 1) * nd], lmax) for f in range(3)])


@pytest.mark.parametrize("lam", [1.0, 8.0])
def test_fixed_point_is_dense_pol_wiener_filter(lam):
    nside, lmax = 4, 8
    cls, nz, mt, mp, d = pol_problem(nside, lmax, 5)
    ref = dense_pol_wf(nside, lmax, cls, nz, mt, mp, d, lam)
    res = PO.solve_pol(nside, lmax, cls, nz, mt, mp, d, schedule=[(lam, 2500)])
    for f in range(3):
        assert O.rel_l2(res.alm[f], ref[f], lmax) < 1e-9, f
    assert res.history[-1]["rel_incr"] < 1e-12


def test_chi2_lambda_monotone_within_level():
    nside, lmax = 8, 16
    cls, nz, mt, mp, d = pol_problem(nside, lmax, 6)
    for lam in (1.0, 40.0):
        res = PO.solve_pol(nside, lmax, cls, nz, mt, mp, d, schedule=[(lam, 40)])
        c = np.array([h["chi2_lambda"] for h in res.history])
        assert np.all(np.diff(c) <= 1e-12 * c[1:]), np.diff(c).max()


def test_temperature_only_limit_is_the_scalar_iteration():
    """With every polarisation pixel masked and C_TE = 0, the temperature part is
    the scalar messenger iteration of the T map, and E, B stay zero."""
    nside, lmax = 8, 16
    cls, nz, mt, mp, d = pol_problem(nside, lmax, 7)
    cls = (cls[0], cls[1], cls[2], np.zeros(lmax + 1))
    opts = O.Options(tol=1e-7, max_iter=3000, band_limit=False)
    res = PO.solve_pol(nside, lmax, cls, nz, mt, np.zeros_like(mp), d, opts)
    ref = O.solve(nside, lmax, cls[0], nz[:, 0], mt, d[0], opts)
    assert res.iters == ref.iters
    assert O.rel_l2(res.alm[0], ref.alm, lmax) < 1e-12
    assert np.all(res.alm[1:] == 0)
