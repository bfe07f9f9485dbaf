"""Pins of the oracle's several-messenger-field iteration (Sect. 4: more than
one messenger field for a joint analysis of several observations) against
the single-field iteration, the dense joint Wiener filter and the
inverse-variance combination of maps that share a beam."""
import math

import numpy as np
import pytest

from oracle import dense as D
from oracle import multi as MU
from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I


def two_detectors(nside, lmax, seed, same_beam=False):
    rng = np.random.default_rng(seed)
    z, phi = I.pixel_centres(nside)
    npix = z.size
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1)
    cl[2:] = 1.0 / (l * (l + 1.0))
    ell = np.arange(lmax + 1)
    beams = [np.exp(-0.5 * ell * (ell + 1) * 0.02 ** 2), np.exp(-0.5 * ell * (ell + 1) * 0.08 ** 2)]
    if same_beam:
        beams[1] = beams[0].copy()
    var = [2e-3 * (1 + 3 * rng.random(npix)), 5e-3 * (1 + rng.random(npix))]
    masks = [(np.abs(z) > 0.3).astype(np.uint8), (z > -0.5).astype(np.uint8)]
    a = I.draw_alm(cl, rng)
    ds = [O.alm2map(nside, lmax, b[O.l_of_index(lmax)] * a) + rng.standard_normal(npix) * np.sqrt(v)
          for b, v in zip(beams, var)]
    return cl, beams, var, masks, ds, z, phi


def dense_joint_wf(nside, lmax, cl, beams, noise_vars, masks, ds, lam=1.0):
    """(D S^-1 + sum_k B_k Y^T W_k Y B_k) x = sum_k B_k Y^T W_k d_k on the real degrees of
    freedom with C_l > 0, W_k the inverse of N_k + (lambda - 1) tau_k (0 where masked)."""
    z, phi = I.pixel_centres(nside)
    Y = D.synthesis_matrix(z, phi, lmax)
    cl_dof, wgt, l_dof = cl[D.dof_l(lmax)], D.dof_weight(lmax), D.dof_l(lmax)
    good = cl_dof > 0
    A = np.diag(wgt[good] / cl_dof[good])
    rhs = np.zeros(good.sum())
    for b, v, m, d in zip(beams, noise_vars, masks, ds):
        tau = O.messenger_tau(v, m)
        w = np.where(m != 0, 1.0 / (np.where(m != 0, v, 1.0) + (lam - 1.0) * tau), 0.0)
        YB = Y[:, good] * b[l_dof][good][None, :]
        A += YB.T @ (w[:, None] * YB)
        rhs += YB.T @ (w * d)
    x = np.zeros(Y.shape[1])
    x[good] = np.linalg.solve(A, rhs)
    return D.unpack(x, lmax)


def test_one_detector_with_unit_beam_is_the_single_field_iteration():
    p = I.small_problem(seed=4, nside=8, lmax=16)
    d = p.data(O.alm2map(8, 16, p.alm_true))
    opts = O.Options(tol=1e-6, max_iter=5000, band_limit=False)
    single = O.solve(8, 16, p.cl, p.noise_var, p.mask, d, opts)
    multi = MU.solve_multi(8, 16, p.cl, [np.ones(17)], [p.noise_var], [p.mask], [d], opts)
    assert multi.iters == single.iters and multi.converged
    assert [h["lam"] for h in multi.history] == [h["lam"] for h in single.history]
    assert O.rel_l2(multi.alm, single.alm, 16) < 1e-12
    for hm, hs in zip(multi.history, single.history):
        assert hm["chi2"] == pytest.approx(hs["chi2"], rel=1e-12)


@pytest.mark.parametrize("lam", [1.0, 20.0])
def test_fixed_point_is_dense_joint_wiener_filter(lam):
    """Converged iterates at fixed lambda equal the dense joint Wiener filter of
    the two maps (different beams, masks and noise) with noise N_k + (lambda - 1) T_k."""
    nside, lmax = 4, 8
    cl, beams, var, masks, ds, z, phi = two_detectors(nside, lmax, 3)
    ref = dense_joint_wf(nside, lmax, cl, beams, var, masks, ds, lam)
    res = MU.solve_multi(nside, lmax, cl, beams, var, masks, ds, schedule=[(lam, 3000)])
    assert O.rel_l2(res.alm, ref, lmax) < 1e-10
    inc = [h["rel_incr"] for h in res.history]
    assert inc[-1] < 1e-12 and inc[200] < inc[20]            # geometric convergence


def test_chi2_lambda_monotone_within_level():
    nside, lmax = 8, 16
    cl, beams, var, masks, ds, z, phi = two_detectors(nside, lmax, 5)
    for lam in (1.0, 50.0):
        res = MU.solve_multi(nside, lmax, cl, beams, var, masks, ds, schedule=[(lam, 60)])
        c = np.array([h["chi2_lambda"] for h in res.history])
        assert np.all(np.diff(c) <= 1e-12 * c[1:]), np.diff(c).max()


def test_shared_beam_equals_inverse_variance_combination():
    """Two maps with the same beam carry the information of their
    inverse-variance combination: the joint filter equals the single-map
    filter of w = w_1 + w_2, d = (w_1 d_1 + w_2 d_2) / w (masked where neither
    observes), by the cooled solve with its default schedule."""
    nside, lmax = 8, 16
    cl, beams, var, masks, ds, z, phi = two_detectors(nside, lmax, 7, same_beam=True)
    w = [O.inverse_noise(v, m) for v, m in zip(var, masks)]
    wsum = w[0] + w[1]
    obs = wsum > 0
    dcomb = np.where(obs, (w[0] * ds[0] + w[1] * ds[1]) / np.where(obs, wsum, 1.0), 0.0)
    vcomb = np.where(obs, 1.0 / np.where(obs, wsum, 1.0), 1.0)
    clb = cl * beams[0] ** 2     # the single-map solve has the beam folded into C_l
    opts = O.Options(tol=1e-12, max_iter=20000, band_limit=False)
    single = O.solve(nside, lmax, clb, vcomb, obs.astype(np.uint8), dcomb, opts)
    multi = MU.solve_multi(nside, lmax, cl, beams, var, masks, ds, opts)
    assert multi.converged and multi.history[-1]["lam"] == 1.0
    b = beams[0][O.l_of_index(lmax)]
    assert O.rel_l2(b * multi.alm, single.alm, lmax, cl=cl) < 1e-9
