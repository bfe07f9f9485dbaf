"""Constrained realisations on the device (Sect. 3: Wiener filter plus a
fluctuation map, with the correct signal variance) against the oracle's, on
the same counter-based draws, and their statistics."""
import math

import numpy as np
import pytest

from oracle import cr as CR
from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I
from paper_1211_0585_gb300 import wf

from gpu_util import FP64_PATHS, problem

pytestmark = pytest.mark.gpu


def oracle_cr(p, d, nreal, seed, opts):
    """The oracle's realisations from the same draws: (cr list, s_WF(d), s_WF of each fluctuation map)."""
    wf_d = O.solve(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, O.Options(**opts)).alm
    crs, sols = [], []
    for i in range(nreal):
        xi = CR.draw_signal(seed, i, p.lmax, p.cl)
        n = CR.draw_noise(seed, i, p.noise_var, p.mask)
        sol = O.solve(p.nside, p.lmax, p.cl, p.noise_var, p.mask, O.alm2map(p.nside, p.lmax, xi) + n,
                      O.Options(**opts)).alm
        crs.append(wf_d + xi - sol)
        sols.append(sol)
    return crs, wf_d, sols


@pytest.mark.parametrize("prec", ["fp64-table", "fp64-native"])
def test_fp64_realisations_match_oracle(prec):
    nside, lmax, nreal, seed = 16, 32, 3, 2024
    p, d = problem("wmap-cooled", seed=21, nside=nside, lmax=lmax)
    opts = dict(tol=1e-8, max_iter=4000)
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec], **opts))
    cr, wf_d, stats, status = P.constrained_realisations(d, nreal, seed)
    assert status == wf.WF_OK and len(stats) == nreal + 1
    ref, ref_wf, _ = oracle_cr(p, d, nreal, seed, opts)
    assert O.rel_l2(wf_d, ref_wf, lmax) < 1e-10
    for i in range(nreal):
        assert O.rel_l2(cr[i], ref[i], lmax) < 1e-10, i


def test_mixed_realisations_match_oracle():
    """Seven realisations and d in one batch of the mixed engine. Each part
    (s_WF(d), s_WF of the fluctuation map) is within the mixed bar plus one
    increment of the oracle's, so the realisation is within that bar of the
    sum of their sizes."""
    nside, lmax, nreal, seed = 16, 32, 7, 77
    p, d = problem("wmap-cooled", seed=22, nside=nside, lmax=lmax)
    opts = dict(tol=1e-6, max_iter=4000)
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask,
                wf.options(precision=wf.WF_PREC_MIXED, batch_slots=8, **opts))
    cr, wf_d, stats, status = P.constrained_realisations(d, nreal, seed)
    assert status == wf.WF_OK
    ref, ref_wf, sols = oracle_cr(p, d, nreal, seed, opts)
    bar = 1e-6 + 2 * opts["tol"]
    wgt = O.alm_weight(lmax)
    norm = lambda a: math.sqrt(float(np.sum(wgt * np.abs(a) ** 2)))
    assert O.rel_l2(wf_d, ref_wf, lmax) < bar
    for i in range(nreal):
        assert norm(cr[i] - ref[i]) <= bar * (norm(ref_wf) + norm(sols[i])), i


def test_realisations_carry_prior_power_where_data_do_not():
    """Over data drawn from the model (8 maps, 7 realisations each, mixed
    engine): at high l, where noise dominates, the realisations' power per l
    is C_l within sampling error while the Wiener filter's falls well short;
    in the masked pixels the realisations' variance is the prior pixel
    variance sum_l (2l + 1) C_l / 4 pi while the Wiener filter's is smaller."""
    nside, lmax, nreal = 32, 64, 7
    p0 = I.wmap_problem(seed=23, nside=nside, lmax=lmax, ndisc=5, noise_scale=(nside / 512.0) ** 2)
    P = wf.Plan(nside, lmax, p0.cl, p0.noise_var, p0.mask,
                wf.options(precision=wf.WF_PREC_MIXED, batch_slots=8, tol=1e-6, max_iter=4000))
    rng = np.random.default_rng(5)
    ls, ms = O.l_of_index(lmax), O.m_of_index(lmax)
    wgt = np.where(ms == 0, 1.0, 2.0)
    p_cr, p_wf = np.zeros(lmax + 1), np.zeros(lmax + 1)
    masked = p0.mask == 0
    v_cr = v_wf = 0.0
    ndata = 8
    for k in range(ndata):
        a = I.draw_alm(p0.cl, rng)
        d = O.alm2map(nside, lmax, a) + rng.standard_normal(p0.npix) * np.sqrt(p0.noise_var)
        cr, wf_d, _, status = P.constrained_realisations(d, nreal, seed=1000 + k)
        assert status == wf.WF_OK
        for i in range(nreal):
            p_cr += np.bincount(ls, weights=wgt * np.abs(cr[i]) ** 2, minlength=lmax + 1)
            v_cr += float(np.mean(O.alm2map(nside, lmax, cr[i])[masked] ** 2))
        p_wf += nreal * np.bincount(ls, weights=wgt * np.abs(wf_d) ** 2, minlength=lmax + 1)
        v_wf += nreal * float(np.mean(O.alm2map(nside, lmax, wf_d)[masked] ** 2))
    n = ndata * nreal
    band = np.arange(48, lmax + 1)
    nmode = 2 * band + 1
    r_cr = np.sum(p_cr[band] / n) / np.sum(nmode * p0.cl[band])
    r_wf = np.sum(p_wf[band] / n) / np.sum(nmode * p0.cl[band])
    assert abs(r_cr - 1.0) < 0.1, r_cr
    assert r_wf < 0.75, r_wf
    prior_var = float(np.sum((2 * np.arange(lmax + 1) + 1) * p0.cl) / (4 * math.pi))
    assert 0.75 < v_cr / n / prior_var < 1.33, v_cr / n / prior_var
    assert v_wf / n < 0.8 * v_cr / n
