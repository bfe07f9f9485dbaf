"""Several messenger fields on the device (Sect. 4: one messenger per
observation, combined in one analysis) against the oracle's iteration."""
import numpy as np
import pytest

from oracle import multi as MU
from oracle import oracle as O
from paper_1211_0585_gb300 import wf

from gpu_util import FP64_PATHS, problem
from test_oracle_multi import two_detectors

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.mark.parametrize("prec", list(FP64_PATHS))
@pytest.mark.parametrize("nside,lmax,l_iter0", [(8, 16, 4), (16, 32, 8)])
def test_two_detectors_match_oracle(nside, lmax, l_iter0, prec):
    """Two maps with different beams, masks and noise: the device controller
    takes the oracle's decisions (same lambda levels and iteration count) and
    the joint result matches within the FP64 bar, as do the chi^2 records."""
    cl, beams, var, masks, ds, z, phi = two_detectors(nside, lmax, 13)
    opts = dict(tol=1e-8, max_iter=4000, l_iter0=l_iter0)
    ores = MU.solve_multi(nside, lmax, cl, beams, var, masks, ds, O.Options(**opts, band_limit=False))
    assert ores.converged and len({h["lam"] for h in ores.history}) >= 2     # it cooled
    M = wf.Multi(nside, lmax, cl, var, masks, beams, wf.options(**FP64_PATHS[prec], **opts))
    alm, st, status, recs = M.solve(ds, history=opts["max_iter"] + 1)
    assert status == wf.WF_OK and st["iters"] == ores.iters
    assert [r["lam"] for r in recs] == pytest.approx([h["lam"] for h in ores.history], rel=1e-14)
    assert O.rel_l2(alm, ores.alm, lmax) < TOL
    for r, h in zip(recs, ores.history):
        assert r["chi2"] == pytest.approx(h["chi2"], rel=TOL)
    M.close()


def test_three_detectors_match_oracle():
    """Three maps (on the table form the maps' transforms run two per launch, the
    third alone): the joint result and the chi^2 records match the oracle's."""
    nside, lmax = 8, 16
    cl, beams, var, masks, ds, z, phi = two_detectors(nside, lmax, 17)
    rng = np.random.default_rng(18)
    ell = np.arange(lmax + 1)
    beams = beams + [np.exp(-0.5 * ell * (ell + 1) * 0.05 ** 2)]
    var = var + [3e-3 * (1 + rng.random(z.size))]
    masks = masks + [(z < 0.6).astype(np.uint8)]
    # the third map: the first one's sky (its data minus its noise) through the third beam, plus noise
    a_sky = O.map2alm(nside, lmax, ds[0])   # a noisy stand-in for the sky: any a_lm makes valid data
    ds = ds + [O.alm2map(nside, lmax, beams[2][O.l_of_index(lmax)] * a_sky) +
               rng.standard_normal(z.size) * np.sqrt(var[2])]
    opts = dict(tol=1e-8, max_iter=4000, l_iter0=4)
    ores = MU.solve_multi(nside, lmax, cl, beams, var, masks, ds, O.Options(**opts, band_limit=False))
    assert ores.converged
    M = wf.Multi(nside, lmax, cl, var, masks, beams, wf.options(**opts))
    alm, st, status, recs = M.solve(ds, history=opts["max_iter"] + 1)
    assert status == wf.WF_OK and st["iters"] == ores.iters
    assert O.rel_l2(alm, ores.alm, lmax) < TOL
    for r, h in zip(recs, ores.history):
        assert r["chi2"] == pytest.approx(h["chi2"], rel=TOL)
    M.close()


def test_one_detector_equals_single_plan():
    """One map with a unit beam is the single-field solve (full band)."""
    p, d = problem("wmap-cooled", seed=14, nside=16, lmax=32)
    opts = dict(tol=1e-8, max_iter=4000, band_limit=0)
    single, st1, _, _ = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(**opts)).solve(d)
    M = wf.Multi(16, 32, p.cl, [p.noise_var], [p.mask], None, wf.options(**opts))
    alm, st, status, _ = M.solve([d])
    assert status == wf.WF_OK and st["iters"] == st1["iters"]
    assert O.rel_l2(alm, single, 32) < TOL


def test_mixed_precision_is_rejected():
    p, d = problem("small", seed=1, nside=8, lmax=16)
    with pytest.raises(wf.WFError) as ei:
        wf.Multi(8, 16, p.cl, [p.noise_var], [p.mask], None, wf.options(precision=wf.WF_PREC_MIXED))
    assert ei.value.status == wf.WF_EINVAL
