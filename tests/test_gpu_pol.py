"""Temperature and polarisation on the device (Sect. 4: the filter on T and P
maps together) against the oracle: the (T, E, B) <-> (T, Q, U) transform pair
element by element, and the cooled joint solve."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import pol as PO
from paper_1211_0585_gb300 import inputs as I
from paper_1211_0585_gb300 import wf

from gpu_util import FP64_PATHS
from test_oracle_pol import pol_problem, rand_alm3

pytestmark = pytest.mark.gpu

PATHS = ["fp64-table", "fp64-native"]


def unit_pol(nside, lmax, prec):
    npix = 12 * nside * nside
    cls = [np.ones(lmax + 1)] * 3 + [np.zeros(lmax + 1)]
    noise = np.tile([1.0, 1.0, 0.0, 1.0], (npix, 1))
    return wf.Pol(nside, lmax, cls, noise, opts=wf.options(**FP64_PATHS[prec]))


@pytest.mark.parametrize("prec", PATHS)
@pytest.mark.parametrize("nside,lmax", [(2, 6), (4, 8), (8, 16), (16, 32), (16, 48), (32, 64), (64, 128)])
def test_transform_pair(nside, lmax, prec):
    import torch
    rng = np.random.default_rng(nside * 31 + lmax)
    a = rand_alm3(lmax, rng)
    ref_map = PO.pol_alm2map(nside, lmax, a)
    Q = unit_pol(nside, lmax, prec)
    ad = torch.from_numpy(a.view(np.float64).copy()).cuda()
    m = torch.empty(3 * 12 * nside * nside, dtype=torch.float64, device="cuda")
    Q.alm2map(ad.data_ptr(), m.data_ptr())
    torch.cuda.synchronize()
    got = m.cpu().numpy().reshape(3, -1)
    assert np.max(np.abs(got - ref_map)) <= 1e-12 * np.max(np.abs(ref_map))
    f = rng.standard_normal((3, 12 * nside * nside))
    ref_alm = PO.pol_map2alm(nside, lmax, f)
    fd = torch.from_numpy(f.copy()).cuda()
    out = torch.zeros(3 * 2 * Q.nalm, dtype=torch.float64, device="cuda")
    Q.map2alm(fd.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    got_alm = out.cpu().numpy().view(np.complex128).reshape(3, -1)
    assert np.max(np.abs(got_alm - ref_alm)) <= 1e-12 * np.max(np.abs(ref_alm))
    Q.close()


_oracle_runs = {}


def oracle_pol_solve(nside, lmax, l_iter0, tol):
    key = (nside, lmax, l_iter0, tol)
    if key not in _oracle_runs:
        cls, nz, mt, mp, d = pol_problem(nside, lmax, 11, noise=2e-2)
        opts = dict(tol=tol, max_iter=4000, l_iter0=l_iter0)
        ores = PO.solve_pol(nside, lmax, cls, nz, mt, mp, d, O.Options(**opts, band_limit=False))
        _oracle_runs[key] = (cls, nz, mt, mp, d, opts, ores)
    return _oracle_runs[key]


@pytest.mark.parametrize("prec", PATHS)
@pytest.mark.parametrize("nside,lmax,l_iter0,tol", [(8, 16, 4, 1e-7), (16, 32, 8, 1e-6)])
def test_cooled_pol_solve_matches_oracle(nside, lmax, l_iter0, tol, prec):
    """Same lambda levels and iteration count as the oracle's controller, every
    field of the result within the FP64 bar, and the chi^2 records (the
    polarised problem converges slowly: E and B are weak against the noise)."""
    cls, nz, mt, mp, d, opts, ores = oracle_pol_solve(nside, lmax, l_iter0, tol)
    assert ores.converged and len({h["lam"] for h in ores.history}) >= 2
    Q = wf.Pol(nside, lmax, cls, nz, mt, mp, wf.options(**FP64_PATHS[prec], **opts))
    alm, st, status, recs = Q.solve(d, history=opts["max_iter"] + 1)
    assert status == wf.WF_OK and st["iters"] == ores.iters
    assert [r["lam"] for r in recs] == pytest.approx([h["lam"] for h in ores.history], rel=1e-14)
    for f in range(3):
        assert O.rel_l2(alm[f], ores.alm[f], lmax) < 1e-10, f
    for r, h in zip(recs, ores.history):
        assert r["chi2"] == pytest.approx(h["chi2"], rel=1e-10)
    Q.close()


def test_bad_polarisation_inputs_rejected():
    nside, lmax = 4, 8
    npix = 12 * nside * nside
    cls = [np.ones(lmax + 1), np.ones(lmax + 1), np.ones(lmax + 1), 2 * np.ones(lmax + 1)]   # C_TE^2 > TT EE
    noise = np.tile([1.0, 1.0, 0.0, 1.0], (npix, 1))
    with pytest.raises(wf.WFError):
        wf.Pol(nside, lmax, cls, noise)
    cls[3] = np.zeros(lmax + 1)
    noise[5] = [1.0, 1.0, 2.0, 1.0]                     # Q-U block not positive definite
    with pytest.raises(wf.WFError):
        wf.Pol(nside, lmax, cls, noise)
    with pytest.raises(wf.WFError):
        wf.Pol(nside, lmax, cls, np.tile([1.0, 1.0, 0.0, 1.0], (npix, 1)), opts=wf.options(precision=1))
