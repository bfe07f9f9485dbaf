"""GPU messenger iteration (Eqs. 3-4), chi^2 monitor and cooled solve
(Sect. 3) against the oracle on the same seeded inputs.

Bar: 1e-10 relative L2 in a_lm for the FP64 path (m > 0 weighted x2), chi^2
records to 1e-10 relative."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1211_0585_gb300 import wf

from gpu_util import FP64_PATHS, dev, host_alm, problem

pytestmark = pytest.mark.gpu

TOL = 1e-10


def run_oracle_schedule(p, d, schedule):
    states = []
    res = O.solve(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, schedule=schedule,
                  callback=lambda k, rec, s: states.append(s.copy()))
    return res, states


PRECS = list(FP64_PATHS)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind,nside,lmax,lam,lsht,n", [
    ("small", 16, 32, 1.0, 32, 4),
    ("small", 16, 32, 500.0, 20, 4),
    ("small", 8, 24, 3.0, 24, 3),
    ("wmap", 32, 64, 1.0, 64, 3),
    ("wmap", 64, 128, 2.5, 100, 2),
])
def test_iterates_match(kind, nside, lmax, lam, lsht, n, prec):
    import torch
    p, d = problem(kind, seed=2, nside=nside, lmax=lmax)
    res, states = run_oracle_schedule(p, d, [(lam, lsht, n)])
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec]))
    dd = dev(d)
    s = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    for k in range(n):
        recs = P.iterate(dd.data_ptr(), s.data_ptr(), lam, lsht, 1, reset=(k == 0))
        got = host_alm(s)
        assert O.rel_l2(got, states[k], lmax) < TOL, k
        h = res.history[k]
        for key in ("chi2_prior", "chi2_noise", "chi2_lambda"):
            assert recs[0][key] == pytest.approx(h[key], rel=TOL, abs=1e-300), key
        assert math.sqrt(recs[0]["incr2"] / recs[0]["norm2"]) == pytest.approx(h["rel_incr"], rel=1e-8)


@pytest.mark.parametrize("prec", PRECS)
def test_config1_two_hundred_iterations(prec):
    """Nside 16, lmax 32, C_l = 1/(l(l+1)), 200 plain iterations at lambda = 1."""
    import torch
    p, d = problem("small", seed=1)
    res, _ = run_oracle_schedule(p, d, [(1.0, 32, 200)])
    P = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec]))
    s = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    recs = P.iterate(dev(d).data_ptr(), s.data_ptr(), 1.0, 32, 200, reset=True)
    assert O.rel_l2(host_alm(s), res.alm, 32) < TOL
    chi2_gpu = np.array([r["chi2"] for r in recs])
    chi2_orc = np.array([h["chi2"] for h in res.history])
    assert np.allclose(chi2_gpu, chi2_orc, rtol=TOL, atol=0)


@pytest.mark.parametrize("kind,nside,lmax,opts", [
    ("small", 16, 40, dict(tol=1e-7, max_iter=600, lmax_margin=5)),
    ("wmap", 32, 64, dict(tol=1e-8, max_iter=2000)),
    ("wmap", 64, 128, dict(tol=1e-6, max_iter=2000, l_iter0=8, lmax_margin=20)),
])
def test_cooled_solve_matches(kind, nside, lmax, opts):
    """Default precision (double-float Legendre stage)."""
    """The device-resident controller takes the oracle's decisions: same
    lambda levels, band limits and iteration count, same result."""
    p, d = problem(kind, seed=5, nside=nside, lmax=lmax)
    ores = O.solve(nside, lmax, p.cl, p.noise_var, p.mask, d, O.Options(**opts))
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**opts))
    alm, st, status, recs = P.solve(d, history=opts["max_iter"] + 1)
    assert st["iters"] == ores.iters
    assert bool(st["converged"]) == ores.converged
    assert [(r["lam"], r["lsht"]) for r in recs] == [(h["lam"], h["lsht"]) for h in ores.history]
    assert O.rel_l2(alm, ores.alm, lmax) < TOL
    assert st["chi2"] == pytest.approx(ores.history[-1]["chi2"], rel=TOL)


def test_solve_on_device_buffers_and_warm_start():
    import torch
    p, d = problem("wmap", seed=9, nside=16, lmax=32)
    P = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(tol=1e-9))
    alm_h, st_h, _, _ = P.solve(d)
    dd = dev(d)
    out = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    _, st_d, _, _ = P.solve(dd.data_ptr(), out.data_ptr(), on_device=True)
    assert np.array_equal(host_alm(out), alm_h)          # bitwise: fixed reduction order
    assert st_d["iters"] == st_h["iters"]
    # warm start from the answer: converges at once, stays put
    alm_w, st_w, _, _ = P.solve(d, alm_init=alm_h)
    assert st_w["iters"] < st_h["iters"]
    assert O.rel_l2(alm_w, alm_h, 32) < 1e-8


@pytest.mark.parametrize("prec", PRECS)
def test_posterior_gradient_reported(prec):
    """wf_stats.rel_posterior_grad of an FP64 solve is the oracle's posterior
    residual of the returned a_lm (Eq. 2 normal equations on the grid); it is
    not computed with posterior_grad = 0 or on the mixed path (-1)."""
    p, d = problem("wmap", seed=4, nside=16, lmax=32)
    P = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec], tol=1e-9))
    alm, st, status, _ = P.solve(d)
    assert status == wf.WF_OK
    ref = O.posterior_residual(16, 32, alm, p.cl, p.noise_var, p.mask, d)
    assert 0 < ref < 1e-6          # the fixed point solves the grid normal equations of Eq. 2
    # r is a difference of two terms of size ||b||: rounding leaves about 1e-15 of absolute error
    assert abs(st["rel_posterior_grad"] - ref) <= 1e-6 * ref + 1e-13
    P.set_options(wf.options(**FP64_PATHS[prec], tol=1e-9, posterior_grad=0))
    assert P.solve(d)[1]["rel_posterior_grad"] == -1.0
    Q = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(precision=wf.WF_PREC_MIXED, batch_slots=1))
    assert Q.solve(d)[1]["rel_posterior_grad"] == -1.0


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_first_iteration_nside512(prec):
    """WMAP-shaped Nside 512 / lmax 1024 at the bench's launch shapes: the
    first iteration from s = 0 is s_lm = f_l (Y^dagger a d)_lm; sampled
    modes are checked against the oracle one by one."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    nside, lmax = 512, 1024
    p = I.wmap_problem(seed=1, nside=nside, lmax=lmax)
    rng = np.random.default_rng(7)
    d = rng.standard_normal(p.npix) * np.sqrt(p.noise_var) + 50.0 * np.cos(3 * np.arange(p.npix) / p.npix)
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec]))
    lam = 4.0
    s = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    recs = P.iterate(dev(d).data_ptr(), s.data_ptr(), lam, lmax, 1, reset=True)
    got = host_alm(s)
    tau = O.messenger_tau(p.noise_var, p.mask)
    w = O.inverse_noise(p.noise_var, p.mask)
    omega = 4 * math.pi / p.npix
    u = O.pixel_gain(lam, tau, w) * d
    f = O.harmonic_filter(lam, tau, omega, p.cl)
    ls = np.array([2, 3, 10, 100, 1024, 700, 513, 1000, 37, 64])
    ms = np.array([0, 2, 7, 50, 0, 699, 1, 999, 30, 64])
    ref = f[ls] * O.map2alm_modes(nside, lmax, u, ls, ms)
    scale = np.sqrt(np.mean(np.abs(got) ** 2))
    assert np.max(np.abs(got[O.alm_index(lmax, ls, ms)] - ref)) <= 1e-10 * scale
    chi2n = float(np.sum(w * d * d))
    assert recs[0]["chi2_noise"] == pytest.approx(chi2n, rel=1e-12)
    assert recs[0]["chi2_prior"] == 0.0


# lambda levels of the bench's cooled solve (WMAP-shaped, Nside 512 / lmax 1024, seed 1): (lambda, lmax_SHT)
BENCH_LEVELS = [(6.1793721184416155, 120), (1.575, 140), (1.0, 1024)]


def test_full_vector_iterations_nside512_bench_levels():
    """The bench's problem and launch shapes (Nside 512, lmax 1024, every FP64
    form): three iterations at each lambda level / band limit of its cooled
    solve, every one of the 525,825 a_lm of every iterate against the oracle's
    messenger step, element by element, plus the chi^2 records."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    nside, lmax = 512, 1024
    p = I.wmap_problem(seed=1, nside=nside, lmax=lmax)
    d = p.data(O.alm2map(nside, lmax, p.alm_true))
    schedule = [(lam, lsht, 3) for lam, lsht in BENCH_LEVELS]
    res, states = run_oracle_schedule(p, d, schedule)
    dd = dev(d)
    for prec in PRECS:
        P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec]))
        s = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
        k = 0
        for li, (lam, lsht, n) in enumerate(schedule):
            for j in range(n):
                rec = P.iterate(dd.data_ptr(), s.data_ptr(), lam, lsht, 1, reset=(k == 0))[0]
                got, ref = host_alm(s), states[k]
                scale = np.max(np.abs(ref))
                assert np.max(np.abs(got - ref)) <= 1e-10 * scale, (prec, k)
                assert O.rel_l2(got, ref, lmax) < TOL, (prec, k)
                h = res.history[k]
                for key in ("chi2_prior", "chi2_noise", "chi2_lambda"):
                    assert rec[key] == pytest.approx(h[key], rel=TOL, abs=1e-300), (prec, k, key)
                k += 1
        P.close()


def test_cooled_solve_nside128_matches_oracle():
    """A whole cooled solve at Nside 128 / lmax 256 (noise power per steradian
    of the Nside 512 map, so lambda cools through three levels as in the
    bench): same levels, band limits and iteration count as the oracle's
    controller, and the result within 1e-10."""
    nside, lmax = 128, 256
    p, d = problem("wmap-cooled", seed=5, nside=nside, lmax=lmax)
    opts = dict(tol=1e-6, max_iter=3000)
    ores = O.solve(nside, lmax, p.cl, p.noise_var, p.mask, d, O.Options(**opts))
    assert len(O.schedule_of(ores)) >= 3
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**opts))
    alm, st, status, recs = P.solve(d, history=opts["max_iter"] + 1)
    assert status == wf.WF_OK and st["iters"] == ores.iters
    assert [(r["lam"], r["lsht"]) for r in recs] == [(h["lam"], h["lsht"]) for h in ores.history]
    assert O.rel_l2(alm, ores.alm, lmax) < TOL
    assert st["chi2"] == pytest.approx(ores.history[-1]["chi2"], rel=TOL)


@pytest.mark.parametrize("prec", ["fp64-table", "fp64-native"])
def test_paper_stop_rule_stops_on_oracle_iteration(prec):
    """Sect. 3's stop rule alone (Delta chi^2 < 1e-4 sigma_chi2 at lambda = 1,
    the increment rule off): a cooled solve on the device stops on the
    oracle's iteration with the oracle's result."""
    nside, lmax = 32, 64
    p, d = problem("wmap-cooled", seed=8, nside=nside, lmax=lmax)
    opts = dict(tol=0.0, final_dchi2=1e-4, max_iter=5000)
    ores = O.solve(nside, lmax, p.cl, p.noise_var, p.mask, d, O.Options(**opts))
    assert ores.converged and ores.iters < opts["max_iter"]
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec], **opts))
    alm, st, status, recs = P.solve(d, history=opts["max_iter"] + 1)
    assert status == wf.WF_OK and st["converged"] == 1
    assert st["iters"] == ores.iters
    assert [(r["lam"], r["lsht"]) for r in recs] == [(h["lam"], h["lsht"]) for h in ores.history]
    assert O.rel_l2(alm, ores.alm, lmax) < TOL


def test_table_form_first_iteration_nside1024():
    """The lambda-table form at Nside 1024 / lmax 2048 (34 GB table, ring pairs in two analysis chunks of
    1024), as the serving pool runs it on a large GPU: the first iteration from s = 0 on sampled modes
    against the oracle, one by one."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    nside, lmax = 1024, 2048
    p = I.wmap_problem(seed=2, nside=nside, lmax=lmax, ndisc=50, noise_scale=4.0)
    rng = np.random.default_rng(8)
    d = rng.standard_normal(p.npix) * np.sqrt(p.noise_var) + 30.0 * np.sin(5 * np.arange(p.npix) / p.npix)
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, wf.options(legendre_table_bytes=48 << 30))
    held, _ = P.legendre_table(lmax)
    assert held > 30e9
    lam = 3.0
    s = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    P.iterate(dev(d).data_ptr(), s.data_ptr(), lam, lmax, 1, reset=True)
    got = host_alm(s)
    tau = O.messenger_tau(p.noise_var, p.mask)
    w = O.inverse_noise(p.noise_var, p.mask)
    u = O.pixel_gain(lam, tau, w) * d
    f = O.harmonic_filter(lam, tau, 4 * math.pi / p.npix, p.cl)
    ls = np.array([2, 17, 300, 1024, 2048, 1500, 1100, 2000, 64, 1030])
    ms = np.array([0, 3, 299, 0, 2047, 1490, 1, 1999, 64, 1025])
    ref = f[ls] * O.map2alm_modes(nside, lmax, u, ls, ms)
    scale = np.sqrt(np.mean(np.abs(got) ** 2))
    assert np.max(np.abs(got[O.alm_index(lmax, ls, ms)] - ref)) <= 1e-10 * scale
    P.close()
