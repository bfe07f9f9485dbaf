"""Failure paths, cancellation and resume, all made on the host (no GPU
fault is provoked): every status code the library documents for a solve or
a served request is produced and checked, and an iteration can be stopped
and resumed from its a_lm state with bitwise the same result."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1211_0585_gb300 import wf

from gpu_util import FP64_PATHS, dev, host_alm, problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64-table", "fp64-native"])
def test_not_converged_writes_result(prec):
    """WF_ENOTCONVERGED when max_iter ends the solve before the stop rule; the
    result is still written and is the oracle's state after those iterations."""
    p, d = problem("wmap-cooled", seed=3, nside=16, lmax=32)
    opts = dict(tol=1e-9, max_iter=3)
    ores = O.solve(16, 32, p.cl, p.noise_var, p.mask, d, O.Options(**opts))
    assert not ores.converged and ores.iters == 3
    P = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(**FP64_PATHS[prec], **opts))
    alm, st, status, _ = P.solve(d)
    assert status == wf.WF_ENOTCONVERGED
    assert st["iters"] == 3 and st["converged"] == 0
    assert O.rel_l2(alm, ores.alm, 32) < 1e-10


@pytest.mark.parametrize("opts", [dict(precision=0), dict(precision=2),
                                  dict(precision=1, batch_slots=1)])
def test_nan_data_gives_enumeric_and_plan_stays_usable(opts):
    """A NaN written into d on an observed pixel (on the host, before the
    solve) makes chi^2 non-finite: the controller stops the solve and the call
    returns WF_ENUMERIC; the same plan then solves clean data normally."""
    p, d = problem("wmap", seed=4, nside=16, lmax=32)
    bad = d.copy()
    obs = np.flatnonzero(p.mask)
    bad[obs[len(obs) // 2]] = np.nan
    mixed = opts["precision"] == 1
    tol = 1e-6 if mixed else 1e-8     # the mixed path's increments stall near 1e-7
    P = wf.Plan(16, 32, p.cl, p.noise_var, p.mask, wf.options(tol=tol, **opts))
    with pytest.raises(wf.WFError) as ei:
        P.solve(bad)
    assert ei.value.status == wf.WF_ENUMERIC
    alm, st, status, _ = P.solve(d)
    assert status == wf.WF_OK and np.all(np.isfinite(alm))
    ref = O.solve(16, 32, p.cl, p.noise_var, p.mask, d, O.Options(tol=tol))
    # mixed: the mixed bar plus one increment, should the stop fall one iteration off the oracle's
    assert O.rel_l2(alm, ref.alm, 32) < (1e-6 + 2 * tol if mixed else 1e-10)


def test_server_enomem_when_nothing_fits_budget():
    """A server whose HBM budget is smaller than any plan of the shape rejects
    the request at submit, and the shape at warm-up, with WF_ENOMEM."""
    p, d = problem("wmap", seed=2, nside=64, lmax=128)
    S = wf.Server(hbm_budget_bytes=1 << 20, max_batch=4)
    for tol in (1e-8, 1e-5):
        with pytest.raises(wf.WFError) as ei:
            S.submit(64, 128, p.cl, p.noise_var, p.mask, d, tol)
        assert ei.value.status == wf.WF_ENOMEM
    for prec in (wf.WF_PREC_FP64, wf.WF_PREC_MIXED):
        with pytest.raises(wf.WFError) as ei:
            S.warm(64, 128, prec)
        assert ei.value.status == wf.WF_ENOMEM
    S.drain(1000)          # nothing was admitted
    S.close()


def test_server_drain_timeout_then_completes():
    """wf_server_drain with a zero timeout while requests are queued gives
    WF_ETIMEOUT; a later drain waits for them and every result is correct."""
    p, d = problem("wmap", seed=6, nside=32, lmax=64)
    S = wf.Server(max_batch=4)
    tickets = [S.submit(32, 64, p.cl, p.noise_var, p.mask, d, 1e-8) for _ in range(4)]
    with pytest.raises(wf.WFError) as ei:
        S.drain(0)
    assert ei.value.status == wf.WF_ETIMEOUT
    S.drain(600000)
    ref = O.solve(32, 64, p.cl, p.noise_var, p.mask, d, O.Options(tol=1e-8))
    for t in tickets:
        alm, st, status = S.poll(t)
        assert status == wf.WF_OK
        assert O.rel_l2(alm, ref.alm, 64) < 1e-10
        assert st["ms_latency"] >= st["ms_device"] > 0
    S.close()


@pytest.mark.parametrize("tol", [1e-8, 1e-5])
def test_server_cancel(tol):
    """wf_cancel: queued requests are dropped and report WF_ECANCELLED from
    wf_poll with no a_lm; the others finish normally; a collected ticket is
    unknown (WF_ENOTFOUND) and a finished one cannot be cancelled (WF_EINVAL)."""
    p, d = problem("wmap", seed=7, nside=32, lmax=64)
    S = wf.Server(max_batch=2)
    tickets = [S.submit(32, 64, p.cl, p.noise_var, p.mask, d, tol) for _ in range(8)]
    cancelled = tickets[5:]
    codes = [S.cancel(t) for t in cancelled]
    S.drain(600000)
    ref = O.solve(32, 64, p.cl, p.noise_var, p.mask, d, O.Options(tol=tol))
    bar = 1e-10 if tol <= 1e-7 else 1e-6 + 2 * tol
    for t, code in zip(cancelled, codes):
        alm, st, status = S.poll(t)
        if code == wf.WF_OK:
            assert status == wf.WF_ECANCELLED and alm is None
        else:                       # it had finished before the cancel: the result stands
            assert code == wf.WF_EINVAL and status == wf.WF_OK
    assert sum(c == wf.WF_OK for c in codes) >= 1
    for t in tickets[:5]:
        alm, st, status = S.poll(t)
        assert status == wf.WF_OK
        assert O.rel_l2(alm, ref.alm, 64) < bar
        assert S.cancel(t) == wf.WF_ENOTFOUND
    S.close()


@pytest.mark.parametrize("prec", list(FP64_PATHS))
def test_resume_from_state_is_bitwise(prec):
    """Checkpoint / resume of the iteration: N + M iterations in one call equal
    N iterations, then M more continuing on the same plan, and equal N
    iterations, a copy of the a_lm state to the host, then M iterations on a
    fresh plan restarted from that copy -- bit for bit on the FP64 paths."""
    import torch
    nside, lmax, lam, lsht, N, M = 32, 64, 1.6, 64, 5, 7
    p, d = problem("wmap-cooled", seed=9, nside=nside, lmax=lmax)
    dd = dev(d)
    opts = wf.options(**FP64_PATHS[prec])
    P = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, opts)
    s_all = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    P.iterate(dd.data_ptr(), s_all.data_ptr(), lam, lsht, N + M, reset=True)
    s_two = torch.zeros_like(s_all)
    P.iterate(dd.data_ptr(), s_two.data_ptr(), lam, lsht, N, reset=True)
    checkpoint = host_alm(s_two).copy()
    P.iterate(dd.data_ptr(), s_two.data_ptr(), lam, lsht, M, reset=False)
    assert np.array_equal(host_alm(s_all), host_alm(s_two))
    Q = wf.Plan(nside, lmax, p.cl, p.noise_var, p.mask, opts)
    s_res = dev(checkpoint)
    Q.iterate(dd.data_ptr(), s_res.data_ptr(), lam, lsht, M, reset=True)
    assert np.array_equal(host_alm(s_all), host_alm(s_res))
