"""Serving: continuous batching of requests of different shapes, noise, masks
and tolerances. Every result must match the oracle solve of the same request
(mixed bar 1e-6, FP64 bar 1e-10) and the same request solved alone; wf_poll
never blocks; latency percentiles are reported."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I
from paper_1211_0585_gb300 import wf

pytestmark = pytest.mark.gpu


def make_request(seed, nside, lmax):
    rng = np.random.default_rng(seed)
    p = I.wmap_problem(seed=seed, nside=nside, lmax=lmax, ndisc=int(rng.integers(0, 12)))
    amp = rng.uniform(0.5, 2.0)
    cl = p.cl * amp
    alm = I.draw_alm(cl, rng)
    d = O.alm2map(nside, lmax, alm) + p.noise
    return dict(nside=nside, lmax=lmax, cl=cl, noise=p.noise_var, mask=p.mask, d=d)


def test_server_mixed_and_fp64_requests():
    reqs = []
    shapes = [(16, 32), (32, 64)]
    for i in range(7):
        ns, lm = shapes[i % 2]
        r = make_request(100 + i, ns, lm)
        r["tol"] = 1e-8 if i % 3 == 2 else 1e-6
        reqs.append(r)
    S = wf.Server(hbm_budget_bytes=8 << 30, max_batch=2)
    tickets = []
    for r in reqs:
        tickets.append(S.submit(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], r["d"], r["tol"]))
        time.sleep(0.01)
    t0 = time.perf_counter()
    early = S.poll(tickets[0])          # never blocks; may already hold the result
    assert time.perf_counter() - t0 < 0.05
    S.drain(300000)
    st = S.stats()
    assert st["completed"] == len(reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    for r, t in zip(reqs, tickets):
        res = early if (t == tickets[0] and early is not None) else S.poll(t)
        assert res is not None
        alm, stats, status = res
        assert status == wf.WF_OK
        opts = O.Options(tol=r["tol"], max_iter=10000)
        ref = O.solve(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], r["d"], opts)
        bar = 1e-10 if r["tol"] <= 1e-7 else 1e-6
        assert O.rel_l2(alm, ref.alm, r["lmax"]) <= bar
        # the same request alone: within the mixed bar for the batched engine
        # (slots share FP32 ring FFTs in pairs), parity for FP64
        prec = wf.WF_PREC_FP64 if r["tol"] <= 1e-7 else wf.WF_PREC_MIXED
        P = wf.Plan(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"],
                    wf.options(precision=prec, tol=r["tol"], batch_slots=1))
        alone, _, _, _ = P.solve(r["d"])
        if prec == wf.WF_PREC_MIXED:
            assert O.rel_l2(alm, alone, r["lmax"]) <= 1e-6
        else:
            assert O.rel_l2(alm, alone, r["lmax"]) < 1e-12
    with pytest.raises(wf.WFError):
        S.poll(tickets[0])            # already collected
    S.close()


def test_server_fp64_plan_reuse():
    """FP64 requests of one shape that arrive one after another run on the same
    resident plan, re-pointed at each request's C_l, noise and mask: each
    result is bitwise the result of a fresh plan for that request."""
    S = wf.Server(hbm_budget_bytes=8 << 30, max_batch=1)
    S.warm(32, 64, wf.WF_PREC_FP64)          # the first request already finds a resident plan
    S.warm(16, 32, wf.WF_PREC_MIXED)
    with pytest.raises(wf.WFError):
        S.warm(16, 32, 7)
    for i, seed in enumerate((301, 302, 303)):
        r = make_request(seed, 32, 64)
        if i == 1:
            r["mask"] = None
        t = S.submit(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], r["d"], 1e-8)
        S.drain(300000)
        alm, _, status = S.poll(t)
        assert status == wf.WF_OK
        P = wf.Plan(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], wf.options(precision=0, tol=1e-8))
        alone, _, _, _ = P.solve(r["d"])
        assert np.array_equal(alm, alone)
    S.close()


def test_server_rejects_bad_requests():
    S = wf.Server(hbm_budget_bytes=1 << 30, max_batch=1)
    npix = 12 * 4 * 4
    with pytest.raises(wf.WFError):
        S.submit(4, 8, np.ones(9), -np.ones(npix), None, np.zeros(npix), 1e-6)
    with pytest.raises(wf.WFError):
        S.submit(3, 8, np.ones(9), np.ones(108), None, np.zeros(108), 1e-6)
    S.close()


def test_server_lone_mixed_request_runs_on_fp64_pool():
    """A mixed-tolerance request that finds its shape's engine without live
    slots runs on the FP64 pool (faster for one request than a near-empty
    engine): its result is the FP64 solve's at its tolerance."""
    r = make_request(401, 32, 64)
    S = wf.Server(hbm_budget_bytes=8 << 30, max_batch=4)
    t = S.submit(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], r["d"], 1e-6)
    S.drain(300000)
    alm, stats, status = S.poll(t)
    assert status == wf.WF_OK
    P = wf.Plan(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], wf.options(precision=0, tol=1e-6))
    alone, _, _, _ = P.solve(r["d"])
    assert np.array_equal(alm, alone)
    assert stats["rel_posterior_grad"] > 0      # computed: the FP64 path ran
    S.close()


def test_server_fp64_pool_evicts_idle_plans_for_other_shapes():
    """With a budget that holds one FP64 plan of these shapes, a request of a
    second shape evicts the idle plan of the first; both results are right."""
    reqs = [make_request(501, 16, 32), make_request(502, 32, 64), make_request(503, 16, 32)]
    S = wf.Server(hbm_budget_bytes=4_800_000, max_batch=1)  # FP64 plans: about 0.9 MB and 4.1 MB
    for r in reqs:
        t = S.submit(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], r["d"], 1e-8)
        S.drain(300000)
        alm, _, status = S.poll(t)
        assert status == wf.WF_OK
        P = wf.Plan(r["nside"], r["lmax"], r["cl"], r["noise"], r["mask"], wf.options(precision=0, tol=1e-8))
        assert np.array_equal(alm, P.solve(r["d"])[0])
    S.close()
