"""Helpers shared by the GPU tests: device buffers through torch, seeded
problems whose data map comes from the oracle's synthesis."""
import numpy as np

from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I


# The FP64-accurate paths: the double-float Legendre stage reading the
# precomputed lambda table (the default where it fits), the same stage running
# the recurrence, and every step in native FP64.
FP64_PATHS = {
    "fp64-table": dict(precision=0),
    "fp64-recurrence": dict(precision=0, legendre_table_bytes=0),
    "fp64-native": dict(precision=2),
}


def dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.complex128:
        a = a.view(np.float64)
    return torch.from_numpy(a.copy()).cuda()


def host_alm(t):
    return t.cpu().numpy().view(np.complex128)


def problem(kind, seed=1, nside=16, lmax=32):
    if kind == "small":
        p = I.small_problem(seed=seed, nside=nside, lmax=lmax)
    elif kind == "wmap":
        p = I.wmap_problem(seed=seed, nside=nside, lmax=lmax, ndisc=max(5, 12 * nside * nside // 6000))
    elif kind == "wmap-cooled":
        # the WMAP-shaped problem with the noise power per steradian of the Nside 512 map, so that
        # lambda starts above 1 and the solve cools through levels as the bench's does
        p = I.wmap_problem(seed=seed, nside=nside, lmax=lmax, ndisc=max(5, 12 * nside * nside // 6000),
                           noise_scale=(nside / 512.0) ** 2)
    else:
        raise ValueError(kind)
    d = p.data(O.alm2map(p.nside, p.lmax, p.alm_true))
    return p, d


def _oracle_solve(args):
    """One oracle solve in a worker process (see oracle_solves): the stopping
    iteration k and the iterates k - extra .. k + extra (the last ones by
    further iterations at lambda = 1 and full band, as the solve's last level)."""
    nside, lmax, cl, var, mask, d, opts, extra = args
    keep = {}
    res = O.solve(nside, lmax, cl, var, mask, d, O.Options(**opts),
                  callback=lambda k, rec, s: keep.__setitem__(k, s.copy()))
    k = res.iters
    states = {i: keep[i] for i in range(max(1, k - extra), k + 1)}
    if extra:
        import math
        tau = O.messenger_tau(var, mask)
        w = O.inverse_noise(var, mask)
        omega = 4.0 * math.pi / (12 * nside * nside)
        s = res.alm
        for i in range(k + 1, k + extra + 1):
            s = O.messenger_step(nside, lmax, lmax, s, d, w, O.pixel_gain(1.0, tau, w),
                                 O.harmonic_filter(1.0, tau, omega, cl), cl, 1.0, tau).s_alm
            states[i] = s
    return k, states


def _one_thread():
    import os
    os.environ["OMP_NUM_THREADS"] = "1"


def oracle_solves(jobs, workers=None):
    """Oracle solves of many small problems in parallel, one OpenMP thread per
    worker process. The pool is started with `spawn`, so it is safe after the
    test process has used the GPU."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    n = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    with ProcessPoolExecutor(n, mp_context=mp.get_context("spawn"), initializer=_one_thread) as ex:
        return list(ex.map(_oracle_solve, jobs))
