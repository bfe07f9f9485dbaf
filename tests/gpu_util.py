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
    else:
        raise ValueError(kind)
    d = p.data(O.alm2map(p.nside, p.lmax, p.alm_true))
    return p, d
