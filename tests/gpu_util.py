"""Helpers shared by the GPU tests: device buffers through torch, seeded
problems whose data map comes from the oracle's synthesis."""
import numpy as np

from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I


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
