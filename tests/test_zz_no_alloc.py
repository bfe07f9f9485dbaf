"""wf_map2alm_noalloc: the plan-free map2alm for callers that cannot allocate
device memory (code running under a memory budget owned by another allocator,
such as a framework's caching allocator or a fixed pool, or a latency-critical
loop that cannot take cudaMalloc's implicit device synchronisation).

Two calls in a row on fresh maps (every call reuses the same static scratch)
must match the oracle's map2alm within the transforms' parity bar (1e-12 of
the largest coefficient), and wf_map2alm of a plan that runs the same native
FP64 kernels to rounding (1e-14: the plan builds its FFT tables and ring
classes on its own). The largest sizes the static scratch accepts are
included. This file is collected last so that a failure here
comes after every other test has run."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1211_0585_gb300 import wf

pytestmark = pytest.mark.gpu


# (16, 40), (64, 128): ordinary sizes; (128, 512) and (256, 243): the largest
# lmax the 16 MiB scratch takes at Nside 128 and 256 (one ring class over all
# rings, the largest Bluestein rings and table offsets)
@pytest.mark.parametrize("nside,lmax", [(16, 40), (64, 128), (128, 512), (256, 243)])
def test_noalloc_matches_oracle_and_native_plan(nside, lmax):
    import torch
    npix = 12 * nside * nside
    nalm = (lmax + 1) * (lmax + 2) // 2
    rng = np.random.default_rng(nside + lmax)
    P = wf.Plan(nside, lmax, np.ones(lmax + 1), np.ones(npix), opts=wf.options(precision=wf.WF_PREC_FP64_NATIVE))
    for call in range(2):
        f_host = rng.standard_normal(npix)
        f = torch.from_numpy(f_host).cuda()
        ref = torch.zeros(2 * nalm, dtype=torch.float64, device="cuda")
        P.map2alm(lmax, f.data_ptr(), ref.data_ptr())
        got = torch.full((2 * nalm,), 3.0, dtype=torch.float64, device="cuda")
        wf.map2alm_noalloc(nside, lmax, f.data_ptr(), got.data_ptr())
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.max(np.abs(g - r)) <= 1e-14 * np.max(np.abs(r)), f"call {call}: native FP64 plan"
        orc = O.map2alm(nside, lmax, f_host).view(np.float64)
        assert np.max(np.abs(g - orc)) <= 1e-12 * np.max(np.abs(orc)), f"call {call}: oracle"
    P.close()


@pytest.mark.parametrize("nside,lmax", [(256, 512), (256, 244), (512, 0)])
def test_noalloc_rejects_sizes_beyond_scratch(nside, lmax):
    import torch
    m = torch.zeros(12 * nside * nside, dtype=torch.float64, device="cuda")
    a = torch.zeros(2 * ((lmax + 1) * (lmax + 2) // 2), dtype=torch.float64, device="cuda")
    with pytest.raises(wf.WFError) as ei:
        wf.map2alm_noalloc(nside, lmax, m.data_ptr(), a.data_ptr())
    assert ei.value.status == wf.WF_EINVAL
    assert "bytes of scratch" in str(ei.value)
