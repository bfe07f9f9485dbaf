"""wf_map2alm_noalloc: the plan-free map2alm for callers that cannot allocate
device memory (a framework-owned memory budget, or a latency-critical loop
that cannot take cudaMalloc's implicit synchronisation). Its output must match
the planned wf_map2alm within the transforms' parity bar (1e-12 of the largest
coefficient) on two calls in a row, since every call reuses the same static
scratch. This file is collected last so that a failure here comes after every
other test has run."""
import numpy as np
import pytest

from paper_1211_0585_gb300 import wf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nside,lmax", [(16, 40), (64, 128)])
def test_noalloc_matches_planned_map2alm(nside, lmax):
    import torch
    npix = 12 * nside * nside
    nalm = (lmax + 1) * (lmax + 2) // 2
    rng = np.random.default_rng(nside + lmax)
    P = wf.Plan(nside, lmax, np.ones(lmax + 1), np.ones(npix))
    for call in range(2):
        f = torch.from_numpy(rng.standard_normal(npix)).cuda()
        ref = torch.zeros(2 * nalm, dtype=torch.float64, device="cuda")
        P.map2alm(lmax, f.data_ptr(), ref.data_ptr())
        got = torch.full((2 * nalm,), 3.0, dtype=torch.float64, device="cuda")
        wf.map2alm_noalloc(nside, lmax, f.data_ptr(), got.data_ptr())
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.max(np.abs(g - r)) <= 1e-12 * np.max(np.abs(r)), f"call {call}"
    P.close()


def test_noalloc_rejects_sizes_beyond_scratch():
    import torch
    m = torch.zeros(12 * 256 * 256, dtype=torch.float64, device="cuda")
    a = torch.zeros(2 * (513 * 514 // 2), dtype=torch.float64, device="cuda")
    with pytest.raises(wf.WFError) as ei:
        wf.map2alm_noalloc(256, 512, m.data_ptr(), a.data_ptr())
    assert ei.value.status == wf.WF_EINVAL
    assert "bytes of scratch" in str(ei.value)
