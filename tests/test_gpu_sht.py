"""GPU spherical harmonic transform pair against the oracle, element by
element (bar: 1e-12 relative to the largest value)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1211_0585_gb300 import inputs as I
from paper_1211_0585_gb300 import wf

from gpu_util import FP64_PATHS, dev, host_alm

pytestmark = pytest.mark.gpu

CASES = [(1, 2), (2, 6), (4, 8), (4, 13), (8, 16), (16, 32), (16, 64), (32, 64), (64, 128), (64, 40),
         (1, 0), (1, 4), (2, 8), (8, 0), (8, 32)]  # degenerate: lmax 0, lmax = 4 nside


PRECS = list(FP64_PATHS)


def plan_for(nside, lmax, prec="fp64-table"):
    return wf.Plan(nside, lmax, np.ones(lmax + 1), np.ones(12 * nside * nside), opts=wf.options(**FP64_PATHS[prec]))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nside,lmax", CASES)
def test_alm2map(nside, lmax, prec):
    import torch
    rng = np.random.default_rng(nside * 1000 + lmax)
    alm = I.draw_alm(np.ones(lmax + 1), rng)
    ref = O.alm2map(nside, lmax, alm)
    P = plan_for(nside, lmax, prec)
    a = dev(alm)
    m = torch.empty(12 * nside * nside, dtype=torch.float64, device="cuda")
    P.alm2map(lmax, a.data_ptr(), m.data_ptr())
    torch.cuda.synchronize()
    got = m.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nside,lmax", CASES)
def test_map2alm(nside, lmax, prec):
    import torch
    rng = np.random.default_rng(nside * 7 + lmax)
    f = rng.standard_normal(12 * nside * nside)
    ref = O.map2alm(nside, lmax, f)
    P = plan_for(nside, lmax, prec)
    a = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    P.map2alm(lmax, dev(f).data_ptr(), a.data_ptr())
    torch.cuda.synchronize()
    got = host_alm(a)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64-table", "fp64-recurrence"])
@pytest.mark.parametrize("nside,lmax,lsht", [(16, 48, 20), (32, 64, 0), (32, 64, 5), (32, 64, 63)])
def test_band_limited(nside, lmax, lsht, prec):
    """With band limit lsht only l <= lsht take part; analysis zeroes the rest."""
    import torch
    rng = np.random.default_rng(3)
    alm = I.draw_alm(np.ones(lmax + 1), rng)
    ref = O.alm2map(nside, lsht, O.truncate_alm(alm, lmax, lsht))
    P = plan_for(nside, lmax, prec)
    m = torch.empty(12 * nside * nside, dtype=torch.float64, device="cuda")
    P.alm2map(lsht, dev(alm).data_ptr(), m.data_ptr())
    f = rng.standard_normal(12 * nside * nside)
    a = dev(np.full(P.nalm, 7.0 + 0j))
    P.map2alm(lsht, dev(f).data_ptr(), a.data_ptr())
    torch.cuda.synchronize()
    assert np.max(np.abs(m.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    refa = O.embed_alm(O.map2alm(nside, lsht, f), lsht, lmax)
    got = host_alm(a)
    assert np.max(np.abs(got - refa)) <= 1e-12 * np.max(np.abs(refa))


@pytest.mark.parametrize("prec", PRECS)
def test_sampled_full_size_nside512(prec):
    """At the WMAP-shaped size (Nside 512, lmax 1024): sampled pixels of the
    synthesis and sampled modes of the analysis, each computed one by one by
    the oracle."""
    import torch
    nside, lmax = 512, 1024
    rng = np.random.default_rng(512)
    cl = I.cl_lcdm_like(lmax, 13.0)
    alm = I.draw_alm(cl, rng)
    P = plan_for(nside, lmax, prec)
    m = torch.empty(12 * nside * nside, dtype=torch.float64, device="cuda")
    P.alm2map(lmax, dev(alm).data_ptr(), m.data_ptr())
    f = rng.standard_normal(12 * nside * nside)
    a = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    P.map2alm(lmax, dev(f).data_ptr(), a.data_ptr())
    torch.cuda.synchronize()
    got_map = m.cpu().numpy()
    pix = np.concatenate([rng.integers(0, f.size, 24), [0, 1, 5, f.size - 1, f.size // 2]])
    ref = O.alm2map_pixels(nside, lmax, alm, pix)
    scale = np.max(np.abs(got_map))
    assert np.max(np.abs(got_map[pix] - ref)) <= 1e-11 * scale
    ls = np.array([0, 1, 2, 100, 1024, 1024, 700, 513, 1000, 37])
    ms = np.array([0, 0, 2, 50, 0, 1024, 699, 1, 999, 30])
    refa = O.map2alm_modes(nside, lmax, f, ls, ms)
    got = host_alm(a)[O.alm_index(lmax, ls, ms)]
    assert np.max(np.abs(got - refa)) <= 1e-11 * np.max(np.abs(host_alm(a)))


@pytest.mark.parametrize("prec", ["fp64-recurrence", "fp64-native"])
def test_sampled_full_size_nside2048(prec):
    """At the Planck-shaped size (Nside 2048, lmax 4096), where the polar rings
    with Bluestein buffers of 16384 points run their FFTs in global scratch and
    the analysis state is split into ring-pair chunks: sampled pixels (among
    them pixels of those rings, in both caps) and sampled modes up to m = 4096,
    each computed one by one by the oracle. Bar: the FP64 path's 1e-10,
    relative to the largest value (the recurrence runs to l = 4096 and its
    rounding grows with l; it is largest at the poles, where lambda_l0 peaks)."""
    import torch
    nside, lmax = 2048, 4096
    npix = 12 * nside * nside
    rng = np.random.default_rng(2048)
    cl = I.cl_lcdm_like(lmax, 5.0)
    alm = I.draw_alm(cl, rng)
    P = plan_for(nside, lmax, prec)
    m = torch.empty(npix, dtype=torch.float64, device="cuda")
    P.alm2map(lmax, dev(alm).data_ptr(), m.data_ptr())
    f = rng.standard_normal(npix)
    a = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    P.map2alm(lmax, dev(f).data_ptr(), a.data_ptr())
    torch.cuda.synchronize()
    got_map = m.cpu().numpy()
    # ring i (1-based, north cap) starts at pixel 2 i (i - 1); rings 1025 .. 2047 use global scratch
    big_north = [2 * i * (i - 1) + j for i, j in ((1025, 3), (1500, 100), (2047, 8187))]
    big_south = [npix - 1 - p for p in big_north]
    pix = np.concatenate([rng.integers(0, npix, 16), big_north, big_south, [0, 1, npix - 1, npix // 2]])
    ref = O.alm2map_pixels(nside, lmax, alm, pix)
    scale = np.max(np.abs(got_map))
    assert np.max(np.abs(got_map[pix] - ref)) <= 1e-10 * scale
    ls = np.array([0, 2, 100, 4096, 4096, 3000, 2049, 4000, 37, 1500])
    ms = np.array([0, 2, 50, 0, 4096, 2999, 1, 3999, 30, 1024])
    refa = O.map2alm_modes(nside, lmax, f, ls, ms)
    got = host_alm(a)[O.alm_index(lmax, ls, ms)]
    assert np.max(np.abs(got - refa)) <= 1e-10 * np.max(np.abs(host_alm(a)))


def test_lambda_table_held_where_it_fits():
    """The FP64 plan holds the precomputed lambda table when it fits the
    option's limit (Nside 512 / lmax 1024: 4.3 GB), not at a limit of 0, not
    for other precisions; one pass needs less of it than it holds (the rows
    below the 2^-60 cut are never read)."""
    ones = lambda n: np.ones(n)
    nside, lmax = 512, 1024
    P = wf.Plan(nside, lmax, ones(lmax + 1), ones(12 * nside * nside), opts=wf.options(precision=0))
    held, per_pass = P.legendre_table(lmax)
    rows = sum((lmax - m + 2) // 2 for m in range(lmax + 1))
    assert held == rows * 2 * nside * 16  # 2 nside ring pairs: a multiple of 32
    ev, full = P.legendre_terms(lmax)
    assert ev * 8 <= per_pass < held
    _, per_pass_low = P.legendre_table(100)
    assert per_pass_low < per_pass
    del P
    for o in (dict(precision=0, legendre_table_bytes=0), dict(precision=2), dict(precision=1)):
        Q = wf.Plan(64, 128, ones(129), ones(12 * 64 * 64), opts=wf.options(**o))
        assert Q.legendre_table(128)[0] == 0
