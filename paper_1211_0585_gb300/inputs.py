"""Seeded synthetic inputs shaped like the WMAP/Planck temperature workloads.

This module holds no arithmetic of the Wiener-filter method: no spherical
harmonic transform, no messenger update. It draws random numbers and builds
the fixed ingredients of a problem instance -- the signal spectrum C_l (beam
folded in), Gaussian a_lm drawn from it, a noise-variance map from a hit
pattern, a mask, and a white-noise realisation. The data map d = Y a + n
needs the synthesis operator Y; each caller applies its own Y to the drawn
a_lm (the test suite uses the oracle's, the benchmark uses the library's).

The paper's application (Sect. 3) is WMAP7 V-band data with the extended
temperature masks (sky fraction about 70 %). That data set is not available
here; the recipes below stand in for it:

* small case   : Nside 16, lmax 32, C_l = 1/(l(l+1)) for l >= 2,
                 sigma^2 = 1e-3 C_2 / h, h = 1 + 2 |sin beta|, mask |b| < 10 deg.
* WMAP-shaped  : Nside 512, lmax 1024, C_l = A/(l(l+1)) exp(-(l/800)^2) B_l^2,
                 A = 2 pi 1000 uK^2, 13' FWHM Gaussian beam, sigma = 2200 uK / sqrt(h),
                 h = 1 + 7 |sin beta| (1 .. 8), mask |b| < asin(0.2) (20 % of the sky)
                 plus 500 discs of radius 0.5 deg at uniform random positions.
* Planck-shaped: Nside 2048, lmax 4096, the same spectrum with a 5' beam,
                 h lognormal (sigma 0.5) per pixel, mask |b| < asin(0.25).

beta is an ecliptic-like latitude, sin beta = n . (sin 60deg, 0, cos 60deg);
b is the latitude of the HEALPix frame. Pixel centres for shaping masks and
hit maps are computed here from the public HEALPix ring definition
(Gorski et al. 2005); nothing here feeds a transform.

a_lm layout: m >= 0 only, m-major, index(l, m) = m (2 lmax + 1 - m) / 2 + l,
complex128.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def npix_of(nside: int) -> int:
    return 12 * nside * nside


def nalm_of(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def alm_lm_arrays(lmax: int):
    """l and m of every a_lm slot in m-major order."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def pixel_centres(nside: int):
    """(z, phi) of every pixel centre in HEALPix RING order."""
    npix = npix_of(nside)
    z = np.empty(npix)
    phi = np.empty(npix)
    p = 0
    for i in range(1, 4 * nside):
        if i < nside:
            n, zz, shift = 4 * i, 1.0 - i * i / (3.0 * nside * nside), 0.5
        elif i <= 3 * nside:
            n, zz = 4 * nside, 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            shift = 0.5 if (i - nside) % 2 == 0 else 0.0
        else:
            ip = 4 * nside - i
            n, zz, shift = 4 * ip, -(1.0 - ip * ip / (3.0 * nside * nside)), 0.5
        z[p:p + n] = zz
        phi[p:p + n] = (np.arange(n) + shift) * (2.0 * math.pi / n)
        p += n
    return z, phi


# --------------------------------------------------------------------------
# spectra


def cl_inverse_square(lmax: int) -> np.ndarray:
    """C_l = 1 / (l (l + 1)) for l >= 2, C_0 = C_1 = 0."""
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    cl[2:] = 1.0 / (l * (l + 1.0))
    return cl


def gaussian_beam(lmax: int, fwhm_arcmin: float) -> np.ndarray:
    sigma = math.radians(fwhm_arcmin / 60.0) / math.sqrt(8.0 * math.log(2.0))
    l = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * l * (l + 1.0) * sigma * sigma)


def cl_lcdm_like(lmax: int, fwhm_arcmin: float, amp: float = 2.0 * math.pi * 1000.0) -> np.ndarray:
    """A / (l (l + 1)) exp(-(l / 800)^2) B_l^2 for l >= 2 (uK^2), C_0 = C_1 = 0."""
    cl = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    cl[2:] = amp / (l * (l + 1.0)) * np.exp(-(l / 800.0) ** 2)
    return cl * gaussian_beam(lmax, fwhm_arcmin) ** 2


def draw_alm(cl: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Gaussian a_lm with <|a_lm|^2> = C_l: a_l0 real N(0, C_l); for m > 0
    real and imaginary parts N(0, C_l / 2) each."""
    lmax = len(cl) - 1
    ls, ms = alm_lm_arrays(lmax)
    var = cl[ls]
    re = rng.standard_normal(len(ls))
    im = rng.standard_normal(len(ls))
    alm = np.where(ms == 0, re * np.sqrt(var), re * np.sqrt(var / 2.0)) + 1j * np.where(
        ms == 0, 0.0, im * np.sqrt(var / 2.0))
    return alm.astype(np.complex128)


# --------------------------------------------------------------------------
# noise and masks


def sin_ecliptic_latitude(z: np.ndarray, phi: np.ndarray) -> np.ndarray:
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return s * np.cos(phi) * math.sin(math.radians(60.0)) + z * math.cos(math.radians(60.0))


def mask_band(z: np.ndarray, sin_b: float) -> np.ndarray:
    """1 = observed, 0 = masked where |sin b| < sin_b."""
    return (np.abs(z) >= sin_b).astype(np.uint8)


def _rings_of(z):
    """Start index of each HEALPix ring in a RING-ordered z array (z is constant along a ring)."""
    starts = np.flatnonzero(np.diff(z) != 0.0) + 1
    return np.concatenate([[0], starts, [z.size]])


def mask_discs(z, phi, mask, ndisc: int, radius_deg: float, rng) -> np.ndarray:
    """Zero `ndisc` discs of radius `radius_deg` at uniform random positions
    (every pixel whose centre is within the radius)."""
    out = mask.copy()
    if ndisc <= 0:
        return out
    cz = rng.uniform(-1.0, 1.0, ndisc)
    cphi = rng.uniform(0.0, 2.0 * math.pi, ndisc)
    cs = np.sqrt(1.0 - cz * cz)
    cosr = math.cos(math.radians(radius_deg))
    sinr = math.sin(math.radians(radius_deg))
    rb = _rings_of(z)
    zr = z[rb[:-1]]                      # ring z, decreasing
    nzr = -zr
    for k in range(ndisc):
        # rings within the disc's z range, and on each the pixels within its phi range (candidates),
        # then the exact angle test on the candidates
        r0 = np.searchsorted(nzr, -min(1.0, cz[k] + sinr) - 1e-12, side="left")
        r1 = np.searchsorted(nzr, -max(-1.0, cz[k] - sinr) + 1e-12, side="right")
        for r in range(r0, r1):
            a, b = rb[r], rb[r + 1]
            n = b - a
            sr = math.sqrt(max(0.0, 1.0 - zr[r] * zr[r]))
            den = sr * cs[k]
            num = cosr - zr[r] * cz[k]
            if den <= 0.0:
                cand = np.arange(a, b) if num <= 0.0 else np.arange(0)
            else:
                c = num / den
                if c > 1.0:
                    continue
                if c <= -1.0:
                    cand = np.arange(a, b)
                else:
                    dphi = math.acos(c)
                    step = 2.0 * math.pi / n
                    j0 = int(math.floor((cphi[k] - dphi - phi[a]) / step)) - 1
                    j1 = int(math.ceil((cphi[k] + dphi - phi[a]) / step)) + 1
                    if j1 - j0 + 1 >= n:
                        cand = np.arange(a, b)
                    else:
                        cand = a + np.mod(np.arange(j0, j1 + 1), n)
            if cand.size:
                dot = sr * np.cos(phi[cand]) * cs[k] * math.cos(cphi[k]) + \
                    sr * np.sin(phi[cand]) * cs[k] * math.sin(cphi[k]) + zr[r] * cz[k]
                out[cand[dot >= cosr]] = 0
    return out


@dataclass
class Problem:
    """One Wiener-filter problem instance (everything but the synthesis)."""
    nside: int
    lmax: int
    cl: np.ndarray          # [lmax+1], beam folded in
    noise_var: np.ndarray   # [Npix] sigma^2 per pixel (finite, > 0)
    mask: np.ndarray        # [Npix] uint8, 1 = observed
    alm_true: np.ndarray    # [nalm] complex128 signal realisation
    noise: np.ndarray       # [Npix] white-noise realisation
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def npix(self) -> int:
        return npix_of(self.nside)

    def data(self, signal_map: np.ndarray) -> np.ndarray:
        """d = s + n (Eq. 1) given the synthesised signal map Y a_true."""
        return np.ascontiguousarray(signal_map + self.noise)


def small_problem(seed: int = 1, nside: int = 16, lmax: int = 32) -> Problem:
    rng = np.random.default_rng(seed)
    cl = cl_inverse_square(lmax)
    z, phi = pixel_centres(nside)
    h = 1.0 + 2.0 * np.abs(sin_ecliptic_latitude(z, phi))
    var = 1e-3 * cl[2] / h
    mask = mask_band(z, math.sin(math.radians(10.0)))
    alm = draw_alm(cl, rng)
    noise = rng.standard_normal(len(z)) * np.sqrt(var)
    return Problem(nside, lmax, cl, var, mask, alm, noise, name=f"small_ns{nside}_l{lmax}_s{seed}")


def wmap_problem(seed: int = 1, nside: int = 512, lmax: int = 1024, ndisc: int = 500,
                 fwhm_arcmin: float = 13.0, noise_scale: float = 1.0) -> Problem:
    """noise_scale multiplies every pixel variance; (nside / 512)^2 keeps the
    noise power per steradian of the Nside 512 map at a smaller nside."""
    rng = np.random.default_rng(seed)
    cl = cl_lcdm_like(lmax, fwhm_arcmin)
    z, phi = pixel_centres(nside)
    h = 1.0 + 7.0 * np.abs(sin_ecliptic_latitude(z, phi))
    var = 2200.0 ** 2 / h * noise_scale
    mask = mask_band(z, 0.2)
    mask = mask_discs(z, phi, mask, ndisc, 0.5, rng)
    alm = draw_alm(cl, rng)
    noise = rng.standard_normal(len(z)) * np.sqrt(var)
    return Problem(nside, lmax, cl, var, mask, alm, noise, name=f"wmap_ns{nside}_l{lmax}_s{seed}")


def planck_problem(seed: int = 1, nside: int = 2048, lmax: int = 4096) -> Problem:
    rng = np.random.default_rng(seed)
    cl = cl_lcdm_like(lmax, 5.0)
    z, phi = pixel_centres(nside)
    h = np.exp(0.5 * rng.standard_normal(len(z)))
    var = 2200.0 ** 2 / (16.0 * h)
    mask = mask_band(z, 0.25)
    alm = draw_alm(cl, rng)
    noise = rng.standard_normal(len(z)) * np.sqrt(var)
    return Problem(nside, lmax, cl, var, mask, alm, noise, name=f"planck_ns{nside}_l{lmax}_s{seed}")


@dataclass
class PolProblem:
    """A temperature-polarisation problem: spectra (TT, EE, BB, TE), per-pixel noise (TT, QQ, QU, UU),
    temperature and polarisation masks, the true (T, E, B) a_lm and a noise realisation [3][Npix]."""
    nside: int
    lmax: int
    cls: tuple
    noise_cov: np.ndarray
    mask_t: np.ndarray
    mask_p: np.ndarray
    alm_true: np.ndarray
    noise: np.ndarray


def pol_wmap_problem(seed: int = 1, nside: int = 512, lmax: int = 1024, ndisc: int = 500,
                     fwhm_arcmin: float = 13.0) -> PolProblem:
    """WMAP-shaped T + P: C_TT as wmap_problem, C_EE = C_TT / 30, C_BB = C_TT / 1000, C_TE = 0.3 sqrt(TT EE);
    noise sigma_T^2 = 2200^2 / h, Q and U twice that with a Q-U correlation of up to 0.2; temperature mask as
    wmap_problem, polarisation mask a 30 % band cut plus the same discs."""
    rng = np.random.default_rng(seed)
    tt = cl_lcdm_like(lmax, fwhm_arcmin)
    ee, bb = tt / 30.0, tt / 1000.0
    te = 0.3 * np.sqrt(tt * ee)
    z, phi = pixel_centres(nside)
    npix = z.size
    h = 1.0 + 7.0 * np.abs(sin_ecliptic_latitude(z, phi))
    cov = np.zeros((npix, 4))
    cov[:, 0] = 2200.0 ** 2 / h
    cov[:, 1] = 2.0 * cov[:, 0]
    cov[:, 3] = 2.0 * cov[:, 0]
    cov[:, 2] = 0.2 * cov[:, 1] * rng.uniform(-1.0, 1.0, npix)
    mt = mask_discs(z, phi, mask_band(z, 0.2), ndisc, 0.5, rng)
    mp = mt & mask_band(z, 0.3)
    g1, g2, g3 = draw_alm(np.ones(lmax + 1), rng), draw_alm(np.ones(lmax + 1), rng), draw_alm(np.ones(lmax + 1), rng)
    ls, _ = alm_lm_arrays(lmax)
    safe = np.where(tt[ls] > 0, tt[ls], 1.0)
    a_t = np.sqrt(tt[ls]) * g1
    a_e = np.where(tt[ls] > 0, te[ls] / np.sqrt(safe), 0.0) * g1 + \
        np.sqrt(np.maximum(ee[ls] - np.where(tt[ls] > 0, te[ls] ** 2 / safe, 0.0), 0.0)) * g2
    a_b = np.sqrt(bb[ls]) * g3
    e1, e2, e3 = rng.standard_normal(npix), rng.standard_normal(npix), rng.standard_normal(npix)
    l11 = np.sqrt(cov[:, 1])
    l21 = cov[:, 2] / l11
    l22 = np.sqrt(cov[:, 3] - l21 ** 2)
    noise = np.array([np.sqrt(cov[:, 0]) * e1, l11 * e2, l21 * e2 + l22 * e3])
    return PolProblem(nside, lmax, (tt, ee, bb, te), cov, mt, mp, np.array([a_t, a_e, a_b]), noise)


def fluctuation_draws(prob: Problem, nrhs: int, seed0: int = 1):
    """Per-RHS signal and noise fluctuations for constrained-realisation style
    batches: a_i ~ N(0, C_l), n_i ~ N(0, sigma^2), seeds seed0 .. seed0+nrhs-1."""
    out = []
    for i in range(nrhs):
        rng = np.random.default_rng(1000003 * (seed0 + i))
        a = draw_alm(prob.cl, rng)
        n = rng.standard_normal(prob.npix) * np.sqrt(prob.noise_var)
        out.append((a, n))
    return out
