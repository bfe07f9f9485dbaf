"""FP64 CPU oracle of the messenger-field Wiener filter (arXiv:1211.0585).

TEST INFRASTRUCTURE ONLY: the slow, plainly written reference that the CUDA
library is checked against. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module. It shares no code with
the CUDA library (paper_1211_0585_gb300/csrc) and does not import it.

What it computes, in the paper's order and notation:

* Eq. 1-2 : the Wiener filter solves (S^-1 + N^-1) s = N^-1 d, with N diagonal
  in pixel space (masked pixels: N^-1 = 0) and S = diag(C_l) in harmonic space.
* Sect. 2 : the messenger field t with covariance T = tau * 1,
  tau = min diag(N) (over observed pixels), Nbar = N - T, and the pair
    Eq. 3  (Nbar^-1 + (lambda T)^-1) t = Nbar^-1 d + (lambda T)^-1 s   (pixel space)
    Eq. 4  (S^-1 + (lambda T)^-1) s = (lambda T)^-1 t                  (harmonic space)
  solved in turn starting from s = t = 0, the basis change being the HEALPix
  map2alm / alm2map pair of wf_oracle.c, applied to the increment t - s
  (the band-limited s keeps its own coefficients; see messenger_step).
  Solving Eq. 3 per pixel with w = 1/sigma^2 (0 where masked) gives
    t_p = s_p + a_p (d_p - s_p),  a_p = lambda tau w_p / (1 + (lambda - 1) tau w_p);
  solving Eq. 4 per (l, m) with white pixel variance tau having harmonic
  power tau * Omega (Omega = 4 pi / Npix) gives
    s_lm = f_l t_lm,  f_l = C_l / (C_l + lambda tau Omega).
* Sect. 3 : the chi^2 = s^+ S^-1 s + (d - s)^+ N^-1 (d - s) monitor; the
  cooling of lambda (start at the signal-to-messenger ratio at l_iter = 20,
  on a chi^2 plateau double l_iter and lower lambda to the ratio there, down
  to 1); the band limit lmax_SHT = l_iter + 100 while lambda > 1; the stop
  rule at lambda = 1.

Readings of points the paper leaves open:
  the ratio that sets lambda is C_l / (tau Omega), clamped to >= 1, so that
  the harmonic filter f_l has its half-power point at l_iter; sigma_chi2 =
  sqrt(2 n_obs); the plateau test is |chi2_k - chi2_{k-1}| < eps * sigma_chi2
  between two iterates of the same level; the band limit is exactly
  min(lmax, l_iter + margin); the primary stop test is the relative increment
  ||s_k - s_{k-1}|| / ||s_k|| <= tol at lambda = 1, the paper's
  Delta chi^2 < 1e-4 sigma_chi2 rule being the alternative.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile wf_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        L.orc_ring_info.argtypes = [i64, i64, dp, ctypes.POINTER(i64), dp, ctypes.POINTER(i64)]
        L.orc_pixel_angles.argtypes = [i64, dp, dp]
        L.orc_lambda.argtypes = [i32, i32, ctypes.c_double, dp]
        L.orc_alm2map.argtypes = [i64, i32, dp, dp]
        L.orc_map2alm.argtypes = [i64, i32, dp, dp]
        L.orc_alm2map_pixels.argtypes = [i64, i32, dp, i64, ctypes.POINTER(i64), dp]
        L.orc_map2alm_modes.argtypes = [i64, i32, dp, i64, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), dp]
        for f in ("orc_ring_info", "orc_pixel_angles", "orc_lambda", "orc_alm2map", "orc_map2alm",
                  "orc_alm2map_pixels", "orc_map2alm_modes"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# --------------------------------------------------------------------------
# geometry, Legendre functions, transforms


def nalm_of(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def ring_info(nside, ring):
    z, phi0 = ctypes.c_double(), ctypes.c_double()
    nphi, off = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().orc_ring_info(nside, ring, ctypes.byref(z), ctypes.byref(nphi), ctypes.byref(phi0),
                               ctypes.byref(off)), "ring_info")
    return z.value, nphi.value, phi0.value, off.value


def pixel_angles(nside):
    npix = 12 * nside * nside
    z, phi = np.empty(npix), np.empty(npix)
    _check(lib().orc_pixel_angles(nside, _dp(z), _dp(phi)), "pixel_angles")
    return z, phi


def legendre(lmax, m, x):
    """lambda_lm(x) for l = 0..lmax (zero for l < m)."""
    out = np.zeros(lmax + 1)
    _check(lib().orc_lambda(lmax, m, float(x), _dp(out)), "lambda")
    return out


def alm2map(nside, lmax, alm):
    """f = Y a (synthesis)."""
    a = np.ascontiguousarray(np.asarray(alm, dtype=np.complex128)).view(np.float64)
    assert a.size == 2 * nalm_of(lmax)
    out = np.empty(12 * nside * nside)
    _check(lib().orc_alm2map(nside, lmax, _dp(a), _dp(out)), "alm2map")
    return out


def map2alm(nside, lmax, f):
    """a = Y^dagger f = Omega Y^T f (uniform weights, no iteration)."""
    m = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    assert m.size == 12 * nside * nside
    out = np.empty(2 * nalm_of(lmax))
    _check(lib().orc_map2alm(nside, lmax, _dp(m), _dp(out)), "map2alm")
    return out.view(np.complex128)


def alm2map_pixels(nside, lmax, alm, pix):
    a = np.ascontiguousarray(np.asarray(alm, dtype=np.complex128)).view(np.float64)
    p = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    out = np.empty(p.size)
    _check(lib().orc_alm2map_pixels(nside, lmax, _dp(a), p.size,
                                    p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out)),
           "alm2map_pixels")
    return out


def map2alm_modes(nside, lmax, f, ls, ms):
    m = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    L = np.ascontiguousarray(np.asarray(ls, dtype=np.int32))
    M = np.ascontiguousarray(np.asarray(ms, dtype=np.int32))
    out = np.empty(2 * L.size)
    _check(lib().orc_map2alm_modes(nside, lmax, _dp(m), L.size,
                                   L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   M.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(out)),
           "map2alm_modes")
    return out.view(np.complex128)


def truncate_alm(alm, lmax, lcut):
    """Sub-vector of a_lm with l <= lcut, in the lcut layout."""
    out = np.zeros(nalm_of(lcut), dtype=np.complex128)
    for m in range(lcut + 1):
        out[alm_index(lcut, m, m):alm_index(lcut, lcut, m) + 1] = \
            alm[alm_index(lmax, m, m):alm_index(lmax, lcut, m) + 1]
    return out


def embed_alm(alm_cut, lcut, lmax):
    """Place an lcut-layout a_lm into the lmax layout, zero for l > lcut."""
    out = np.zeros(nalm_of(lmax), dtype=np.complex128)
    for m in range(lcut + 1):
        out[alm_index(lmax, m, m):alm_index(lmax, lcut, m) + 1] = \
            alm_cut[alm_index(lcut, m, m):alm_index(lcut, lcut, m) + 1]
    return out


def l_of_index(lmax):
    ls = []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
    return np.concatenate(ls)


def m_of_index(lmax):
    ms = []
    for m in range(lmax + 1):
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ms)


def alm_weight(lmax):
    """1 for m = 0, 2 for m > 0: a real field's a_lm with m > 0 stand for two modes."""
    return np.where(m_of_index(lmax) == 0, 1.0, 2.0)


# --------------------------------------------------------------------------
# Eqs. 3-4 and the chi^2 of Sect. 3


def messenger_tau(noise_var, mask):
    """T = tau 1 with tau = min diag(N) over observed pixels (Sect. 2)."""
    obs = np.asarray(mask) != 0
    if not obs.any():
        raise ValueError("no observed pixel")
    return float(np.min(np.asarray(noise_var)[obs]))


def inverse_noise(noise_var, mask):
    """w_p = 1/sigma_p^2 on observed pixels, 0 where masked (N^-1 = 0)."""
    obs = np.asarray(mask) != 0
    return np.where(obs, 1.0 / np.where(obs, noise_var, 1.0), 0.0)


def pixel_gain(lam, tau, w):
    """a_p of the per-pixel solution of Eq. 3, t = s + a_p (d - s)."""
    return lam * tau * w / (1.0 + (lam - 1.0) * tau * w)


def harmonic_filter(lam, tau, omega, cl):
    """f_l of the per-mode solution of Eq. 4, s_lm = f_l t_lm (0 where C_l = 0)."""
    cl = np.asarray(cl, dtype=np.float64)
    return np.where(cl > 0, cl / (cl + lam * tau * omega), 0.0)


def chi2_prior(alm, cl, lmax):
    """s^+ S^-1 s = sum over C_l > 0 of (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / C_l."""
    ls = l_of_index(lmax)
    c = np.asarray(cl)[ls]
    good = c > 0
    return float(np.sum(alm_weight(lmax)[good] * np.abs(alm[good]) ** 2 / c[good]))


def alm_norm2(alm, lmax):
    return float(np.sum(alm_weight(lmax) * np.abs(alm) ** 2))


def posterior_residual(nside, lmax, alm, cl, noise_var, mask, d):
    """How far alm is from the posterior mean of Eq. 2 on the grid: with
    Y = synthesis, Y^T = map2alm / Omega and W = N^-1 (0 where masked), the
    residual of the normal equations (S^-1 + Y^T W Y) a = Y^T W d,
        r = Y^T W (d - Y a) - a / C_l        (modes with C_l > 0),
    relative to b = Y^T W d, in the field's norm (m > 0 counted twice)."""
    omega = 4.0 * np.pi / (12 * nside * nside)
    w = inverse_noise(noise_var, mask)
    c = np.asarray(cl, dtype=np.float64)[l_of_index(lmax)]
    good = c > 0
    r = map2alm(nside, lmax, w * (d - alm2map(nside, lmax, alm))) / omega
    r[good] -= alm[good] / c[good]
    b = map2alm(nside, lmax, w * d) / omega
    wt = alm_weight(lmax)[good]
    return float(np.sqrt(np.sum(wt * np.abs(r[good]) ** 2) / np.sum(wt * np.abs(b[good]) ** 2)))


@dataclass
class StepResult:
    s_alm: np.ndarray      # s^(k), lmax layout
    chi2_prior: float      # s^+ S^-1 s of the input state s^(k-1)
    chi2_noise: float      # (d - s)^+ N^-1 (d - s) of the input state
    chi2_lambda: float     # chi^2 with N replaced by N + (lambda - 1) T, input state
    incr2: float           # ||s^(k) - s^(k-1)||^2 (weighted alm norm)
    norm2: float           # ||s^(k)||^2

    @property
    def chi2(self):
        return self.chi2_prior + self.chi2_noise


def messenger_step(nside, lmax, lsht, s_alm, d, w, a_pix, f_l, cl, lam, tau):
    """One iteration of Sect. 2's outline at band limit lsht.

    s_map = Y s (l <= lsht)
    t - s_map = a_p (d - s_map)                               [Eq. 3, per pixel]
    t_lm = s_lm + Y^dagger (t - s_map)                        [basis change]
    s_lm <- f_l t_lm                                          [Eq. 4, per mode]

    The basis change is applied to the pixel-space increment t - s; the
    band-limited part s keeps its own coefficients. With an orthogonal basis
    change this is the same step; on the HEALPix grid it makes the fixed
    point at lambda = 1 the exact discrete solution of Eq. 2.
    Modes with l > lsht are set to zero.
    """
    s_cut = truncate_alm(s_alm, lmax, lsht)
    s_map = alm2map(nside, lsht, s_cut)
    r = d - s_map
    chi2_n = float(np.sum(w * r * r))
    nvar_lam = np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0) + (lam - 1.0) * tau, np.inf)
    chi2_l_n = float(np.sum(np.where(w > 0, r * r / nvar_lam, 0.0)))
    u = a_pix * r
    t_alm = s_cut + map2alm(nside, lsht, u)
    ls = l_of_index(lsht)
    s_new_cut = np.asarray(f_l)[ls] * t_alm
    s_new = embed_alm(s_new_cut, lsht, lmax)
    chi2_p = chi2_prior(s_alm, cl, lmax)
    return StepResult(s_new, chi2_p, chi2_n, chi2_p + chi2_l_n,
                      alm_norm2(s_new - s_alm, lmax), alm_norm2(s_new, lmax))


# --------------------------------------------------------------------------
# cooling schedule and stop rule (Sect. 3)


@dataclass
class Options:
    tol: float = 1e-6            # relative increment at lambda = 1
    max_iter: int = 10000
    cooling: bool = True
    l_iter0: int = 20
    lmax_margin: int = 100
    plateau_eps: float = 1e-2    # plateau: |d chi2| < eps * sigma_chi2
    final_dchi2: float = 0.0     # > 0: also stop when |d chi2| < final_dchi2 * sigma_chi2 at lambda = 1
    min_level_iters: int = 3
    max_level_iters: int = 1000
    band_limit: bool = True


def lambda_for(l_iter, cl, tau, omega, lmax):
    """lambda at scale l_iter: the signal-to-messenger ratio C_l / (tau Omega), >= 1."""
    if l_iter > lmax:
        return 1.0
    return max(1.0, float(cl[l_iter]) / (tau * omega))


@dataclass
class SolveResult:
    alm: np.ndarray
    iters: int
    converged: bool
    history: list = field(default_factory=list)   # per iteration dicts


def solve(nside, lmax, cl, noise_var, mask, d, opts: Options | None = None, schedule=None,
          alm_init=None, callback=None):
    """Messenger-field Wiener filter with the cooling of Sect. 3.

    `schedule`, if given, is a list of (lambda, lsht, n_iter) levels run as is
    (no plateau or stop test); otherwise the controller decides.
    """
    opts = opts or Options()
    npix = 12 * nside * nside
    omega = 4.0 * math.pi / npix
    tau = messenger_tau(noise_var, mask)
    w = inverse_noise(noise_var, mask)
    n_obs = int(np.count_nonzero(mask))
    sigma_chi2 = math.sqrt(2.0 * n_obs)
    s = np.zeros(nalm_of(lmax), dtype=np.complex128) if alm_init is None else \
        np.array(alm_init, dtype=np.complex128)
    hist = []

    def run_step(lam, lsht):
        nonlocal s
        a_pix = pixel_gain(lam, tau, w)
        f_l = harmonic_filter(lam, tau, omega, cl)
        r = messenger_step(nside, lmax, lsht, s, d, w, a_pix, f_l, cl, lam, tau)
        s = r.s_alm
        rec = dict(lam=lam, lsht=lsht, chi2=r.chi2, chi2_prior=r.chi2_prior, chi2_noise=r.chi2_noise,
                   chi2_lambda=r.chi2_lambda, rel_incr=math.sqrt(r.incr2 / r.norm2) if r.norm2 > 0 else 0.0)
        hist.append(rec)
        if callback:
            callback(len(hist), rec, s)
        return rec

    if schedule is not None:
        for lam, lsht, n in schedule:
            for _ in range(n):
                run_step(lam, lsht)
        return SolveResult(s, len(hist), True, hist)

    l_iter = opts.l_iter0
    lam = lambda_for(l_iter, cl, tau, omega, lmax) if opts.cooling else 1.0
    level_iters = 0
    prev_chi2 = None
    converged = False
    for _ in range(opts.max_iter):
        lsht = lmax if (lam <= 1.0 or not opts.band_limit) else min(lmax, l_iter + opts.lmax_margin)
        rec = run_step(lam, lsht)
        level_iters += 1
        dchi2 = abs(rec["chi2"] - prev_chi2) if (prev_chi2 is not None and level_iters >= 3) else None
        prev_chi2 = rec["chi2"]
        if lam > 1.0:
            plateau = dchi2 is not None and dchi2 < opts.plateau_eps * sigma_chi2 \
                and level_iters >= opts.min_level_iters
            if plateau or level_iters >= opts.max_level_iters:
                l_iter *= 2
                lam = min(lam, lambda_for(l_iter, cl, tau, omega, lmax))
                level_iters = 0
                prev_chi2 = None
        else:
            if level_iters >= 2 and rec["rel_incr"] <= opts.tol:
                converged = True
                break
            if opts.final_dchi2 > 0 and dchi2 is not None and dchi2 < opts.final_dchi2 * sigma_chi2:
                converged = True
                break
    return SolveResult(s, len(hist), converged, hist)


def schedule_of(result: SolveResult):
    """Compress a solve's history into (lambda, lsht, n_iter) levels."""
    out = []
    for h in result.history:
        if out and out[-1][0] == h["lam"] and out[-1][1] == h["lsht"]:
            out[-1][2] += 1
        else:
            out.append([h["lam"], h["lsht"], 1])
    return [tuple(x) for x in out]


def rel_l2(a, b, lmax, cl=None):
    """Relative L2 distance of two a_lm vectors (m > 0 weighted x2), optionally
    restricted to modes with C_l > 0."""
    wgt = alm_weight(lmax)
    if cl is not None:
        wgt = wgt * (np.asarray(cl)[l_of_index(lmax)] > 0)
    num = np.sum(wgt * np.abs(a - b) ** 2)
    den = np.sum(wgt * np.abs(b) ** 2)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)
