"""Temperature and polarisation (oracle).

TEST INFRASTRUCTURE ONLY (part of the oracle; used by tests/ and the smoke
check). Shares no code with the CUDA library.

Sect. 4 (Conclusion) and the power-spectra figure: the method filters
temperature and polarisation maps together and stays robust there. Reading
used here (the paper gives no polarisation equations): a pixel carries the
Stokes vector d_p = (T, Q, U), the noise covariance N_p is 3 x 3 per pixel
(T independent of Q, U; a 2 x 2 Q-U block), with separate temperature and
polarisation masks (N^-1 = 0 on the masked components); the signal is
S = diag over (l, m) of the 3 x 3 blocks [[C_TT, C_TE, 0], [C_TE, C_EE, 0],
[0, 0, C_BB]] on (a^T, a^E, a^B). The messenger covariance stays T = tau 1,
now over all three components, tau = the smallest eigenvalue of N_p over the
observed components, so Nbar = N - T is positive semi-definite and
  Eq. 3, per pixel (3 x 3):  t_p = s_p + A_p (d_p - s_p),
                             A_p = lambda tau (N_p + (lambda - 1) tau 1)^-1
                                 = lambda tau W_p (1 + (lambda - 1) tau W_p)^-1,  W_p = N_p^-1,
  Eq. 4, per mode:           s_lm = S_l (S_l + lambda tau Omega 1)^-1 t_lm
(the 2 x 2 (T, E) block and B alone), with the basis change applied to the
increment t - s as in the temperature iteration.

Basis change. T uses the spin-0 transforms of wf_oracle.c. (Q, U) use the
spin-2 harmonics, Q +- iU = - sum_lm (a^E_lm +- i a^B_lm) _{+-2}Y_lm, with
_sY_lm = _s lambda_lm(theta) e^{i m phi} and, from the spin-raising operator
(eth eta = -(sin theta)^s (d_theta + i csc theta d_phi)(sin theta)^-s eta) applied twice
to Y_lm and the Legendre equation,
  F+_lm = (_2 lambda + _-2 lambda) / 2 = N_l [(2 (m^2 - l) / s^2 - l (l - 1)) lambda_lm + 2 x c_lm lambda_{l-1,m} / s^2]
  F-_lm = (_2 lambda - _-2 lambda) / 2 = N_l (2 m / s^2) [c_lm lambda_{l-1,m} - (l - 1) x lambda_lm]
with x = cos theta, s^2 = 1 - x^2, N_l = ((l - 1) l (l + 1) (l + 2))^-1/2,
c_lm = sqrt((2 l + 1) / (2 l - 1) (l^2 - m^2)), zero for l < 2. Per ring
(m >= 0; negative m are the complex conjugates, the maps being real):
  Q_m = - sum_l (F+ a^E + i F- a^B),   U_m = - sum_l (F+ a^B - i F- a^E)          (synthesis)
  a^E = - Omega sum_rings (F+ Q~_m + i F- U~_m),  a^B = - Omega sum_rings (F+ U~_m - i F- Q~_m)
with Q~_m = sum_j Q_j e^{-i m phi_j} (the adjoint of the synthesis, uniform weights).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import oracle as O


def spin2_functions(lmax, m, x):
    """(F+, F-)[l] for l = 0 .. lmax at x = cos theta (|x| < 1), zero for l < max(2, m)."""
    lam = O.legendre(lmax, m, x)
    fp, fm = np.zeros(lmax + 1), np.zeros(lmax + 1)
    s2 = (1.0 - x) * (1.0 + x)
    for l in range(max(2, m), lmax + 1):
        nl = 1.0 / math.sqrt((l - 1.0) * l * (l + 1.0) * (l + 2.0))
        c = math.sqrt((2.0 * l + 1.0) / (2.0 * l - 1.0) * (l * l - m * m))
        lm1 = lam[l - 1] if l - 1 >= m else 0.0
        fp[l] = nl * ((2.0 * (m * m - l) / s2 - l * (l - 1.0)) * lam[l] + 2.0 * x * c * lm1 / s2)
        fm[l] = nl * (2.0 * m / s2) * (c * lm1 - (l - 1.0) * x * lam[l])
    return fp, fm


_cache = {}


def _rings(nside, lmax):
    """Per ring: (z, nphi, phi0, offset, F+ [m][l], F- [m][l])."""
    key = (nside, lmax)
    if key not in _cache:
        out = []
        for r in range(4 * nside - 1):
            z, nphi, phi0, off = O.ring_info(nside, r)
            FP = np.zeros((lmax + 1, lmax + 1))
            FM = np.zeros((lmax + 1, lmax + 1))
            for m in range(lmax + 1):
                FP[m], FM[m] = spin2_functions(lmax, m, z)
            out.append((z, nphi, phi0, off, FP, FM))
        _cache[key] = out
    return _cache[key]


def _lm(lmax):
    return O.l_of_index(lmax), O.m_of_index(lmax)


def pol_alm2map(nside, lmax, alm):
    """alm [3][nalm] (T, E, B) -> maps [3][Npix] (T, Q, U)."""
    npix = 12 * nside * nside
    out = np.zeros((3, npix))
    out[0] = O.alm2map(nside, lmax, alm[0])
    ls, ms = _lm(lmax)
    aE, aB = np.asarray(alm[1]), np.asarray(alm[2])
    for z, nphi, phi0, off, FP, FM in _rings(nside, lmax):
        fp, fm = FP[ms, ls], FM[ms, ls]                  # per a_lm entry
        Qm = np.zeros(lmax + 1, dtype=np.complex128)
        Um = np.zeros(lmax + 1, dtype=np.complex128)
        np.add.at(Qm, ms, -(fp * aE + 1j * fm * aB))
        np.add.at(Um, ms, -(fp * aB - 1j * fm * aE))
        phi = phi0 + 2.0 * math.pi * np.arange(nphi) / nphi
        E = np.exp(1j * np.outer(phi, np.arange(lmax + 1)))    # [nphi][m]
        wgt = np.where(np.arange(lmax + 1) == 0, 1.0, 2.0)
        out[1, off:off + nphi] = (E @ (wgt * Qm)).real
        out[2, off:off + nphi] = (E @ (wgt * Um)).real
    return out


def pol_map2alm(nside, lmax, maps):
    """maps [3][Npix] (T, Q, U) -> alm [3][nalm] (T, E, B) = Y^dagger maps (Omega Y^T)."""
    npix = 12 * nside * nside
    omega = 4.0 * math.pi / npix
    ls, ms = _lm(lmax)
    nalm = O.nalm_of(lmax)
    out = np.zeros((3, nalm), dtype=np.complex128)
    out[0] = O.map2alm(nside, lmax, maps[0])
    for z, nphi, phi0, off, FP, FM in _rings(nside, lmax):
        phi = phi0 + 2.0 * math.pi * np.arange(nphi) / nphi
        E = np.exp(-1j * np.outer(np.arange(lmax + 1), phi))   # [m][nphi]
        Qt = omega * (E @ maps[1, off:off + nphi])
        Ut = omega * (E @ maps[2, off:off + nphi])
        fp, fm = FP[ms, ls], FM[ms, ls]
        out[1] += -(fp * Qt[ms] + 1j * fm * Ut[ms])
        out[2] += -(fp * Ut[ms] - 1j * fm * Qt[ms])
    return out


# ---------------------------------------------------------------- noise and signal blocks


def inverse_noise_pol(noise, mask_t, mask_p):
    """W_p = N_p^-1 on the observed components: noise [Npix][4] = (TT, QQ, QU, UU) variances;
    returns [Npix][4] = (w_T, w_QQ, w_QU, w_UU) with zeros where masked."""
    nt, nqq, nqu, nuu = noise[:, 0], noise[:, 1], noise[:, 2], noise[:, 3]
    det = nqq * nuu - nqu * nqu
    ot, op = np.asarray(mask_t) != 0, np.asarray(mask_p) != 0
    w = np.zeros_like(noise)
    w[:, 0] = np.where(ot, 1.0 / np.where(ot, nt, 1.0), 0.0)
    safe = np.where(op, det, 1.0)
    w[:, 1] = np.where(op, nuu / safe, 0.0)
    w[:, 2] = np.where(op, -nqu / safe, 0.0)
    w[:, 3] = np.where(op, nqq / safe, 0.0)
    return w


def messenger_tau_pol(noise, mask_t, mask_p):
    """tau = smallest eigenvalue of N_p over the observed components of every pixel."""
    ot, op = np.asarray(mask_t) != 0, np.asarray(mask_p) != 0
    vals = []
    if ot.any():
        vals.append(np.min(noise[ot, 0]))
    if op.any():
        a, b, c = noise[op, 1], noise[op, 2], noise[op, 3]
        vals.append(np.min(0.5 * (a + c) - np.sqrt(0.25 * (a - c) ** 2 + b * b)))
    if not vals:
        raise ValueError("no observed component")
    return float(min(vals))


def pixel_update(lam, tau, w, r):
    """Eq. 3 per pixel: (u, chi2_N, chi2_lambda_N) with u = A (d - s), A = lambda tau W (1 + c W)^-1,
    c = (lambda - 1) tau, for residuals r [3][Npix]; W given as [Npix][4]."""
    c = (lam - 1.0) * tau
    wt, wqq, wqu, wuu = w[:, 0], w[:, 1], w[:, 2], w[:, 3]
    u = np.zeros_like(r)
    gt = wt / (1.0 + c * wt)                           # T: 1 / (sigma^2 + c), 0 where masked
    u[0] = lam * tau * gt * r[0]
    # (1 + c W)^-1 for the Q-U block, then G = W (1 + c W)^-1 = (N + c)^-1 (0 where masked)
    a11, a12, a21, a22 = 1.0 + c * wqq, c * wqu, c * wqu, 1.0 + c * wuu
    det = a11 * a22 - a12 * a21
    i11, i12, i21, i22 = a22 / det, -a12 / det, -a21 / det, a11 / det
    g11 = wqq * i11 + wqu * i21
    g12 = wqq * i12 + wqu * i22
    g22 = wqu * i12 + wuu * i22
    u[1] = lam * tau * (g11 * r[1] + g12 * r[2])
    u[2] = lam * tau * (g12 * r[1] + g22 * r[2])
    chi2_n = float(np.sum(wt * r[0] ** 2 + wqq * r[1] ** 2 + 2 * wqu * r[1] * r[2] + wuu * r[2] ** 2))
    chi2_l = float(np.sum(gt * r[0] ** 2 + g11 * r[1] ** 2 + 2 * g12 * r[1] * r[2] + g22 * r[2] ** 2))
    return u, chi2_n, chi2_l


def harmonic_update(lam, tau, omega, cls, t, lmax):
    """Eq. 4 per mode: s = S_l (S_l + lambda tau Omega)^-1 t; cls = (TT, EE, BB, TE) [lmax+1]."""
    ls = O.l_of_index(lmax)
    tt, ee, bb, te = (np.asarray(c, dtype=np.float64)[ls] for c in cls)
    k = lam * tau * omega
    a11, a12, a22 = tt + k, te, ee + k
    det = a11 * a22 - a12 * a12
    # S (S + k)^-1 on (T, E): [[tt, te], [te, ee]] [[a22, -a12], [-a12, a11]] / det
    m11 = (tt * a22 - te * a12) / det
    m12 = (-tt * a12 + te * a11) / det
    m21 = (te * a22 - ee * a12) / det
    m22 = (-te * a12 + ee * a11) / det
    s = np.zeros_like(t)
    s[0] = m11 * t[0] + m12 * t[1]
    s[1] = m21 * t[0] + m22 * t[1]
    s[2] = np.where(bb > 0, bb / (bb + k), 0.0) * t[2]
    return s


def chi2_prior_pol(alm, cls, lmax):
    """s^+ S^-1 s over the modes whose covariance block is non-zero (m > 0 counted twice)."""
    ls = O.l_of_index(lmax)
    tt, ee, bb, te = (np.asarray(c, dtype=np.float64)[ls] for c in cls)
    wgt = O.alm_weight(lmax)
    det = tt * ee - te * te
    full = det > 0
    onlyt = (~full) & (tt > 0)
    aT, aE, aB = alm
    q = np.zeros(ls.size)
    q[full] = (ee[full] * np.abs(aT[full]) ** 2 - 2 * te[full] * (aT[full] * np.conj(aE[full])).real
               + tt[full] * np.abs(aE[full]) ** 2) / det[full]
    q[onlyt] = np.abs(aT[onlyt]) ** 2 / tt[onlyt]
    q += np.where(bb > 0, np.abs(aB) ** 2 / np.where(bb > 0, bb, 1.0), 0.0)
    return float(np.sum(wgt * q))


@dataclass
class PolResult:
    alm: np.ndarray
    iters: int
    converged: bool
    history: list = field(default_factory=list)


def lambda_for(l_iter, cls, tau, omega, lmax):
    """lambda from the ratio at l_iter with C_TT (the paper's choice), clamped to >= 1."""
    if l_iter > lmax:
        return 1.0
    return max(1.0, float(cls[0][l_iter]) / (tau * omega))


def solve_pol(nside, lmax, cls, noise, mask_t, mask_p, d, opts: O.Options | None = None, schedule=None,
              callback=None):
    """Joint Wiener filter of (T, Q, U) maps d [3][Npix] by the messenger iteration with the 3 x 3
    messenger (full band), the cooling and stop rules of oracle.solve; `schedule` runs fixed
    (lambda, n_iter) levels."""
    opts = opts or O.Options()
    npix = 12 * nside * nside
    omega = 4.0 * math.pi / npix
    w = inverse_noise_pol(noise, mask_t, mask_p)
    tau = messenger_tau_pol(noise, mask_t, mask_p)
    n_obs = int(np.count_nonzero(mask_t)) + 2 * int(np.count_nonzero(mask_p))
    sigma_chi2 = math.sqrt(2.0 * n_obs)
    s = np.zeros((3, O.nalm_of(lmax)), dtype=np.complex128)
    hist = []

    def run(lam):
        nonlocal s
        smap = pol_alm2map(nside, lmax, s)
        r = d - smap
        u, chi2_n, chi2_l = pixel_update(lam, tau, w, r)
        t = s + pol_map2alm(nside, lmax, u)
        s_new = harmonic_update(lam, tau, omega, cls, t, lmax)
        chi2_p = chi2_prior_pol(s, cls, lmax)
        incr2 = sum(O.alm_norm2(s_new[i] - s[i], lmax) for i in range(3))
        norm2 = sum(O.alm_norm2(s_new[i], lmax) for i in range(3))
        s = s_new
        rec = dict(lam=lam, chi2_prior=chi2_p, chi2_noise=chi2_n, chi2_lambda=chi2_p + chi2_l,
                   chi2=chi2_p + chi2_n, incr2=incr2, norm2=norm2,
                   rel_incr=math.sqrt(incr2 / norm2) if norm2 > 0 else 0.0)
        hist.append(rec)
        if callback:
            callback(len(hist), rec, s)
        return rec

    if schedule is not None:
        for lam, n in schedule:
            for _ in range(n):
                run(lam)
        return PolResult(s, len(hist), True, hist)
    l_iter = opts.l_iter0
    lam = lambda_for(l_iter, cls, tau, omega, lmax) if opts.cooling else 1.0
    level_iters, prev, converged = 0, None, False
    for _ in range(opts.max_iter):
        rec = run(lam)
        level_iters += 1
        dchi2 = abs(rec["chi2"] - prev) if (prev is not None and level_iters >= 3) else None
        prev = rec["chi2"]
        if lam > 1.0:
            plateau = dchi2 is not None and dchi2 < opts.plateau_eps * sigma_chi2 \
                and level_iters >= opts.min_level_iters
            if plateau or level_iters >= opts.max_level_iters:
                l_iter *= 2
                lam = min(lam, lambda_for(l_iter, cls, tau, omega, lmax))
                level_iters, prev = 0, None
        else:
            if level_iters >= 2 and rec["rel_incr"] <= opts.tol:
                converged = True
                break
            if opts.final_dchi2 > 0 and dchi2 is not None and dchi2 < opts.final_dchi2 * sigma_chi2:
                converged = True
                break
    return PolResult(s, len(hist), converged, hist)
