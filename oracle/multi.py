"""Several messenger fields for several observations of one sky (oracle).

TEST INFRASTRUCTURE ONLY (part of the oracle; used by tests/ and the smoke
check). Shares no code with the CUDA library.

Sect. 4 (Conclusion) names more than one messenger field as an extension,
for combining several observations, e.g. of different detectors, in one
analysis. Reading used here: K maps of one sky on one HEALPix grid,
    d_k = Y B_k s + n_k,   k = 1 .. K,
with a beam B_k = diag(b_k,l) per detector (harmonic space), noise N_k
diagonal in pixel space (masked pixels: N_k^-1 = 0) and the signal
covariance S = diag(C_l). The joint Wiener filter (Eq. 2 for all maps) is
    (S^-1 + sum_k B_k Y^T N_k^-1 Y B_k) s = sum_k B_k Y^T N_k^-1 d_k.
Each map gets its own messenger field t_k with covariance T_k = tau_k 1,
tau_k = min diag(N_k) over its observed pixels, Nbar_k = N_k - T_k, and the
pair of Eqs. 3-4 becomes
    Eq. 3 (each k, pixel space)  (Nbar_k^-1 + (lambda T_k)^-1) t_k = Nbar_k^-1 d_k + (lambda T_k)^-1 Y B_k s
    Eq. 4 (harmonic space)       (S^-1 + sum_k B_k (lambda T_k)^-1 B_k) s = sum_k B_k (lambda T_k)^-1 t_k.
Per pixel, Eq. 3 is t_k = Y B_k s + a_k,p (d_k - Y B_k s) with the
single-field gain a_p of oracle.pixel_gain for tau_k; per mode, with T_k of
harmonic power tau_k Omega and g_k = 1 / (lambda tau_k Omega),
    s_lm = sum_k g_k b_k,l t_k,lm / (1 / C_l + sum_k g_k b_k,l^2)   (0 where C_l = 0).
As in the single-field iteration, the basis change is applied to the pixel
increment, t_k,lm = b_k,l s_lm + (Y^dagger u_k)_lm with u_k = t_k - Y B_k s,
so that the fixed point at lambda = 1 is the joint Wiener filter on the grid
(and at lambda > 1 the joint filter with noise N_k + (lambda - 1) T_k). For
K = 1 and b = 1 this is oracle.messenger_step.
Cooling: lambda at scale l is the signal-to-messenger ratio of the combined
filter, C_l sum_k b_k,l^2 / (tau_k Omega) (the value where its gain is 1/2),
clamped to >= 1; the schedule, plateau and stop rules are those of
oracle.solve, with sigma_chi2 = sqrt(2 sum_k n_obs,k). The band limit stays at
lmax (no lmax_SHT reduction while cooling).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import oracle as O


@dataclass
class MultiResult:
    alm: np.ndarray
    iters: int
    converged: bool
    history: list = field(default_factory=list)


def multi_step(nside, lmax, s_alm, ds, ws, gains, beams, taus, cl, lam):
    """One iteration with K messenger fields (full band)."""
    omega = 4.0 * math.pi / (12 * nside * nside)
    ls = O.l_of_index(lmax)
    c = np.asarray(cl, dtype=np.float64)[ls]
    num = np.zeros_like(s_alm)
    den = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 0.0)
    chi2_n = chi2_l_n = 0.0
    for d, w, a_pix, b, tau in zip(ds, ws, gains, beams, taus):
        bl = np.asarray(b, dtype=np.float64)[ls]
        s_map = O.alm2map(nside, lmax, bl * s_alm)            # Y B_k s
        r = d - s_map
        chi2_n += float(np.sum(w * r * r))
        nvar = np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0) + (lam - 1.0) * tau, np.inf)
        chi2_l_n += float(np.sum(np.where(w > 0, r * r / nvar, 0.0)))
        t_alm = bl * s_alm + O.map2alm(nside, lmax, a_pix * r)   # Eq. 3, basis change of t_k - Y B_k s
        g = 1.0 / (lam * tau * omega)
        num += g * bl * t_alm
        den = den + g * bl * bl
    s_new = np.where(c > 0, num / den, 0.0)                    # Eq. 4
    chi2_p = O.chi2_prior(s_alm, cl, lmax)
    return s_new, dict(chi2_prior=chi2_p, chi2_noise=chi2_n, chi2_lambda=chi2_p + chi2_l_n,
                       incr2=O.alm_norm2(s_new - s_alm, lmax), norm2=O.alm_norm2(s_new, lmax))


def lambda_for(l_iter, cl, beams, taus, omega, lmax):
    if l_iter > lmax:
        return 1.0
    r = float(cl[l_iter]) * sum(float(b[l_iter]) ** 2 / (t * omega) for b, t in zip(beams, taus))
    return max(1.0, r)


def solve_multi(nside, lmax, cl, beams, noise_vars, masks, ds, opts: O.Options | None = None, schedule=None,
                callback=None):
    """Joint Wiener filter of K maps by K messenger fields, with the cooling
    and stop rules of oracle.solve; `schedule` runs fixed (lambda, n_iter) levels."""
    opts = opts or O.Options()
    omega = 4.0 * math.pi / (12 * nside * nside)
    taus = [O.messenger_tau(v, m) for v, m in zip(noise_vars, masks)]
    ws = [O.inverse_noise(v, m) for v, m in zip(noise_vars, masks)]
    n_obs = sum(int(np.count_nonzero(m)) for m in masks)
    sigma_chi2 = math.sqrt(2.0 * n_obs)
    s = np.zeros(O.nalm_of(lmax), dtype=np.complex128)
    hist = []

    def run(lam):
        nonlocal s
        gains = [O.pixel_gain(lam, t, w) for t, w in zip(taus, ws)]
        s, rec = multi_step(nside, lmax, s, ds, ws, gains, beams, taus, cl, lam)
        rec.update(lam=lam, chi2=rec["chi2_prior"] + rec["chi2_noise"],
                   rel_incr=math.sqrt(rec["incr2"] / rec["norm2"]) if rec["norm2"] > 0 else 0.0)
        hist.append(rec)
        if callback:
            callback(len(hist), rec, s)
        return rec

    if schedule is not None:
        for lam, n in schedule:
            for _ in range(n):
                run(lam)
        return MultiResult(s, len(hist), True, hist)
    l_iter = opts.l_iter0
    lam = lambda_for(l_iter, cl, beams, taus, omega, lmax) if opts.cooling else 1.0
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
                lam = min(lam, lambda_for(l_iter, cl, beams, taus, omega, lmax))
                level_iters, prev = 0, None
        else:
            if level_iters >= 2 and rec["rel_incr"] <= opts.tol:
                converged = True
                break
            if opts.final_dchi2 > 0 and dchi2 is not None and dchi2 < opts.final_dchi2 * sigma_chi2:
                converged = True
                break
    return MultiResult(s, len(hist), converged, hist)
