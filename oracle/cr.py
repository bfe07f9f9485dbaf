"""Constrained realisations (oracle).

TEST INFRASTRUCTURE ONLY (part of the oracle; used by tests/, the smoke
check and the benchmark's CPU-baseline leg). Shares no code with the CUDA
library.

Sect. 3 (WMAP analysis, last paragraph, and the power-spectra figure): a
Wiener-filter map can be augmented to a constrained realisation, the sum of
the Wiener filter solution and a fluctuation map, which has the correct signal
variance. With s_WF(x) the Wiener filter of data x (Eq. 2), a signal draw
xi ~ N(0, S) and a noise draw n' ~ N(0, N), the constrained realisation is

    s_CR = s_WF(d) + xi - s_WF(Y xi + n'),

a draw from the posterior of s given d: its mean is s_WF(d) and the
fluctuation xi - s_WF(Y xi + n') has the posterior covariance
(S^-1 + Y^T N^-1 Y)^-1, so that over data drawn from the model the
realisation has covariance S.

Random numbers: the draws come from a counter-based generator so that the
CUDA library can draw the same numbers on the device. The generator is
Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011): a 256-bit counter (four 64-bit words) and a
128-bit key, ten rounds of two 64 x 64 -> 128-bit products with multipliers
M0, M1, the high and low halves mixed with the other two words and the key,
and the key advanced by the Weyl constants W0, W1 between rounds. Uniforms are
u = (x >> 11 + 1/2) 2^-53 in (0, 1); normals come in pairs by Box and
Muller's transform, z0 = r cos(2 pi u1), z1 = r sin(2 pi u1),
r = sqrt(-2 ln u0), from words (0, 1) and (2, 3) of each block.

Stream layout of realisation i with seed `seed`: key (seed, 0); counter
(j, kind, i, 0) for block j; kind 0 draws the signal (normal number
2 q + part for a_lm entry q, part 0 = real, 1 = imaginary), kind 1 the noise
(normal number p for pixel p).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """(high, low) 64-bit halves of the 128-bit product of uint64 arrays a, b,
    from four 32 x 32 -> 64-bit partial products."""
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _LO32) + (hl & _LO32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64(counters, key):
    """Philox4x64-10 of counters [n, 4] (uint64) under key (k0, k1): [n, 4] uint64."""
    with np.errstate(over="ignore"):
        x = [np.asarray(counters[:, i], dtype=np.uint64).copy() for i in range(4)]
        k0, k1 = np.uint64(key[0]), np.uint64(key[1])
        for _ in range(10):
            hi0, lo0 = _mulhilo(M0, x[0])
            hi1, lo1 = _mulhilo(M1, x[2])
            x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
            k0 = k0 + W0
            k1 = k1 + W1
    return np.stack(x, axis=1)


def normals(seed, kind, real_index, n):
    """The first n standard normals of stream (kind, realisation real_index)."""
    nblk = (n + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    ctr[:, 1] = np.uint64(kind)
    ctr[:, 2] = np.uint64(real_index)
    w = philox4x64(ctr, (np.uint64(seed), np.uint64(0)))
    u = ((w >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    out = np.empty((nblk, 4))
    for p in (0, 2):
        r = np.sqrt(-2.0 * np.log(u[:, p]))
        out[:, p] = r * np.cos(2.0 * np.pi * u[:, p + 1])
        out[:, p + 1] = r * np.sin(2.0 * np.pi * u[:, p + 1])
    return out.reshape(-1)[:n]


def draw_signal(seed, i, lmax, cl):
    """xi ~ N(0, S): a_l0 = sqrt(C_l) z_re; a_lm = sqrt(C_l / 2) (z_re + i z_im) for m > 0."""
    nalm = O.nalm_of(lmax)
    z = normals(seed, 0, i, 2 * nalm).reshape(nalm, 2)
    ls, ms = O.l_of_index(lmax), O.m_of_index(lmax)
    c = np.asarray(cl, dtype=np.float64)[ls]
    sd = np.where(ms == 0, np.sqrt(c), np.sqrt(c / 2.0))
    return sd * z[:, 0] + 1j * np.where(ms == 0, 0.0, sd * z[:, 1])


def draw_noise(seed, i, noise_var, mask):
    """n' ~ N(0, N): sigma_p z_p on observed pixels, 0 where masked (N^-1 = 0)."""
    var = np.asarray(noise_var, dtype=np.float64)
    z = normals(seed, 1, i, var.size)
    return np.where(np.asarray(mask) != 0, np.sqrt(np.where(np.asarray(mask) != 0, var, 0.0)) * z, 0.0)


def constrained_realisation(nside, lmax, cl, noise_var, mask, d, xi, n_prime, opts=None, wf=None):
    """s_WF(d) + xi - s_WF(Y xi + n'), each Wiener filter by the oracle's
    messenger solve with options `opts`; `wf` may pass s_WF(d) already solved."""
    if wf is None:
        wf = O.solve(nside, lmax, cl, noise_var, mask, d, opts).alm
    fluct_data = O.alm2map(nside, lmax, xi) + n_prime
    return wf + xi - O.solve(nside, lmax, cl, noise_var, mask, fluct_data, opts).alm
