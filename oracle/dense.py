"""Dense FP64 tools for tiny HEALPix maps (Nside <= 8).

TEST INFRASTRUCTURE ONLY (part of the oracle). Builds the synthesis matrix Y
explicitly from scipy.special.sph_harm_y at the HEALPix pixel centres, so the
oracle's own transforms (wf_oracle.c) can be checked against an independent
evaluation, and solves the discretised equations directly:

* the messenger iteration as an affine map x -> G x + b on the real degrees
  of freedom of a_lm, G = F (1 - Y^dagger A Y), b = F Y^dagger A d
  (Eqs. 3-4 with t eliminated), its k-step recursion, its fixed point
  (1 - G) x = b and its spectral radius (Sect. 2: convergence is exponential
  and unconditional);
* the Wiener filter itself, Eq. 2, in the same discretisation:
  (D S^-1 + Y^T W Y) x = Y^T W d over the modes with C_l > 0.

Real degrees of freedom of a real field's a_lm (m >= 0, m-major order):
a_l0 is one real number; a_lm for m > 0 is two (Re, Im). D is 1 for m = 0
entries and 2 otherwise, so that x^T D x = sum over all m of |a_lm|^2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import sph_harm_y


def dof_lm(lmax):
    """(l, m, part) of each real degree of freedom; part 0 = Re, 1 = Im."""
    out = []
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            out.append((l, m, 0))
            if m > 0:
                out.append((l, m, 1))
    return out


def pack(alm, lmax):
    x = []
    k = 0
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            x.append(alm[k].real)
            if m > 0:
                x.append(alm[k].imag)
            k += 1
    return np.array(x)


def unpack(x, lmax):
    out = []
    k = 0
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            if m == 0:
                out.append(complex(x[k], 0.0))
                k += 1
            else:
                out.append(complex(x[k], x[k + 1]))
                k += 2
    return np.array(out, dtype=np.complex128)


def dof_weight(lmax):
    return np.array([1.0 if m == 0 else 2.0 for (_, m, _) in dof_lm(lmax)])


def dof_l(lmax):
    return np.array([l for (l, _, _) in dof_lm(lmax)])


def synthesis_matrix(z, phi, lmax):
    """Y with f = Y x: f_p = sum_l a_l0 Y_l0 + 2 Re sum_{m>0} a_lm Y_lm(p)."""
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    cols = []
    for (l, m, part) in dof_lm(lmax):
        y = sph_harm_y(l, m, theta, phi)
        if m == 0:
            cols.append(y.real)
        elif part == 0:
            cols.append(2.0 * y.real)
        else:
            cols.append(-2.0 * y.imag)
    return np.stack(cols, axis=1)


def adjoint_matrix(Y, lmax, npix):
    """Y^dagger with a_lm = Omega sum_p f_p conj(Y_lm(p)), i.e. Omega D^-1 Y^T."""
    omega = 4.0 * math.pi / npix
    return omega * (Y / dof_weight(lmax)[None, :]).T


def affine_map(Y, Ydag, a_pix, f_dof, d):
    """G and b of x_{k+1} = G x_k + b for one messenger iteration,
    x_{k+1} = F (x_k + Y^dagger A (d - Y x_k)): G = F (1 - Y^dagger A Y), b = F Y^dagger A d."""
    n = Y.shape[1]
    G = f_dof[:, None] * (np.eye(n) - Ydag @ (a_pix[:, None] * Y))
    b = f_dof * (Ydag @ (a_pix * d))
    return G, b


def fixed_point(G, b):
    return np.linalg.solve(np.eye(G.shape[0]) - G, b)


def spectral_radius(G):
    return float(np.max(np.abs(np.linalg.eigvals(G))))


def posterior_wf(Y, w, cl_dof, wgt, d):
    """Eq. 2 in the discretisation: minimise x^T D C^-1 x + (d - Y x)^T W (d - Y x)."""
    good = cl_dof > 0
    Yg = Y[:, good]
    A = np.diag(wgt[good] / cl_dof[good]) + Yg.T @ (w[:, None] * Yg)
    x = np.zeros(Y.shape[1])
    x[good] = np.linalg.solve(A, Yg.T @ (w * d))
    return x


def chi2(x, Y, w, d, cl_dof, wgt):
    good = cl_dof > 0
    r = d - Y @ x
    return float(np.sum(wgt[good] * x[good] ** 2 / cl_dof[good]) + np.sum(w * r * r))
