/*
 * FP64 CPU oracle for the messenger-field Wiener filter (Elsner & Wandelt,
 * "Fast Wiener filtering of CMB maps", arXiv:1211.0585).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plainly written reference
 * that the CUDA path is checked against. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Contents (all arithmetic in IEEE double, no blocking or fusion):
 *   - HEALPix RING geometry (Gorski et al. 2005, the public pixelisation
 *     definition): ring latitudes, ring lengths, azimuth offsets.
 *   - orthonormal associated Legendre functions lambda_lm(cos theta) with the
 *     Condon-Shortley phase, by the textbook three-term recurrence in l; the
 *     start value lambda_mm is built by its product formula with power-of-two
 *     rescaling so that sin^m(theta) never underflows.
 *   - alm2map (the synthesis operator Y) and map2alm (Y^dagger = Omega * Y^T,
 *     uniform quadrature weight Omega = 4 pi / Npix, no iteration), both
 *     written as the plain double sums over l and over pixels, the azimuthal
 *     sum being a brute-force DFT evaluated with exact integer reduction of
 *     the phase index.  These are the basis change between pixel space and
 *     harmonic space of Sect. 2 (the "transform ... and transform back" of the
 *     algorithm outline).
 *
 * The messenger iteration itself (Eqs. 3-4), the chi^2 monitor and the
 * cooling schedule of Sect. 3 are written in numpy on top of these functions
 * (oracle/oracle.py).
 *
 * Conventions: a_lm for m >= 0 only (real field), stored m-major,
 * index(l, m) = m (2 lmax + 1 - m) / 2 + l, complex interleaved (re, im).
 * Maps are in HEALPix RING order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* HEALPix RING geometry                                                     */
/* ------------------------------------------------------------------------ */

/* Ring `ring` (0-based, 0 .. 4 nside - 2, north to south).
 * z      : cos(theta) of the ring's pixel centres
 * nphi   : number of pixels in the ring
 * phi0   : azimuth of the ring's first pixel centre
 * offset : RING index of the ring's first pixel
 * Returns 0, or -1 for an out-of-range ring. */
int orc_ring_info(int64_t nside, int64_t ring, double *z, int64_t *nphi, double *phi0,
                  int64_t *offset) {
  int64_t nrings = 4 * nside - 1;
  int64_t npix = 12 * nside * nside;
  if (nside < 1 || ring < 0 || ring >= nrings) return -1;
  int64_t i = ring + 1; /* 1-based ring number counted from the north pole */
  if (i < nside) {      /* north polar cap */
    *z = 1.0 - (double)(i * i) / (3.0 * (double)(nside * nside));
    *nphi = 4 * i;
    *phi0 = M_PI / (4.0 * (double)i);
    *offset = 2 * i * (i - 1);
  } else if (i <= 3 * nside) { /* equatorial belt */
    *z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)nside);
    *nphi = 4 * nside;
    /* rings with (i - nside) even are shifted by half a pixel */
    *phi0 = ((i - nside) % 2 == 0) ? M_PI / (4.0 * (double)nside) : 0.0;
    *offset = 2 * nside * (nside - 1) + (i - nside) * 4 * nside;
  } else { /* south polar cap: mirror of north ring 4 nside - i */
    int64_t ip = 4 * nside - i;
    *z = -(1.0 - (double)(ip * ip) / (3.0 * (double)(nside * nside)));
    *nphi = 4 * ip;
    *phi0 = M_PI / (4.0 * (double)ip);
    *offset = npix - 2 * ip * (ip + 1);
  }
  return 0;
}

/* z = cos(theta) and phi of every pixel centre, RING order. */
int orc_pixel_angles(int64_t nside, double *z_out, double *phi_out) {
  int64_t nrings = 4 * nside - 1;
  for (int64_t r = 0; r < nrings; ++r) {
    double z, phi0;
    int64_t nphi, off;
    if (orc_ring_info(nside, r, &z, &nphi, &phi0, &off)) return -1;
    for (int64_t j = 0; j < nphi; ++j) {
      z_out[off + j] = z;
      phi_out[off + j] = phi0 + 2.0 * M_PI * (double)j / (double)nphi;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Orthonormal associated Legendre functions                                 */
/* ------------------------------------------------------------------------ */

/* lambda_lm(x) with Y_lm(theta, phi) = lambda_lm(cos theta) e^{i m phi},
 * normalised so that 2 pi * integral_{-1}^{1} lambda_lm^2 dx = 1, with the
 * Condon-Shortley phase (-1)^m.
 *
 *   lambda_00      = 1 / sqrt(4 pi)
 *   lambda_mm      = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1}
 *   lambda_{m+1,m} = x sqrt(2m+3) lambda_mm
 *   lambda_lm      = sqrt((4l^2-1)/(l^2-m^2))
 *                    * (x lambda_{l-1,m} - sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)) lambda_{l-2,m})
 *
 * A value is carried as v * 2^(-SCALE * k) with an integer k >= 0; the
 * recurrences are linear, so v can be rescaled by 2^SCALE at any step as long
 * as k is adjusted. Values reported while k > 0 are below 2^-(SCALE/2) and are
 * returned as their (possibly zero) double value.
 *
 * out[l] is written for l = 0 .. lmax; out[l] = 0 for l < m. */
#define ORC_SCALE 512
#define ORC_BIG 0x1p256  /* 2^(SCALE/2) */
#define ORC_SMALL 0x1p-256

int orc_lambda(int lmax, int m, double x, double *out) {
  if (lmax < 0 || m < 0 || m > lmax || !(x >= -1.0 && x <= 1.0)) return -1;
  for (int l = 0; l < m; ++l) out[l] = 0.0;
  double sint = sqrt((1.0 - x) * (1.0 + x));
  double v = 1.0 / sqrt(4.0 * M_PI);
  int k = 0;
  for (int mm = 1; mm <= m; ++mm) {
    v *= -sqrt((2.0 * mm + 1.0) / (2.0 * mm)) * sint;
    if (v != 0.0 && fabs(v) < ORC_SMALL) { v *= 0x1p512; ++k; }
  }
  if (v == 0.0) { /* sin(theta) = 0 and m > 0: the whole column vanishes */
    for (int l = m; l <= lmax; ++l) out[l] = 0.0;
    return 0;
  }
  double vm2 = v; /* value at l-2 (scaled) */
  out[m] = ldexp(v, -ORC_SCALE * k);
  if (m == lmax) return 0;
  double vm1 = x * sqrt(2.0 * m + 3.0) * v; /* value at l-1 (scaled) */
  out[m + 1] = ldexp(vm1, -ORC_SCALE * k);
  for (int l = m + 2; l <= lmax; ++l) {
    double dl = (double)l, dm = (double)m;
    double alpha = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
    double beta = sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
    double vl = alpha * (x * vm1 - beta * vm2);
    vm2 = vm1;
    vm1 = vl;
    if (k > 0 && fabs(vl) > ORC_BIG) {
      vm1 *= 0x1p-512;
      vm2 *= 0x1p-512;
      --k;
    }
    out[l] = (k > 0) ? ldexp(vm1, -ORC_SCALE * k) : vm1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* alm2map and map2alm                                                       */
/* ------------------------------------------------------------------------ */

static inline int64_t alm_index(int lmax, int l, int m) {
  return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

/* Synthesis f = Y a:
 *   f(theta_r, phi_j) = sum_{l,m} a_lm Y_lm = F_0(r) + 2 Re sum_{m>=1} F_m(r) e^{i m phi_j},
 *   F_m(r) = sum_{l>=m} a_lm lambda_lm(z_r).
 * The phase m phi_j = m phi0 + 2 pi (m j mod nphi) / nphi is evaluated with an
 * exact integer reduction of m j. Parallel over rings (independent outputs). */
int orc_alm2map(int64_t nside, int lmax, const double *alm, double *map) {
  if (nside < 1 || lmax < 0) return -1;
  int64_t nrings = 4 * nside - 1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrings; ++r) {
    double z, phi0;
    int64_t nphi, off;
    orc_ring_info(nside, r, &z, &nphi, &phi0, &off);
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
    double *Fre = (double *)malloc(sizeof(double) * (lmax + 1));
    double *Fim = (double *)malloc(sizeof(double) * (lmax + 1));
    double *wc = (double *)malloc(sizeof(double) * nphi);
    double *ws = (double *)malloc(sizeof(double) * nphi);
    if (!lam || !Fre || !Fim || !wc || !ws) {
#pragma omp atomic write
      err = -2;
    } else {
      for (int m = 0; m <= lmax; ++m) {
        orc_lambda(lmax, m, z, lam);
        double sr = 0.0, si = 0.0;
        for (int l = m; l <= lmax; ++l) {
          int64_t idx = alm_index(lmax, l, m);
          sr += alm[2 * idx] * lam[l];
          si += alm[2 * idx + 1] * lam[l];
        }
        /* fold the ring's azimuth offset in: G_m = F_m e^{i m phi0} */
        double c0 = cos(m * phi0), s0 = sin(m * phi0);
        Fre[m] = sr * c0 - si * s0;
        Fim[m] = sr * s0 + si * c0;
      }
      for (int64_t q = 0; q < nphi; ++q) {
        wc[q] = cos(2.0 * M_PI * (double)q / (double)nphi);
        ws[q] = sin(2.0 * M_PI * (double)q / (double)nphi);
      }
      for (int64_t j = 0; j < nphi; ++j) {
        double f = Fre[0];
        for (int m = 1; m <= lmax; ++m) {
          /* e^{i m phi_j} = e^{i m phi0} e^{2 pi i (m j mod nphi) / nphi} */
          int64_t q = ((int64_t)m * j) % nphi;
          f += 2.0 * (Fre[m] * wc[q] - Fim[m] * ws[q]);
        }
        map[off + j] = f;
      }
    }
    free(lam); free(Fre); free(Fim); free(wc); free(ws);
  }
  return err;
}

/* Adjoint synthesis with uniform quadrature weight (map2alm, Y^dagger):
 *   a_lm = Omega * sum_r lambda_lm(z_r) T_m(r),
 *   T_m(r) = sum_j f_j e^{-i m phi_j},   Omega = 4 pi / Npix.
 * Parallel over m (independent outputs). */
int orc_map2alm(int64_t nside, int lmax, const double *map, double *alm) {
  if (nside < 1 || lmax < 0) return -1;
  int64_t nrings = 4 * nside - 1;
  int64_t npix = 12 * nside * nside;
  double omega = 4.0 * M_PI / (double)npix;
  /* per-pixel table of e^{2 pi i q / nphi}, q = 0 .. nphi - 1, for every ring */
  double *wc = (double *)malloc(sizeof(double) * npix);
  double *ws = (double *)malloc(sizeof(double) * npix);
  if (!wc || !ws) { free(wc); free(ws); return -2; }
  for (int64_t r = 0; r < nrings; ++r) {
    double z, phi0;
    int64_t nphi, off;
    orc_ring_info(nside, r, &z, &nphi, &phi0, &off);
    for (int64_t q = 0; q < nphi; ++q) {
      wc[off + q] = cos(2.0 * M_PI * (double)q / (double)nphi);
      ws[off + q] = sin(2.0 * M_PI * (double)q / (double)nphi);
    }
  }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int m = 0; m <= lmax; ++m) {
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
    double *are = (double *)calloc(lmax + 1, sizeof(double));
    double *aim = (double *)calloc(lmax + 1, sizeof(double));
    if (!lam || !are || !aim) {
#pragma omp atomic write
      err = -2;
    } else {
      for (int64_t r = 0; r < nrings; ++r) {
        double z, phi0;
        int64_t nphi, off;
        orc_ring_info(nside, r, &z, &nphi, &phi0, &off);
        /* T_m(r) = e^{-i m phi0} sum_j f_j e^{-2 pi i (m j mod nphi) / nphi} */
        double ur = 0.0, ui = 0.0;
        for (int64_t j = 0; j < nphi; ++j) {
          int64_t q = ((int64_t)m * j) % nphi;
          ur += map[off + j] * wc[off + q];
          ui -= map[off + j] * ws[off + q];
        }
        double c0 = cos(m * phi0), s0 = sin(m * phi0);
        double tr = ur * c0 + ui * s0;
        double ti = ui * c0 - ur * s0;
        orc_lambda(lmax, m, z, lam);
        for (int l = m; l <= lmax; ++l) {
          are[l] += lam[l] * tr;
          aim[l] += lam[l] * ti;
        }
      }
      for (int l = m; l <= lmax; ++l) {
        int64_t idx = alm_index(lmax, l, m);
        alm[2 * idx] = omega * are[l];
        alm[2 * idx + 1] = omega * aim[l];
      }
    }
    free(lam); free(are); free(aim);
  }
  free(wc); free(ws);
  return err;
}

/* Direct evaluation of f = Y a at selected pixels only (for checks at sizes
 * where a full alm2map is too slow): f_p = sum_{l,m} a_lm Y_lm(theta_p, phi_p). */
int orc_alm2map_pixels(int64_t nside, int lmax, const double *alm, int64_t npick,
                       const int64_t *pix, double *out) {
  if (nside < 1 || lmax < 0) return -1;
  int64_t npix = 12 * nside * nside, nrings = 4 * nside - 1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < npick; ++k) {
    int64_t p = pix[k];
    if (p < 0 || p >= npix) {
#pragma omp atomic write
      err = -1;
      continue;
    }
    double z = 0, phi0 = 0, phi;
    int64_t nphi = 0, off = 0, r;
    for (r = 0; r < nrings; ++r) {
      orc_ring_info(nside, r, &z, &nphi, &phi0, &off);
      if (p < off + nphi) break;
    }
    phi = phi0 + 2.0 * M_PI * (double)(p - off) / (double)nphi;
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
    double f = 0.0;
    for (int m = 0; m <= lmax; ++m) {
      orc_lambda(lmax, m, z, lam);
      double c = cos(m * phi), s = sin(m * phi);
      for (int l = m; l <= lmax; ++l) {
        int64_t idx = alm_index(lmax, l, m);
        double y = alm[2 * idx] * c - alm[2 * idx + 1] * s;
        f += (m == 0 ? 1.0 : 2.0) * lam[l] * y;
      }
    }
    free(lam);
    out[k] = f;
  }
  return err;
}

/* map2alm restricted to selected (l, m) pairs:
 * a_lm = Omega * sum_r lambda_lm(z_r) sum_j f_j e^{-i m phi_j}. */
int orc_map2alm_modes(int64_t nside, int lmax, const double *map, int64_t npick,
                      const int32_t *ls, const int32_t *ms, double *out) {
  if (nside < 1 || lmax < 0) return -1;
  int64_t nrings = 4 * nside - 1;
  double omega = 4.0 * M_PI / (double)(12 * nside * nside);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < npick; ++k) {
    int l = ls[k], m = ms[k];
    if (m < 0 || l < m || l > lmax) {
#pragma omp atomic write
      err = -1;
      continue;
    }
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
    double are = 0.0, aim = 0.0;
    for (int64_t r = 0; r < nrings; ++r) {
      double z, phi0;
      int64_t nphi, off;
      orc_ring_info(nside, r, &z, &nphi, &phi0, &off);
      double tr = 0.0, ti = 0.0;
      for (int64_t j = 0; j < nphi; ++j) {
        int64_t q = ((int64_t)m * j) % nphi;
        double ang = (double)m * phi0 + 2.0 * M_PI * (double)q / (double)nphi;
        tr += map[off + j] * cos(ang);
        ti -= map[off + j] * sin(ang);
      }
      orc_lambda(l, m, z, lam);
      are += lam[l] * tr;
      aim += lam[l] * ti;
    }
    free(lam);
    out[2 * k] = omega * are;
    out[2 * k + 1] = omega * aim;
  }
  return err;
}
