// Temperature and polarisation (Sect. 4, Conclusion: the method on T and P
// maps together, robust at their higher condition number; the power-spectra
// figure's TT, EE and TE).
//
// A pixel carries (T, Q, U) with a 3 x 3 noise covariance N_p (T independent
// of the Q-U block), separate temperature and polarisation masks (N^-1 = 0 on
// the masked components), and the signal S_l = [[TT, TE, 0], [TE, EE, 0],
// [0, 0, BB]] on (a^T, a^E, a^B). With T = tau 1 over all three components
// (tau = the smallest eigenvalue of N_p over the observed components) one
// iteration is
//   (s_T, s_Q, s_U) = Y s                    T: spin-0 synthesis; Q, U: spin-2 Legendre stage, ring FFTs
//   u_p = A_p (d_p - s_p),  A_p = lambda tau W_p (1 + (lambda - 1) tau W_p)^-1,  W_p = N_p^-1
//                                            Eq. 3, 3 x 3 per pixel
//   t = s + Y^dagger u                       ring FFTs, spin-0 and spin-2 Legendre analyses
//   s_lm = S_l (S_l + lambda tau Omega)^-1 t_lm   Eq. 4, the (T, E) block and B
// with Q +- iU = - sum (a^E +- i a^B) _{+-2}Y_lm: per ring and m,
//   Q_m = - sum_l (F+ a^E + i F- a^B),  U_m = - sum_l (F+ a^B - i F- a^E),
//   a^E = - sum_rings (F+ Q~_m + i F- U~_m),  a^B = - sum_rings (F+ U~_m - i F- Q~_m),
//   F+- = (_2 lambda_lm +- _-2 lambda_lm) / 2
//       F+ = N_l [(2 (m^2 - l) / s^2 - l (l - 1)) lambda_lm + 2 x c_lm lambda_{l-1,m} / s^2]
//       F- = N_l (2 m / s^2) [c_lm lambda_{l-1,m} - (l - 1) x lambda_lm]
// (N_l = ((l-1) l (l+1) (l+2))^-1/2, c_lm = sqrt((2l+1)/(2l-1) (l^2 - m^2)), x = cos theta,
// s^2 = 1 - x^2; zero for l < 2). On the south ring of a pair F+ takes the
// parity (-1)^{l-m} of lambda_lm and F- the opposite.
//
// The T channel, the azimuthal transforms of all three maps and the
// controller are the scalar plan's kernels (its precision). The spin-2
// Legendre stage reads a precomputed table of (F+, F-) per (l, m, ring pair):
// in double-float with compensated dot products on the FP32 pipe for
// WF_PREC_FP64 plans (GB300's FP64 pipe runs at 1/63 of it), in FP64 for
// WF_PREC_FP64_NATIVE plans. Rows below the first l at which lambda_lm(x_k)
// reaches 2^-100 hold zeros and are not read.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "df.cuh"
#include "wf_internal.h"
#include "wf_plan.h"

struct wf_pol_s {
  virtual ~wf_pol_s() = default;
};

namespace wfk {
namespace {

constexpr int kPolThreads = 256;
constexpr int kPixBlocks = 1024;   // pixel kernel: fixed grid, so its chi^2 partials sum in a fixed order
constexpr size_t kSpin2TableMax = size_t(64) << 30;

__device__ __forceinline__ size_t idx_lm(int lmax, int l, int m) { return (size_t)m * (2 * lmax + 1 - m) / 2 + l; }

// (F+, F-) of every (l, m) at the north ring of pair k: one thread per (m, k), the FP64 recurrence
// from the scalar plan's start values (first l with |lambda| >= 2^-100 and the two values there)
__global__ void spin2_table_kernel(const double *xk, const double2 *rec, const int *ls, const double2 *sv, int lmax,
                                   int RP, double2 *tab, int df) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(lmax + 1) * RP) return;
  const int m = (int)(id / RP), k = (int)(id % RP);
  const double x = xk[k];
  const double s2 = (1.0 - x) * (1.0 + x);
  const size_t base = idx_lm(lmax, m, m);
  const int l0 = ls[id];
  double p1 = 0.0, p2 = 0.0;   // lambda_{l-1}, lambda_{l-2}
  for (int l = m; l <= lmax; ++l) {
    double lam = 0.0;
    if (l >= l0) {
      if (l == l0) lam = sv[id].x;
      else if (l == l0 + 1) lam = sv[id].y;
      else {
        const double2 ab = rec[base + (l - m)];
        lam = ab.x * x * p1 - ab.y * p2;
      }
    }
    double fp = 0.0, fm = 0.0;
    if (l >= 2 && l >= l0) {
      const double dl = l;
      const double nl = 1.0 / sqrt((dl - 1.0) * dl * (dl + 1.0) * (dl + 2.0));
      const double c = sqrt((2.0 * dl + 1.0) / (2.0 * dl - 1.0) * (dl * dl - (double)m * m));
      const double lm1 = l > m ? p1 : 0.0;
      fp = nl * ((2.0 * ((double)m * m - dl) / s2 - dl * (dl - 1.0)) * lam + 2.0 * x * c * lm1 / s2);
      fm = nl * (2.0 * m / s2) * (c * lm1 - (dl - 1.0) * x * lam);
    }
    if (df) {   // (F+ hi, F+ lo, F- hi, F- lo)
      const dfl a = df_from(fp), b = df_from(fm);
      reinterpret_cast<float4 *>(tab)[(base + (l - m)) * RP + k] = make_float4(a.h, a.l, b.h, b.l);
    } else {
      tab[(base + (l - m)) * RP + k] = make_double2(fp, fm);
    }
    p2 = p1;
    p1 = lam;
  }
}

// spin-2 analysis: (a^E, a^B)_lm = - sum over ring pairs of the F+- terms; one CTA per m,
// a warp per l, lanes over ring pairs
__global__ void __launch_bounds__(kPolThreads) spin2_analysis_kernel(const Ctl *gate, const double2 *tab,
                                                                      const double4_32a *FTQ, const double4_32a *FTU,
                                                                      int lmax, int RP, double2 *aE, double2 *aB) {
  if (gate && gate->done) return;
  extern __shared__ double4_32a pol_sm[];
  double4_32a *q = pol_sm, *u = pol_sm + RP;
  const int m = blockIdx.x;
  for (int k = threadIdx.x; k < RP; k += blockDim.x) {
    q[k] = FTQ[(size_t)m * RP + k];
    u[k] = FTU[(size_t)m * RP + k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const size_t base = idx_lm(lmax, m, m);
  for (int l = m + warp; l <= lmax; l += nw) {
    const double p = ((l - m) & 1) ? -1.0 : 1.0;
    double er = 0.0, ei = 0.0, br = 0.0, bi = 0.0;
    const double2 *row = tab + (base + (l - m)) * RP;
    for (int k = lane; k < RP; k += 32) {
      const double2 f = row[k];
      const double4_32a Q = q[k], U = u[k];
      // F+ sees Q_N + p Q_S, U_N + p U_S; F- sees Q_N - p Q_S, U_N - p U_S
      const double qpr = Q.x + p * Q.z, qpi = Q.y + p * Q.w, qmr = Q.x - p * Q.z, qmi = Q.y - p * Q.w;
      const double upr = U.x + p * U.z, upi = U.y + p * U.w, umr = U.x - p * U.z, umi = U.y - p * U.w;
      // a^E = -(F+ Q+ + i F- U-),  a^B = -(F+ U+ - i F- Q-)
      er -= f.x * qpr - f.y * umi;
      ei -= f.x * qpi + f.y * umr;
      br -= f.x * upr + f.y * qmi;
      bi -= f.x * upi - f.y * qmr;
    }
    for (int o = 16; o > 0; o >>= 1) {
      er += __shfl_xor_sync(0xffffffffu, er, o);
      ei += __shfl_xor_sync(0xffffffffu, ei, o);
      br += __shfl_xor_sync(0xffffffffu, br, o);
      bi += __shfl_xor_sync(0xffffffffu, bi, o);
    }
    if (lane == 0) {
      aE[base + (l - m)] = l >= 2 ? make_double2(er, ei) : make_double2(0.0, 0.0);
      aB[base + (l - m)] = l >= 2 ? make_double2(br, bi) : make_double2(0.0, 0.0);
    }
  }
}

// spin-2 synthesis: Q_m, U_m on both rings of every pair; one CTA per m, a thread per ring pair
__global__ void __launch_bounds__(kPolThreads) spin2_synthesis_kernel(const Ctl *gate, const double2 *tab,
                                                                       const double2 *aE, const double2 *aB,
                                                                       int lmax, int RP, double4_32a *FSQ,
                                                                       double4_32a *FSU) {
  if (gate && gate->done) return;
  extern __shared__ double2 pol_sa[];
  const int m = blockIdx.x;
  const int Lm = lmax - m + 1;
  double2 *e = pol_sa, *b = pol_sa + Lm;
  const size_t base = idx_lm(lmax, m, m);
  for (int i = threadIdx.x; i < Lm; i += blockDim.x) {
    e[i] = aE[base + i];
    b[i] = aB[base + i];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < RP; k += blockDim.x) {
    double qnr = 0, qni = 0, qsr = 0, qsi = 0, unr = 0, uni = 0, usr = 0, usi = 0;
    for (int i = (m < 2 ? 2 - m : 0); i < Lm; ++i) {
      const double2 f = tab[(base + i) * RP + k];
      const double p = (i & 1) ? -1.0 : 1.0;
      const double2 E = e[i], B = b[i];
      // north: Q = -(F+ E + i F- B), U = -(F+ B - i F- E); south: F+ -> p F+, F- -> -p F-
      const double aqr = f.x * E.x - f.y * B.y, aqi = f.x * E.y + f.y * B.x;   // F+ E + i F- B
      const double bqr = f.x * E.x + f.y * B.y, bqi = f.x * E.y - f.y * B.x;   // F+ E - i F- B
      const double aur = f.x * B.x + f.y * E.y, aui = f.x * B.y - f.y * E.x;   // F+ B - i F- E
      const double bur = f.x * B.x - f.y * E.y, bui = f.x * B.y + f.y * E.x;   // F+ B + i F- E
      qnr -= aqr; qni -= aqi;
      qsr -= p * bqr; qsi -= p * bqi;
      unr -= aur; uni -= aui;
      usr -= p * bur; usi -= p * bui;
    }
    FSQ[(size_t)m * RP + k] = make_double4_32a(qnr, qni, qsr, qsi);
    FSU[(size_t)m * RP + k] = make_double4_32a(unr, uni, usr, usi);
  }
}

// ---- double-float spin-2 Legendre stage
__device__ __forceinline__ float4 cdf(double re, double im) {   // complex double-float (re hi, re lo, im hi, im lo)
  const dfl a = df_from(re), b = df_from(im);
  return make_float4(a.h, a.l, b.h, b.l);
}
__device__ __forceinline__ dfl dneg(dfl a) { return dfl{-a.h, -a.l}; }

// spin-2 analysis in double-float: one CTA per m, a warp per l, lanes over
// ring pairs. Shared memory holds, per ring pair, Q_N + Q_S, Q_N - Q_S, U_N + U_S,
// U_N - U_S (the two parities' combinations of the rings' coefficients).
__global__ void __launch_bounds__(kPolThreads) spin2_analysis_df_kernel(const Ctl *gate, const float4 *tab,
                                                                         const int *ls, const double4_32a *FTQ,
                                                                         const double4_32a *FTU, int lmax, int RP,
                                                                         double2 *aE, double2 *aB) {
  if (gate && gate->done) return;
  extern __shared__ float4 pol_dsm[];   // [RP][4]
  const int m = blockIdx.x;
  for (int k = threadIdx.x; k < RP; k += blockDim.x) {
    const double4_32a Qv = FTQ[(size_t)m * RP + k], Uv = FTU[(size_t)m * RP + k];
    pol_dsm[4 * k + 0] = cdf(Qv.x + Qv.z, Qv.y + Qv.w);
    pol_dsm[4 * k + 1] = cdf(Qv.x - Qv.z, Qv.y - Qv.w);
    pol_dsm[4 * k + 2] = cdf(Uv.x + Uv.z, Uv.y + Uv.w);
    pol_dsm[4 * k + 3] = cdf(Uv.x - Uv.z, Uv.y - Uv.w);
  }
  __syncthreads();
  // a warp takes l and l + 1 (l - m even, then odd): both read the same four combinations, the even
  // l as (Q+, Q-, U+, U-) = (N + S, N - S), the odd one with the two swapped
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const size_t base = idx_lm(lmax, m, m);
  for (int l = m + 2 * warp; l <= lmax; l += 2 * nw) {
    const bool has1 = l + 1 <= lmax;
    float S[8], C[8];   // [0..3]: l, [4..7]: l + 1
#pragma unroll
    for (int j = 0; j < 8; ++j) { S[j] = 0.f; C[j] = 0.f; }
    const float4 *row0 = tab + (base + (l - m)) * RP, *row1 = row0 + RP;
    // two ring pairs per step, every global load of both issued before the products
    auto term = [&](int lsk, float4 f0, float4 f1, int k) {
      if (l + 1 < lsk) return;   // F+- = 0 below the ring pair's first l
      const float4 A = pol_dsm[4 * k + 0], Bq = pol_dsm[4 * k + 1];
      const float4 Cu = pol_dsm[4 * k + 2], Du = pol_dsm[4 * k + 3];
      // a^E = -(F+ Q+ + i F- U-),  a^B = -(F+ U+ - i F- Q-)
      if (l >= lsk) {   // l: Q+ = A, Q- = Bq, U+ = Cu, U- = Du
        const dfl fp = {f0.x, f0.y}, fm = {f0.z, f0.w};
        dot2_acc(S[0], C[0], fp, dneg(dfl{A.x, A.y}));
        dot2_acc(S[0], C[0], fm, dfl{Du.z, Du.w});
        dot2_acc(S[1], C[1], fp, dneg(dfl{A.z, A.w}));
        dot2_acc(S[1], C[1], fm, dneg(dfl{Du.x, Du.y}));
        dot2_acc(S[2], C[2], fp, dneg(dfl{Cu.x, Cu.y}));
        dot2_acc(S[2], C[2], fm, dneg(dfl{Bq.z, Bq.w}));
        dot2_acc(S[3], C[3], fp, dneg(dfl{Cu.z, Cu.w}));
        dot2_acc(S[3], C[3], fm, dfl{Bq.x, Bq.y});
      }
      if (has1) {   // l + 1: Q+ = Bq, Q- = A, U+ = Du, U- = Cu
        const dfl fp = {f1.x, f1.y}, fm = {f1.z, f1.w};
        dot2_acc(S[4], C[4], fp, dneg(dfl{Bq.x, Bq.y}));
        dot2_acc(S[4], C[4], fm, dfl{Cu.z, Cu.w});
        dot2_acc(S[5], C[5], fp, dneg(dfl{Bq.z, Bq.w}));
        dot2_acc(S[5], C[5], fm, dneg(dfl{Cu.x, Cu.y}));
        dot2_acc(S[6], C[6], fp, dneg(dfl{Du.x, Du.y}));
        dot2_acc(S[6], C[6], fm, dneg(dfl{A.z, A.w}));
        dot2_acc(S[7], C[7], fp, dneg(dfl{Du.z, Du.w}));
        dot2_acc(S[7], C[7], fm, dfl{A.x, A.y});
      }
    };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = lane; k < RP; k += 64) {
      const int ka = k, kb = k + 32;
      const int la = ls[(size_t)m * RP + ka], lb = kb < RP ? ls[(size_t)m * RP + kb] : lmax + 2;
      const float4 fa0 = l >= la ? row0[ka] : z4, fa1 = has1 && l + 1 >= la ? row1[ka] : z4;
      const float4 fb0 = l >= lb ? row0[kb] : z4, fb1 = has1 && l + 1 >= lb ? row1[kb] : z4;
      term(la, fa0, fa1, ka);
      if (kb < RP) term(lb, fb0, fb1, kb);
    }
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = (double)S[j] + (double)C[j];
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    if (lane == 0) {
      aE[base + (l - m)] = l >= 2 ? make_double2(v[0], v[1]) : make_double2(0.0, 0.0);
      aB[base + (l - m)] = l >= 2 ? make_double2(v[2], v[3]) : make_double2(0.0, 0.0);
      if (has1) {
        aE[base + (l + 1 - m)] = l + 1 >= 2 ? make_double2(v[4], v[5]) : make_double2(0.0, 0.0);
        aB[base + (l + 1 - m)] = l + 1 >= 2 ? make_double2(v[6], v[7]) : make_double2(0.0, 0.0);
      }
    }
  }
}

// spin-2 synthesis in double-float: one CTA per m, a thread per ring pair.
// The eight products F+ E.re, F- B.im, F+ E.im, F- B.re, F+ B.re, F- E.im,
// F+ B.im, F- E.re are summed separately over even (S0) and odd (S1) l - m;
// the north ring takes even + odd, the south ring (parity (-1)^(l-m) for F+,
// the opposite for F-) even - odd.
__global__ void __launch_bounds__(kPolThreads) spin2_synthesis_df_kernel(const Ctl *gate, const float4 *tab,
                                                                          const int *ls, const double2 *aE,
                                                                          const double2 *aB, int lmax, int RP,
                                                                          double4_32a *FSQ, double4_32a *FSU) {
  if (gate && gate->done) return;
  extern __shared__ float4 pol_dsa[];   // [Lm][2]: E, B as complex double-float
  const int m = blockIdx.x;
  const int Lm = lmax - m + 1;
  const size_t base = idx_lm(lmax, m, m);
  for (int i = threadIdx.x; i < Lm; i += blockDim.x) {
    pol_dsa[2 * i] = cdf(aE[base + i].x, aE[base + i].y);
    pol_dsa[2 * i + 1] = cdf(aB[base + i].x, aB[base + i].y);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < RP; k += blockDim.x) {
    float S0[8], C0[8], S1[8], C1[8];   // compile-time indices: the sums stay in registers
#pragma unroll
    for (int j = 0; j < 8; ++j) { S0[j] = 0.f; C0[j] = 0.f; S1[j] = 0.f; C1[j] = 0.f; }
    auto accum4 = [&](int i, float4 f, float(&Sa)[8], float(&Ca)[8]) {
      const dfl fp = {f.x, f.y}, fm = {f.z, f.w};
      const float4 E = pol_dsa[2 * i], Bv = pol_dsa[2 * i + 1];
      const dfl er = {E.x, E.y}, ei = {E.z, E.w}, br = {Bv.x, Bv.y}, bi = {Bv.z, Bv.w};
      dot2_acc(Sa[0], Ca[0], fp, er);
      dot2_acc(Sa[1], Ca[1], fm, bi);
      dot2_acc(Sa[2], Ca[2], fp, ei);
      dot2_acc(Sa[3], Ca[3], fm, br);
      dot2_acc(Sa[4], Ca[4], fp, br);
      dot2_acc(Sa[5], Ca[5], fm, ei);
      dot2_acc(Sa[6], Ca[6], fp, bi);
      dot2_acc(Sa[7], Ca[7], fm, er);
    };
    auto accum = [&](int i, float(&Sa)[8], float(&Ca)[8]) { accum4(i, tab[(base + i) * RP + k], Sa, Ca); };
    int i = max(m < 2 ? 2 - m : 0, ls[(size_t)m * RP + k] - m);
    if (i < Lm && (i & 1)) accum(i++, S1, C1);
    for (; i + 3 < Lm; i += 4) {   // four rows of the table in flight
      const float4 f0 = tab[(base + i) * RP + k], f1 = tab[(base + i + 1) * RP + k];
      const float4 f2 = tab[(base + i + 2) * RP + k], f3 = tab[(base + i + 3) * RP + k];
      accum4(i, f0, S0, C0);
      accum4(i + 1, f1, S1, C1);
      accum4(i + 2, f2, S0, C0);
      accum4(i + 3, f3, S1, C1);
    }
    for (; i + 1 < Lm; i += 2) {
      accum(i, S0, C0);
      accum(i + 1, S1, C1);
    }
    if (i < Lm) accum(i, S0, C0);
    double e[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      e[j] = (double)S0[j] + (double)C0[j];
      o[j] = (double)S1[j] + (double)C1[j];
    }
    // north: Q = -(F+ E + i F- B), U = -(F+ B - i F- E); south: F+ -> p F+, F- -> -p F-
    const double qnr = -((e[0] + o[0]) - (e[1] + o[1])), qni = -((e[2] + o[2]) + (e[3] + o[3]));
    const double qsr = -((e[0] - o[0]) + (e[1] - o[1])), qsi = -((e[2] - o[2]) - (e[3] - o[3]));
    const double unr = -((e[4] + o[4]) + (e[5] + o[5])), uni = -((e[6] + o[6]) - (e[7] + o[7]));
    const double usr = -((e[4] - o[4]) - (e[5] - o[5])), usi = -((e[6] - o[6]) + (e[7] - o[7]));
    FSQ[(size_t)m * RP + k] = make_double4_32a(qnr, qni, qsr, qsi);
    FSU[(size_t)m * RP + k] = make_double4_32a(unr, uni, usr, usi);
  }
}

// Eq. 3 per pixel with the 3 x 3 messenger and the chi^2 partials (sum r^T W r and r^T (N + (lambda-1) tau)^-1 r).
// The gains (N + (lambda - 1) tau)^-1 depend on lambda only: each block keeps those of its pixels (the grid
// is fixed, so a block always owns the same pixels) with the lambda they belong to, and recomputes them,
// divisions on the FP64 pipe, only when lambda changes.
__global__ void __launch_bounds__(kPolThreads) pol_pixel_kernel(const Ctl *ctl, long long npix, double tau,
                                                                 const double *s, const double *d, const double4_32a *w,
                                                                 double4_32a *gain, double *gainlam, double *u,
                                                                 double *part) {
  __shared__ double red[2][kPolThreads / 32];
  if (ctl->done) return;
  const double lam = ctl->lambda, c = (lam - 1.0) * tau, lt = lam * tau;
  const bool fresh = gainlam[blockIdx.x] == lam;   // this block's gains are already at this lambda
  double c2n = 0.0, c2l = 0.0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    const double4_32a W = w[p];   // (w_T, w_QQ, w_QU, w_UU)
    const double rt = d[p] - s[p], rq = d[npix + p] - s[npix + p], ru = d[2 * npix + p] - s[2 * npix + p];
    double gt, g11, g12, g22;
    if (fresh) {
      const double4_32a G = gain[p];
      gt = G.x; g11 = G.y; g12 = G.z; g22 = G.w;
    } else {
      gt = W.x / (1.0 + c * W.x);
      const double a11 = 1.0 + c * W.y, a12 = c * W.z, a22 = 1.0 + c * W.w;
      const double det = a11 * a22 - a12 * a12;
      const double i11 = a22 / det, i12 = -a12 / det, i22 = a11 / det;
      g11 = W.y * i11 + W.z * i12;
      g12 = W.y * i12 + W.z * i22;
      g22 = W.z * i12 + W.w * i22;
      gain[p] = make_double4_32a(gt, g11, g12, g22);
    }
    u[p] = lt * gt * rt;
    u[npix + p] = lt * (g11 * rq + g12 * ru);
    u[2 * npix + p] = lt * (g12 * rq + g22 * ru);
    c2n += W.x * rt * rt + W.y * rq * rq + 2.0 * W.z * rq * ru + W.w * ru * ru;
    c2l += gt * rt * rt + g11 * rq * rq + 2.0 * g12 * rq * ru + g22 * ru * ru;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c2n += __shfl_xor_sync(0xffffffffu, c2n, o);
    c2l += __shfl_xor_sync(0xffffffffu, c2l, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = c2n; red[1][threadIdx.x >> 5] = c2l; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kPolThreads / 32; ++i) { a += red[0][i]; b += red[1][i]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
    if (!fresh) gainlam[blockIdx.x] = lam;   // after the barrier: every gain of the block is written
  }
}

// Eq. 4 with the (T, E) block and B, the prior chi^2 of the input state, increment and norm per m
__global__ void __launch_bounds__(128) pol_eq4_kernel(const Ctl *ctl, int lmax, long long nalm, double tau,
                                                       double omega, const double *cls, const double2 *ta,
                                                       double2 *s, double *m_part) {
  __shared__ double red[3][4];
  if (ctl->done) return;
  const int m = blockIdx.x;
  const double k = ctl->lambda * tau * omega;
  const double wgt = (m == 0) ? 1.0 : 2.0;
  const double *TT = cls, *EE = cls + (lmax + 1), *BB = cls + 2 * (lmax + 1), *TE = cls + 3 * (lmax + 1);
  double c2 = 0.0, inc = 0.0, nrm = 0.0;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const size_t q = idx_lm(lmax, l, m);
    const double2 sT = s[q], sE = s[nalm + q], sB = s[2 * nalm + q];
    const double2 tT = make_double2(sT.x + ta[q].x, sT.y + ta[q].y);
    const double2 tE = make_double2(sE.x + ta[nalm + q].x, sE.y + ta[nalm + q].y);
    const double2 tB = make_double2(sB.x + ta[2 * nalm + q].x, sB.y + ta[2 * nalm + q].y);
    const double tt = TT[l], ee = EE[l], bb = BB[l], te = TE[l];
    // S (S + k)^-1 on (T, E)
    const double a11 = tt + k, a12 = te, a22 = ee + k, det = a11 * a22 - a12 * a12;
    const double m11 = (tt * a22 - te * a12) / det, m12 = (-tt * a12 + te * a11) / det;
    const double m21 = (te * a22 - ee * a12) / det, m22 = (-te * a12 + ee * a11) / det;
    const double fb = bb > 0.0 ? bb / (bb + k) : 0.0;
    const double2 nT = make_double2(m11 * tT.x + m12 * tE.x, m11 * tT.y + m12 * tE.y);
    const double2 nE = make_double2(m21 * tT.x + m22 * tE.x, m21 * tT.y + m22 * tE.y);
    const double2 nB = make_double2(fb * tB.x, fb * tB.y);
    // prior chi^2 of the input state
    const double sdet = tt * ee - te * te;
    double qf = 0.0;
    if (sdet > 0.0) {
      qf = (ee * (sT.x * sT.x + sT.y * sT.y) - 2.0 * te * (sT.x * sE.x + sT.y * sE.y) +
            tt * (sE.x * sE.x + sE.y * sE.y)) / sdet;
    } else if (tt > 0.0) {
      qf = (sT.x * sT.x + sT.y * sT.y) / tt;
    }
    if (bb > 0.0) qf += (sB.x * sB.x + sB.y * sB.y) / bb;
    c2 += wgt * qf;
    const double d1x = nT.x - sT.x, d1y = nT.y - sT.y, d2x = nE.x - sE.x, d2y = nE.y - sE.y;
    const double d3x = nB.x - sB.x, d3y = nB.y - sB.y;
    inc += wgt * (d1x * d1x + d1y * d1y + d2x * d2x + d2y * d2y + d3x * d3x + d3y * d3y);
    nrm += wgt * (nT.x * nT.x + nT.y * nT.y + nE.x * nE.x + nE.y * nE.y + nB.x * nB.x + nB.y * nB.y);
    s[q] = nT;
    s[nalm + q] = nE;
    s[2 * nalm + q] = nB;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    inc += __shfl_xor_sync(0xffffffffu, inc, o);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = c2; red[1][threadIdx.x >> 5] = inc; red[2][threadIdx.x >> 5] = nrm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, e = 0.0;
    for (int i = 0; i < 4; ++i) { a += red[0][i]; b += red[1][i]; e += red[2][i]; }
    m_part[3 * m] = a;
    m_part[3 * m + 1] = b;
    m_part[3 * m + 2] = e;
  }
}

struct Pol : wf_pol_s {
  Plan *P = nullptr;   // scalar plan: geometry, tables, the T channel's Fourier buffers and stream
  int nside = 0, lmax = 0, RP = 0;
  long long npix = 0, nalm = 0, n_obs = 0;
  double tau = 0.0, omega = 0.0;
  wf_options opt{};
  std::vector<double> h_tt;
  double2 *d_tab = nullptr;                       // (F+, F-) [nalm][RP]: double2, or float4 double-float when df
  bool df = false;                                // double-float spin-2 stage (WF_PREC_FP64 plans)
  double *d_cls = nullptr;                        // [4][lmax+1] TT, EE, BB, TE
  double4_32a *d_w = nullptr;                         // [npix] (w_T, w_QQ, w_QU, w_UU)
  double4_32a *d_gain = nullptr;                      // [npix] cached 3 x 3 gains (g_T, g_QQ, g_QU, g_UU)
  double *d_gainlam = nullptr;                    // [kPixBlocks] lambda of each block's cached gains
  double *d_d = nullptr, *d_map = nullptr, *d_u = nullptr;   // [3][npix]
  double2 *d_s = nullptr, *d_ta = nullptr;        // [3][nalm]
  double4_32a *d_FSQ = nullptr, *d_FSU = nullptr, *d_FTQ = nullptr, *d_FTU = nullptr;
  double *d_part = nullptr, *d_m_part = nullptr;
  Ctl *d_ctl = nullptr, *h_ctl = nullptr;
  wf_iter_record *d_hist = nullptr;
  int hist_cap = 0;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void *> allocs;

  ~Pol() override {
    if (graph) cudaGraphExecDestroy(graph);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (h_ctl) cudaFreeHost(h_ctl);
    for (void *p : allocs) cudaFree(p);
    if (P) wf_plan_destroy(P);
  }
  wf_status dalloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) { *p = nullptr; return cuda_status(e, "cudaMalloc (polarisation)"); }
    allocs.push_back(*p);
    return WF_OK;
  }
  cudaStream_t stream() const { return P->run_stream(); }
  // (T, E, B) a_lm -> (T, Q, U) maps, and back (the adjoint), on the plan's kernels and the spin-2 stage
  void synth(cudaStream_t s, const double2 *alm, double *map, const Ctl *gate) const;
  void analysis(cudaStream_t s, const double *map, double2 *alm, const Ctl *gate) const;
  void enqueue_iteration(cudaStream_t s);
};

void Pol::synth(cudaStream_t s, const double2 *alm, double *map, const Ctl *gate) const {
  LegArgs la = P->leg_args();
  la.lsht = lmax;
  la.alm_in = alm;
  la.gate = gate;
  P->launch_leg(la, s, LEG_SYNTH);                                    // T -> the plan's FS
  if (df) {
    raise_smem_cap(reinterpret_cast<const void *>(spin2_synthesis_df_kernel));
    spin2_synthesis_df_kernel<<<lmax + 1, kPolThreads, sizeof(float4) * 2 * (lmax + 1), s>>>(
        gate, reinterpret_cast<const float4 *>(d_tab), P->d_ls, alm + nalm, alm + 2 * nalm, lmax, RP, d_FSQ, d_FSU);
  } else {
    raise_smem_cap(reinterpret_cast<const void *>(spin2_synthesis_kernel));
    spin2_synthesis_kernel<<<lmax + 1, kPolThreads, sizeof(double2) * 2 * (lmax + 1), s>>>(
        gate, d_tab, alm + nalm, alm + 2 * nalm, lmax, RP, d_FSQ, d_FSU);
  }
  const double4_32a *fs[3] = {P->d_FS, d_FSQ, d_FSU};
  for (int c = 0; c < 3; ++c) {
    RingArgs ra = P->ring_args();
    ra.lsht = lmax;
    ra.FS = fs[c];
    ra.map_out = map + (size_t)c * npix;
    ra.gate = gate;
    P->launch_rng(ra, s, RING_SYNTH);
  }
}

void Pol::analysis(cudaStream_t s, const double *map, double2 *alm, const Ctl *gate) const {
  double4_32a *ft[3] = {P->d_FT, d_FTQ, d_FTU};
  for (int c = 0; c < 3; ++c) {
    RingArgs ra = P->ring_args();
    ra.lsht = lmax;
    ra.FT = ft[c];
    ra.map_in = map + (size_t)c * npix;
    ra.gate = gate;
    P->launch_rng(ra, s, RING_ANALYSIS);
  }
  LegArgs la = P->leg_args();
  la.lsht = lmax;
  la.alm = alm;
  la.gate = gate;
  P->launch_leg(la, s, LEG_ANALYSIS);                                 // T
  if (df) {
    raise_smem_cap(reinterpret_cast<const void *>(spin2_analysis_df_kernel));
    spin2_analysis_df_kernel<<<lmax + 1, kPolThreads, sizeof(float4) * 4 * RP, s>>>(
        gate, reinterpret_cast<const float4 *>(d_tab), P->d_ls, d_FTQ, d_FTU, lmax, RP, alm + nalm, alm + 2 * nalm);
  } else {
    raise_smem_cap(reinterpret_cast<const void *>(spin2_analysis_kernel));
    spin2_analysis_kernel<<<lmax + 1, kPolThreads, sizeof(double4_32a) * 2 * RP, s>>>(
        gate, d_tab, d_FTQ, d_FTU, lmax, RP, alm + nalm, alm + 2 * nalm);
  }
}

void Pol::enqueue_iteration(cudaStream_t s) {
  synth(s, d_s, d_map, d_ctl);
  pol_pixel_kernel<<<kPixBlocks, kPolThreads, 0, s>>>(d_ctl, npix, tau, d_map, d_d, d_w, d_gain, d_gainlam, d_u,
                                                       d_part);
  analysis(s, d_u, d_ta, d_ctl);
  pol_eq4_kernel<<<lmax + 1, 128, 0, s>>>(d_ctl, lmax, nalm, tau, omega, d_cls, d_ta, d_s, d_m_part);
  launch_control(d_ctl, d_part, kPixBlocks, d_m_part, lmax, P->d_cl, d_hist, hist_cap, s);
}

}  // namespace
}  // namespace wfk

using namespace wfk;

#define PO_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

extern "C" {

wf_status wf_pol_create(int nside, int lmax, const double *cls, const double *noise, const uint8_t *mask_t,
                        const uint8_t *mask_p, const wf_options *opt, wf_pol_t *out) {
  if (!out || !cls || !noise) { set_error("wf_pol_create: NULL argument"); return WF_EINVAL; }
  *out = nullptr;
  wf_options o;
  if (opt) o = *opt;
  else wf_options_default(&o);
  if (o.precision == WF_PREC_MIXED) {
    set_error("wf_pol_create: polarisation runs on the FP64 paths (WF_PREC_FP64, WF_PREC_FP64_NATIVE)");
    return WF_EINVAL;
  }
  o.band_limit = 0;
  if (nside < 1 || nside > 2048 || (nside & (nside - 1)) || lmax < 0 || lmax > 4 * nside) {
    set_error("wf_pol_create: nside must be a power of two in [1, 2048] and 0 <= lmax <= 4 nside");
    return WF_EINVAL;
  }
  const long long npix = 12LL * nside * nside;
  const size_t nalm = (size_t)(lmax + 1) * (lmax + 2) / 2;
  const size_t tab_bytes = nalm * (size_t)(2 * nside) * sizeof(double2);
  if (tab_bytes > kSpin2TableMax) {
    set_error("wf_pol_create: the spin-2 table would take " + std::to_string(tab_bytes) + " bytes (limit 64 GiB)");
    return WF_EINVAL;
  }
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l <= lmax; ++l)
      if (!std::isfinite(cls[c * (lmax + 1) + l]) || cls[c * (lmax + 1) + l] < 0.0) {
        set_error("wf_pol_create: C_TT, C_EE, C_BB must be finite and >= 0");
        return WF_EINVAL;
      }
  for (int l = 0; l <= lmax; ++l) {
    const double tt = cls[l], ee = cls[lmax + 1 + l], te = cls[3 * (lmax + 1) + l];
    if (!std::isfinite(te) || te * te > tt * ee * (1.0 + 1e-12)) {
      set_error("wf_pol_create: C_TE must satisfy C_TE^2 <= C_TT C_EE");
      return WF_EINVAL;
    }
  }
  // inverse noise per pixel and the messenger covariance
  std::vector<double4_32a> w(npix);
  double tau = INFINITY;
  long long n_obs = 0;
  for (long long p = 0; p < npix; ++p) {
    const double nt = noise[4 * p], nqq = noise[4 * p + 1], nqu = noise[4 * p + 2], nuu = noise[4 * p + 3];
    double4_32a v = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if (!mask_t || mask_t[p]) {
      if (!std::isfinite(nt) || !(nt > 0.0)) { set_error("wf_pol_create: T noise must be > 0 where observed"); return WF_EINVAL; }
      v.x = 1.0 / nt;
      tau = std::min(tau, nt);
      ++n_obs;
    }
    if (!mask_p || mask_p[p]) {
      const double det = nqq * nuu - nqu * nqu;
      if (!std::isfinite(det) || !(nqq > 0.0) || !(det > 0.0)) {
        set_error("wf_pol_create: the Q-U noise block must be positive definite where observed");
        return WF_EINVAL;
      }
      v.y = nuu / det;
      v.z = -nqu / det;
      v.w = nqq / det;
      tau = std::min(tau, 0.5 * (nqq + nuu) - std::sqrt(0.25 * (nqq - nuu) * (nqq - nuu) + nqu * nqu));
      n_obs += 2;
    }
    w[p] = v;
  }
  if (n_obs == 0) { set_error("wf_pol_create: no observed component"); return WF_EINVAL; }
  Pol *Q = new (std::nothrow) Pol();
  if (!Q) { set_error("out of host memory"); return WF_ENOMEM; }
  Q->opt = o;
  std::vector<double> unit(npix, 1.0);
  wf_plan_t p = nullptr;
  wf_status st = wf_plan_create(nside, lmax, cls, unit.data(), nullptr, &o, &p);   // geometry, tables, T channel
  if (st) { delete Q; return st; }
  Q->P = static_cast<Plan *>(p);
  Q->nside = nside;
  Q->lmax = lmax;
  Q->RP = Q->P->RP;
  Q->npix = npix;
  Q->nalm = (long long)nalm;
  Q->tau = tau;
  Q->omega = Q->P->omega;
  Q->n_obs = n_obs;
  Q->df = o.precision == WF_PREC_FP64;
  const size_t nF = (size_t)(lmax + 1) * Q->RP;
  if ((st = Q->dalloc((void **)&Q->d_tab, tab_bytes)) || (st = Q->dalloc((void **)&Q->d_cls, sizeof(double) * 4 * (lmax + 1))) ||
      (st = Q->dalloc((void **)&Q->d_w, sizeof(double4_32a) * npix)) ||
      (st = Q->dalloc((void **)&Q->d_gain, sizeof(double4_32a) * npix)) ||
      (st = Q->dalloc((void **)&Q->d_gainlam, sizeof(double) * kPixBlocks)) ||
      (st = Q->dalloc((void **)&Q->d_d, sizeof(double) * 3 * npix)) ||
      (st = Q->dalloc((void **)&Q->d_map, sizeof(double) * 3 * npix)) ||
      (st = Q->dalloc((void **)&Q->d_u, sizeof(double) * 3 * npix)) ||
      (st = Q->dalloc((void **)&Q->d_s, sizeof(double2) * 3 * nalm)) ||
      (st = Q->dalloc((void **)&Q->d_ta, sizeof(double2) * 3 * nalm)) ||
      (st = Q->dalloc((void **)&Q->d_FSQ, sizeof(double4_32a) * nF)) || (st = Q->dalloc((void **)&Q->d_FSU, sizeof(double4_32a) * nF)) ||
      (st = Q->dalloc((void **)&Q->d_FTQ, sizeof(double4_32a) * nF)) || (st = Q->dalloc((void **)&Q->d_FTU, sizeof(double4_32a) * nF)) ||
      (st = Q->dalloc((void **)&Q->d_part, sizeof(double) * 2 * kPixBlocks)) ||
      (st = Q->dalloc((void **)&Q->d_m_part, sizeof(double) * 3 * (lmax + 1))) ||
      (st = Q->dalloc((void **)&Q->d_ctl, sizeof(Ctl))) ||
      (st = Q->dalloc((void **)&Q->d_hist, sizeof(wf_iter_record) * (size_t)(o.max_iter + 1)))) {
    delete Q;
    return st;
  }
  Q->hist_cap = o.max_iter + 1;
  cudaStream_t s = Q->stream();
  cudaError_t e = cudaMemcpyAsync(Q->d_cls, cls, sizeof(double) * 4 * (lmax + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Q->d_w, w.data(), sizeof(double4_32a) * npix, cudaMemcpyHostToDevice, s);
  const std::vector<double> no_gains(kPixBlocks, -1.0);   // no gains cached yet: lambda >= 1 never equals -1
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Q->d_gainlam, no_gains.data(), sizeof(double) * kPixBlocks, cudaMemcpyHostToDevice, s);
  // the ring stage never writes the equator pair's south slot: it must read as zero
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->d_FTQ, 0, sizeof(double4_32a) * nF, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->d_FTU, 0, sizeof(double4_32a) * nF, s);
  if (e == cudaSuccess) {
    const long long n = (long long)(lmax + 1) * Q->RP;
    spin2_table_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(Q->P->d_x, Q->P->d_rec, Q->P->d_ls, Q->P->d_sv,
                                                                  lmax, Q->RP, Q->d_tab, Q->df ? 1 : 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMallocHost((void **)&Q->h_ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaEventCreate(&Q->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&Q->ev1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { st = cuda_status(e, "wf_pol_create setup"); delete Q; return st; }
  *out = Q;
  return WF_OK;
}

wf_status wf_pol_destroy(wf_pol_t pol) {
  if (!pol) return WF_OK;
  Pol *Q = static_cast<Pol *>(pol);
  cudaStreamSynchronize(Q->stream());
  delete Q;
  return WF_OK;
}

wf_status wf_pol_alm2map(wf_pol_t pol, const double *alm_dev, double *map_dev) {
  if (!pol || !alm_dev || !map_dev) { set_error("wf_pol_alm2map: NULL argument"); return WF_EINVAL; }
  Pol *Q = static_cast<Pol *>(pol);
  Q->synth(Q->stream(), reinterpret_cast<const double2 *>(alm_dev), map_dev, nullptr);
  PO_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status wf_pol_map2alm(wf_pol_t pol, const double *map_dev, double *alm_dev) {
  if (!pol || !alm_dev || !map_dev) { set_error("wf_pol_map2alm: NULL argument"); return WF_EINVAL; }
  Pol *Q = static_cast<Pol *>(pol);
  Q->analysis(Q->stream(), map_dev, reinterpret_cast<double2 *>(alm_dev), nullptr);
  PO_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status wf_pol_solve(wf_pol_t pol, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                       wf_stats *stats, wf_iter_record *records, int max_records, int *n_records) {
  if (!pol || !d || !alm_out) { set_error("wf_pol_solve: NULL argument"); return WF_EINVAL; }
  Pol *Q = static_cast<Pol *>(pol);
  Plan *P = Q->P;
  cudaStream_t s = Q->stream();
  PO_CUDA(cudaEventRecord(Q->ev0, s));
  PO_CUDA(cudaMemcpyAsync(Q->d_d, d, sizeof(double) * 3 * Q->npix,
                          d_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  PO_CUDA(cudaMemsetAsync(Q->d_s, 0, sizeof(double2) * 3 * Q->nalm, s));
  // lambda from the ratio C_TT / (tau Omega) at l_iter (Sect. 3 names C_TT), clamped to >= 1
  const double lam0 = (Q->opt.cooling && Q->opt.l_iter0 <= Q->lmax)
                          ? std::max(1.0, P->h_cl[Q->opt.l_iter0] / (Q->tau * Q->omega)) : 1.0;
  Ctl c = P->make_ctl(1, lam0, Q->lmax, 0);
  c.band_limit = 0;
  c.tau = Q->tau;
  c.sigma_chi2 = std::sqrt(2.0 * (double)Q->n_obs);
  *Q->h_ctl = c;
  PO_CUDA(cudaMemcpyAsync(Q->d_ctl, Q->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  const int gi = Q->opt.graph_iters;
  if (!Q->graph) {
    cudaGraph_t g;
    PO_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < gi; ++i) Q->enqueue_iteration(s);
    PO_CUDA(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&Q->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate (polarisation)");
  }
  const int max_launch = (Q->opt.max_iter + gi - 1) / gi + 1;
  for (int it = 0; it < max_launch; ++it) {
    PO_CUDA(cudaGraphLaunch(Q->graph, s));
    PO_CUDA(cudaMemcpyAsync(Q->h_ctl, Q->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    PO_CUDA(cudaStreamSynchronize(s));
    if (Q->h_ctl->done) break;
  }
  PO_CUDA(cudaMemcpyAsync(alm_out, Q->d_s, sizeof(double2) * 3 * Q->nalm,
                          alm_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  PO_CUDA(cudaEventRecord(Q->ev1, s));
  const Ctl fin = *Q->h_ctl;
  wf_iter_record last{};
  if (fin.iter > 0)
    PO_CUDA(cudaMemcpyAsync(&last, Q->d_hist + (fin.iter - 1), sizeof(last), cudaMemcpyDeviceToHost, s));
  int nrec = 0;
  if (records && max_records > 0) {
    nrec = fin.iter < max_records ? fin.iter : max_records;
    if (nrec > 0)
      PO_CUDA(cudaMemcpyAsync(records, Q->d_hist, sizeof(wf_iter_record) * nrec, cudaMemcpyDeviceToHost, s));
  }
  PO_CUDA(cudaStreamSynchronize(s));
  if (n_records) *n_records = nrec;
  P->fs_valid = false;
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, Q->ev0, Q->ev1);
    *stats = wf_stats{};
    stats->iters = fin.iter;
    stats->converged = fin.converged;
    stats->levels = fin.level + 1;
    stats->lmax_sht_final = fin.lsht;
    stats->lambda_final = fin.lambda;
    stats->chi2_prior = last.chi2_prior;
    stats->chi2_noise = last.chi2_noise;
    stats->chi2 = last.chi2_prior + last.chi2_noise;
    stats->chi2_per_dof = stats->chi2 / (double)Q->n_obs;
    stats->rel_increment = fin.last_rel;
    stats->ms_device = ms;
    stats->rel_posterior_grad = -1.0;
  }
  if (fin.numeric) { set_error("wf_pol_solve: chi^2 is not finite"); return WF_ENUMERIC; }
  if (!fin.converged) { set_error("wf_pol_solve: max_iter reached before the stop rule"); return WF_ENOTCONVERGED; }
  return WF_OK;
}

}  // extern "C"
