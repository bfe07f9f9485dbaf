// Legendre stage of the HEALPix spherical harmonic transform pair, FP64.
//
// For one m, with x_k = cos(theta) of the north ring of pair k and the
// orthonormal associated Legendre functions lambda_lm (Condon-Shortley phase),
// lambda_lm(-x) = (-1)^(l+m) lambda_lm(x) lets both rings of a pair share one
// recurrence:
//   analysis   a_lm = sum_k lambda_lm(x_k) [T_N(k) + (-1)^(l-m) T_S(k)]
//                   = sum_k lambda_lm(x_k) (E_k if l-m even, O_k if odd),
//              E = T_N + T_S, O = T_N - T_S
//   synthesis  F_N(k) = E'_k + O'_k, F_S(k) = E'_k - O'_k,
//              E'_k = sum_{l-m even} lambda_lm(x_k) s_lm, O'_k = sum_{l-m odd} ...
// lambda_lm is generated on the fly by the three-term recurrence
//   lambda_l = a_l x lambda_{l-1} - b_l lambda_{l-2},
//   a_l = sqrt((4l^2-1)/(l^2-m^2)), b_l = a_l sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
// started at the first l where |lambda_lm(x_k)| >= 2^-100 from a precomputed
// table of (l_start, lambda_{l_start}, lambda_{l_start+1}); smaller terms are
// below double precision of any sum they enter and are not evaluated.
//
// LEG_ITER is one CTA per m doing, in one pass over the ring pairs each:
//   analysis of the increment u (Y^dagger u), the Eq. 4 update
//   s_lm <- f_l (s_lm + (Y^dagger u)_lm), f_l = C_l / (C_l + lambda tau Omega),
//   the chi^2 prior partial sum |s_lm|^2 / C_l of the input state (Sect. 3),
//   the increment and norm partials, and the synthesis of the new s_lm for the
//   next iteration. Nothing but the per-m partials leaves the CTA between the
//   analysis and the synthesis.
#include <cuda_runtime.h>

#include "wf_internal.h"

namespace wfk {

constexpr int kKPT = 2;          // ring pairs held per thread in a pass
constexpr int kNoStart = 1 << 30;  // l_start of a column with no term above 2^-100

__device__ __forceinline__ size_t alm_idx(int lmax, int l, int m) {
  return (size_t)m * (2 * lmax + 1 - m) / 2 + l;
}

// Lane i ends with the sum over the warp's 32 lanes of v[i].
__device__ __forceinline__ double warp_transpose_sum(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < off; ++j) {
      const double send = up ? v[j] : v[j + off];
      const double keep = up ? v[j + off] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// Start values: one thread per (m, k). Scaled recurrence with an explicit
// binary exponent so that sin^m(theta) cannot underflow.
__global__ void start_values_kernel(const double *xk, const double2 *rec, int lmax, int RP, int *ls_out,
                                    double2 *sv_out) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(lmax + 1) * RP) return;
  const int m = (int)(id / RP), k = (int)(id % RP);
  const double x = xk[k];
  const double st = sqrt((1.0 - x) * (1.0 + x));
  int ls = kNoStart;
  double v0 = 0.0, v1 = 0.0;
  if (m == 0 || st > 0.0) {
    // lambda_mm = (-1)^m sqrt((2m+1)/(4 pi) prod_{i<=m} (2i-1)/(2i)) sin^m(theta), as v * 2^e
    double v = 0.28209479177387814347;  // 1 / sqrt(4 pi)
    int e = 0;
    for (int i = 1; i <= m; ++i) {
      v *= -sqrt((2.0 * i + 1.0) / (2.0 * i)) * st;
      if (fabs(v) < 0x1p-400) { v *= 0x1p400; e -= 400; }
    }
    // walk up in l until the true value reaches 2^kStartExp
    double p2 = v;                               // lambda_l (scaled)
    double p1 = x * sqrt(2.0 * m + 3.0) * v;     // lambda_{l+1} (scaled)
    for (int l = m; l <= lmax; ++l) {
      if (p2 != 0.0 && ilogb(p2) + e >= kStartExp) {
        ls = l;
        v0 = ldexp(p2, e);
        v1 = (l + 1 <= lmax) ? ldexp(p1, e) : 0.0;
        break;
      }
      if (l + 2 <= lmax) {
        const double2 ab = rec[alm_idx(lmax, l + 2, m)];
        const double nx = ab.x * x * p1 - ab.y * p2;
        p2 = p1;
        p1 = nx;
        if (fabs(p2) > 0x1p400 || fabs(p1) > 0x1p400) { p1 *= 0x1p-400; p2 *= 0x1p-400; e += 400; }
      } else {
        p2 = p1;
        p1 = 0.0;
      }
    }
  }
  ls_out[id] = ls;
  sv_out[id] = make_double2(v0, v1);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) legendre_kernel(const LegArgs A) {
  extern __shared__ double2 lsm[];
  __shared__ double red[kThreads / 32][32];
  __shared__ double mred[kThreads / 32][3];
  const int m = blockIdx.x;
  const int lmax = A.lmax, RP = A.RP;
  int L = A.lsht;
  double lam = 1.0;
  if (MODE != LEG_ITER && A.gate && A.gate->done) return;
  if (MODE == LEG_ITER) {
    if (A.ctl->done) return;
    L = A.ctl->lsht;
    lam = A.ctl->lambda;
  }
  const size_t base = alm_idx(lmax, m, m);   // index of (l = m, m)
  if (m > L) {
    // column beyond the band limit: the state is zero there (partials of the
    // old state still counted), and so are the synthesis coefficients.
    if (MODE == LEG_ITER || MODE == LEG_ANALYSIS) {
      double c2 = 0.0, inc = 0.0;
      for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        const double2 so = A.alm[base + (l - m)];
        const double wgt = (m == 0) ? 1.0 : 2.0;
        const double a2 = so.x * so.x + so.y * so.y;
        if (MODE == LEG_ITER) {
          if (A.cl[l] > 0.0) c2 += wgt * a2 / A.cl[l];
          inc += wgt * a2;
        }
        A.alm[base + (l - m)] = make_double2(0.0, 0.0);
      }
      if (MODE == LEG_ITER) {
        for (int o = 16; o > 0; o >>= 1) {
          c2 += __shfl_xor_sync(0xffffffffu, c2, o);
          inc += __shfl_xor_sync(0xffffffffu, inc, o);
        }
        if ((threadIdx.x & 31) == 0) { mred[threadIdx.x >> 5][0] = c2; mred[threadIdx.x >> 5][1] = inc; }
        __syncthreads();
        if (threadIdx.x == 0) {
          double a = 0.0, b = 0.0;
          for (int w = 0; w < kThreads / 32; ++w) { a += mred[w][0]; b += mred[w][1]; }
          A.m_part[3 * m] = a;
          A.m_part[3 * m + 1] = b;
          A.m_part[3 * m + 2] = 0.0;
        }
      }
    }
    if (MODE == LEG_ITER || MODE == LEG_SYNTH) {
      for (int k = threadIdx.x; k < RP; k += blockDim.x)
        A.FS[(size_t)m * RP + k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
    return;
  }
  const int Lm = L - m + 1;
  double2 *rc = lsm;            // [Lm + kLB] recurrence coefficients (padded with zeros)
  double2 *tl = lsm + Lm + kLB; // [Lm + kLB] accumulated analysis / state values
  for (int i = threadIdx.x; i < Lm + kLB; i += blockDim.x) {
    rc[i] = (i < Lm) ? A.rec[base + i] : make_double2(0.0, 0.0);
    tl[i] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (MODE == LEG_ANALYSIS || MODE == LEG_ITER) {
    for (int k0 = 0; k0 < RP; k0 += kKPT * kThreads) {
      double x[kKPT], p1[kKPT], p2[kKPT], v0[kKPT], v1[kKPT];
      int ls[kKPT];
      double2 E[kKPT], O[kKPT];
#pragma unroll
      for (int i = 0; i < kKPT; ++i) {
        const int k = k0 + i * kThreads + threadIdx.x;
        p1[i] = p2[i] = 0.0;
        if (k < RP) {
          x[i] = A.x[k];
          const size_t mk = (size_t)m * RP + k;
          ls[i] = A.ls[mk];
          const double2 s2 = A.sv[mk];
          v0[i] = s2.x;
          v1[i] = s2.y;
          const double4_32a t = A.FT[mk];
          E[i] = make_double2(t.x + t.z, t.y + t.w);
          O[i] = make_double2(t.x - t.z, t.y - t.w);
        } else {
          x[i] = 0.0; ls[i] = kNoStart; v0[i] = v1[i] = 0.0;
          E[i] = O[i] = make_double2(0.0, 0.0);
        }
      }
      for (int l0 = m; l0 <= L; l0 += kLB) {
        double acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.0;
#pragma unroll
        for (int j = 0; j < kLB; ++j) {
          const int l = l0 + j;
          const double2 ab = rc[l - m];
#pragma unroll
          for (int i = 0; i < kKPT; ++i) {
            double lv = fma(ab.x * x[i], p1[i], -ab.y * p2[i]);
            lv = (l == ls[i]) ? v0[i] : lv;
            lv = (l == ls[i] + 1) ? v1[i] : lv;
            p2[i] = p1[i];
            p1[i] = lv;
            const double2 X = (j & 1) ? O[i] : E[i];
            acc[2 * j] = fma(lv, X.x, acc[2 * j]);
            acc[2 * j + 1] = fma(lv, X.y, acc[2 * j + 1]);
          }
        }
        const double v = warp_transpose_sum(acc);
        red[warp][lane] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
          double s = 0.0;
#pragma unroll
          for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
          double *t = reinterpret_cast<double *>(&tl[l0 - m + (threadIdx.x >> 1)]);
          t[threadIdx.x & 1] += s;
        }
        __syncthreads();
      }
    }
  }

  if (MODE == LEG_ANALYSIS) {
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x)
      A.alm[base + (l - m)] = (l <= L) ? tl[l - m] : make_double2(0.0, 0.0);
    return;
  }

  if (MODE == LEG_ITER) {
    // Eq. 4 per mode, chi^2 prior of the input state, increment and norm
    double c2 = 0.0, inc = 0.0, nrm = 0.0;
    const double wgt = (m == 0) ? 1.0 : 2.0;
    const double lto = lam * A.tau * A.omega;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const double2 so = A.alm[base + (l - m)];
      const double c = A.cl[l];
      double2 sn = make_double2(0.0, 0.0);
      if (l <= L && c > 0.0) {
        const double f = c / (c + lto);
        const double2 t = tl[l - m];
        sn = make_double2(f * (so.x + t.x), f * (so.y + t.y));
      }
      if (c > 0.0) c2 += wgt * (so.x * so.x + so.y * so.y) / c;
      const double dx = sn.x - so.x, dy = sn.y - so.y;
      inc += wgt * (dx * dx + dy * dy);
      nrm += wgt * (sn.x * sn.x + sn.y * sn.y);
      A.alm[base + (l - m)] = sn;
      if (l <= L) tl[l - m] = sn;
    }
    for (int o = 16; o > 0; o >>= 1) {
      c2 += __shfl_xor_sync(0xffffffffu, c2, o);
      inc += __shfl_xor_sync(0xffffffffu, inc, o);
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    if (lane == 0) { mred[warp][0] = c2; mred[warp][1] = inc; mred[warp][2] = nrm; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) { a += mred[w][0]; b += mred[w][1]; c += mred[w][2]; }
      A.m_part[3 * m] = a;
      A.m_part[3 * m + 1] = b;
      A.m_part[3 * m + 2] = c;
    }
  } else {  // LEG_SYNTH
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) tl[l - m] = A.alm_in[base + (l - m)];
    __syncthreads();
  }

  // ---- synthesis of tl (l = m .. L) onto every ring pair
  for (int k = threadIdx.x; k < RP; k += blockDim.x) {
    const double x = A.x[k];
    const size_t mk = (size_t)m * RP + k;
    const int ls = A.ls[mk];
    const double2 s2 = A.sv[mk];
    double p1 = 0.0, p2 = 0.0;
    double2 E = make_double2(0.0, 0.0), O = make_double2(0.0, 0.0);
    int l = (ls < m) ? m : ls;
    if (l <= L) {
      // the first two values come from the table, then the recurrence
      p2 = s2.x;
      const double2 a0 = tl[l - m];
      if (((l - m) & 1) == 0) { E.x = fma(p2, a0.x, E.x); E.y = fma(p2, a0.y, E.y); }
      else { O.x = fma(p2, a0.x, O.x); O.y = fma(p2, a0.y, O.y); }
      if (l + 1 <= L) {
        p1 = s2.y;
        const double2 a1 = tl[l + 1 - m];
        if (((l + 1 - m) & 1) == 0) { E.x = fma(p1, a1.x, E.x); E.y = fma(p1, a1.y, E.y); }
        else { O.x = fma(p1, a1.x, O.x); O.y = fma(p1, a1.y, O.y); }
      }
      l += 2;
      // keep E/O assignment static: step in pairs aligned to the parity of l - m
      if (((l - m) & 1) == 1 && l <= L) {
        const double2 ab = rc[l - m];
        const double lv = fma(ab.x * x, p1, -ab.y * p2);
        p2 = p1; p1 = lv;
        const double2 a = tl[l - m];
        O.x = fma(lv, a.x, O.x); O.y = fma(lv, a.y, O.y);
        ++l;
      }
      for (; l + 1 <= L; l += 2) {
        const double2 ab0 = rc[l - m], ab1 = rc[l + 1 - m];
        const double le = fma(ab0.x * x, p1, -ab0.y * p2);
        const double lo = fma(ab1.x * x, le, -ab1.y * p1);
        p2 = le; p1 = lo;
        const double2 ae = tl[l - m], ao = tl[l + 1 - m];
        E.x = fma(le, ae.x, E.x); E.y = fma(le, ae.y, E.y);
        O.x = fma(lo, ao.x, O.x); O.y = fma(lo, ao.y, O.y);
      }
      if (l <= L) {
        const double2 ab = rc[l - m];
        const double le = fma(ab.x * x, p1, -ab.y * p2);
        const double2 ae = tl[l - m];
        E.x = fma(le, ae.x, E.x); E.y = fma(le, ae.y, E.y);
      }
    }
    A.FS[mk] = make_double4_32a(E.x + O.x, E.y + O.y, E.x - O.x, E.y - O.y);
  }
}

static size_t leg_smem(int lmax) { return (size_t)2 * (lmax + 1 + kLB) * sizeof(double2); }

void launch_legendre(const LegArgs &a, cudaStream_t s, int mode) {
  const size_t sm = leg_smem(a.lmax);
  const int grid = a.lmax + 1;
  switch (mode) {
    case LEG_SYNTH:
      raise_smem_cap(reinterpret_cast<const void *>(legendre_kernel<LEG_SYNTH>));
      legendre_kernel<LEG_SYNTH><<<grid, kThreads, sm, s>>>(a);
      break;
    case LEG_ANALYSIS:
      raise_smem_cap(reinterpret_cast<const void *>(legendre_kernel<LEG_ANALYSIS>));
      legendre_kernel<LEG_ANALYSIS><<<grid, kThreads, sm, s>>>(a);
      break;
    default:
      raise_smem_cap(reinterpret_cast<const void *>(legendre_kernel<LEG_ITER>));
      legendre_kernel<LEG_ITER><<<grid, kThreads, sm, s>>>(a);
      break;
  }
}

void launch_start_values(const double *x, const double2 *rec, int lmax, int RP, int *ls, double2 *sv,
                         cudaStream_t s) {
  const long long n = (long long)(lmax + 1) * RP;
  const int blocks = (int)((n + 255) / 256);
  start_values_kernel<<<blocks, 256, 0, s>>>(x, rec, lmax, RP, ls, sv);
}

}  // namespace wfk
