// Legendre stage in double-float arithmetic: FP64-accurate results from the
// FP32 pipe.
//
// GB300 runs FP64 FMAs at 1/63 of the FP32 rate, and the FP64 Legendre kernel
// (legendre.cu) is bound by that pipe. Here every value of the inner loops is
// an unevaluated sum of two floats (hi + lo, 48 significant bits) and every
// operation is built from error-free transformations:
//   two_prod(a, b)  p = a b, e = fma(a, b, -p)           (exact)
//   two_sum(a, b)   s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a  (exact)
// Sums over rings and over l use the compensated dot product of Ogita, Rump
// and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005):
// the running sum in a float S with its exact rounding errors collected in a
// float C, which is as accurate as a dot product in twice the working
// precision.
//
// The recurrence is rescaled so that it needs one double-float product and one
// double-float subtraction per step: with lambda_l = g_l mu_l, g_m = g_{m+1} = 1,
// g_l = b_l g_{l-2},
//     mu_l = A_l x mu_{l-1} - mu_{l-2},   A_l = a_l g_{l-1} / g_l,
// (g_l stays within [2^-2.6, 2^0.2] for lmax <= 4096, so mu has lambda's range).
// The factor g_l is applied in double after the cross-ring reduction (analysis)
// and folded into the harmonic coefficients before synthesis.
//
// Terms with |lambda_lm(x)| < 2^-60 (the evanescent region near the poles) are
// not evaluated; they lie below the 48-bit precision of any sum they enter.
//
// Table form (TAB): where the plan holds lambda_lm(x_k) precomputed (FP64
// recurrence, stored as double-float), both passes read it instead of running
// the recurrence, which turns the stage from FP32-issue-bound into HBM-bound:
// 8 bytes per (l, m, ring pair) term and pass against 19 FP32 instructions of
// the recurrence step. Layout: per m, rows of two consecutive l (l - m = 2r and
// 2r + 1, the even and odd parity parts), each row RP float4 (lambda_{m+2r}
// hi, lo, lambda_{m+2r+1} hi, lo) over the ring pairs, stored in tiles of 32
// ring pairs: [m][tile of 32 ring pairs][row][32]. Entries below the 2^-60 cut
// (and the columns past RP of a partial tile) are zero. The analysis gives each
// warp groups of 4 rows, streamed over all tiles, so that a lane sums over ring
// pairs with 4 compensated accumulators and the lanes of a row combine once per
// row group (no block-wide reduction per block of l); the synthesis gives each
// warp tiles (lane = ring pair) walked along the rows. Both keep the next loads
// in flight in registers while they compute on the current ones.
#include <cuda_runtime.h>

#include "df.cuh"
#include "wf_internal.h"

namespace wfk {

constexpr int kNoStartD = 1 << 30;
constexpr int kAnaChunk = 1024;   // ring pairs whose analysis state is held in shared memory at once
constexpr int kTabTiles = kAnaChunk / 32;  // table form: tiles of 32 ring pairs per analysis chunk
constexpr int kSynRows = 4;       // table form: rows per synthesis load batch (two batches in flight)
constexpr int kTabBlocks = 3;     // table form: CTAs per SM the register budget is set for
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ size_t alm_idx_d(int lmax, int l, int m) {
  return (size_t)m * (2 * lmax + 1 - m) / 2 + l;
}

// Lane q ends with the double-float sum over the warp's lanes of (S[q], C[q]).
__device__ __forceinline__ double warp_transpose_sum_df(float (&S)[32], float (&C)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < off; ++j) {
      const float sS = up ? S[j] : S[j + off], sC = up ? C[j] : C[j + off];
      const float kS = up ? S[j + off] : S[j], kC = up ? C[j + off] : C[j];
      const float rS = __shfl_xor_sync(0xffffffffu, sS, off);
      const float rC = __shfl_xor_sync(0xffffffffu, sC, off);
      const float s = kS + rS;
      const float bb = s - kS;
      const float e = (kS - (s - bb)) + (rS - bb);
      S[j] = s;
      C[j] = kC + rC + e;
    }
  }
  return (double)S[0] + (double)C[0];
}

// 16 recurrence steps of one ring pair from l0, accumulating mu * (E or O)
// into the 32 compensated sums; INJECT places the table start values.
template <bool INJECT>
__device__ __forceinline__ void analysis_block(int l0, int m, const float2 *sA, dfl x, dfl &p1, dfl &p2, int ls,
                                               dfl v0, dfl v1, dfl Er, dfl Ei, dfl Or, dfl Oi, float (&S)[32],
                                               float (&C)[32]) {
#pragma unroll
  for (int j = 0; j < kLB; ++j) {
    const int l = l0 + j;
    const float2 a2 = sA[l - m];
    dfl mu = df_step(dfl{a2.x, a2.y}, x, p1, p2);
    if (INJECT) {
      if (l == ls) mu = v0;
      if (l == ls + 1) mu = v1;
    }
    p2 = p1;
    p1 = mu;
    dot2_acc(S[2 * j], C[2 * j], mu, (j & 1) ? Or : Er);
    dot2_acc(S[2 * j + 1], C[2 * j + 1], mu, (j & 1) ? Oi : Ei);
  }
}

// Start values for the double-float recurrence: first l with |lambda| >= 2^-60,
// and mu at that l and the next (mu = lambda / g), one thread per (m, k).
__global__ void start_values_df_kernel(const double *xk, const double2 *rec, const double *g, int lmax, int RP,
                                       int *ls_out, float4 *sv_out) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(lmax + 1) * RP) return;
  const int m = (int)(id / RP), k = (int)(id % RP);
  const double x = xk[k];
  const double st = sqrt((1.0 - x) * (1.0 + x));
  int ls = kNoStartD;
  double v0 = 0.0, v1 = 0.0;
  if (m == 0 || st > 0.0) {
    double v = 0.28209479177387814347;  // 1 / sqrt(4 pi)
    int e = 0;
    for (int i = 1; i <= m; ++i) {
      v *= -sqrt((2.0 * i + 1.0) / (2.0 * i)) * st;
      if (fabs(v) < 0x1p-400) { v *= 0x1p400; e -= 400; }
    }
    double p2 = v, p1 = x * sqrt(2.0 * m + 3.0) * v;
    for (int l = m; l <= lmax; ++l) {
      if (p2 != 0.0 && ilogb(p2) + e >= -60) {
        ls = l;
        v0 = ldexp(p2, e);
        v1 = (l + 1 <= lmax) ? ldexp(p1, e) : 0.0;
        break;
      }
      if (l + 2 <= lmax) {
        const double2 ab = rec[alm_idx_d(lmax, l + 2, m)];
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
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ls != kNoStartD) {
    const size_t base = alm_idx_d(lmax, m, m);
    const dfl a = df_from(v0 / g[base + (ls - m)]);
    const dfl b = (ls + 1 <= lmax) ? df_from(v1 / g[base + (ls + 1 - m)]) : dfl{0.f, 0.f};
    out = make_float4(a.h, a.l, b.h, b.l);
  }
  ls_out[id] = ls;
  sv_out[id] = out;
}

// g_l and A_l of the rescaled recurrence, one CTA per m (serial in l).
__global__ void rescale_coeffs_kernel(const double2 *rec, int lmax, double *g, float2 *A) {
  const int m = blockIdx.x;
  if (threadIdx.x != 0) return;
  const size_t base = alm_idx_d(lmax, m, m);
  double g2 = 1.0, g1 = 1.0;  // g_{l-2}, g_{l-1}
  for (int l = m; l <= lmax; ++l) {
    const double2 ab = rec[base + (l - m)];
    double gl, Al;
    if (l <= m + 1) {
      gl = 1.0;
      Al = ab.x;  // a_{m+1} (a_m = 0)
    } else {
      gl = ab.y * g2;
      Al = ab.x * g1 / gl;
    }
    g[base + (l - m)] = gl;
    const dfl d = df_from(Al);
    A[base + (l - m)] = make_float2(d.h, d.l);
    g2 = g1;
    g1 = gl;
  }
}

// The table: one thread per (m, k) runs the FP64 recurrence from the start
// values of the FP64 kernel and stores lambda as (hi, lo) from the first l of
// the 2^-60 cut on, zeros below it.
__global__ void lam_table_kernel(const double *xk, const double2 *rec, const int *ls64, const double2 *sv64,
                                 const int *ls_df, const long long *poff, int lmax, int RP, float4 *tab) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(lmax + 1) * RP) return;
  const int m = (int)(id / RP), k = (int)(id % RP);
  const int npr = (lmax - m + 2) / 2;
  float4 *col = tab + ((size_t)poff[m] * ((RP + 31) >> 5) + (size_t)(k >> 5) * npr) * 32 + (k & 31);
  const int l64 = ls64[id], ldf = ls_df[id];
  const double x = xk[k];
  const size_t base = alm_idx_d(lmax, m, m);
  double p2 = 0.0, p1 = 0.0;  // lambda_{l-2}, lambda_{l-1}
  dfl ev{0.f, 0.f};           // the row's even part
  for (int l = m; l < m + 2 * npr; ++l) {
    double lam = 0.0;
    if (l <= lmax && l >= l64) {
      if (l == l64) lam = sv64[id].x;
      else if (l == l64 + 1) lam = sv64[id].y;
      else {
        const double2 ab = rec[base + (l - m)];
        lam = ab.x * x * p1 - ab.y * p2;
      }
      p2 = p1;
      p1 = lam;
    }
    const dfl d = (l >= ldf && l <= lmax) ? df_from(lam) : dfl{0.f, 0.f};
    if (((l - m) & 1) == 0) ev = d;
    else col[(size_t)((l - m) >> 1) * 32] = make_float4(ev.h, ev.l, d.h, d.l);
  }
}

// (S, C) += the (S, C) of the lane `off` away (xor), error-free in S: the
// compensated sum of two lanes' partial sums
__device__ __forceinline__ void df_xor_sum(float &S, float &C, int off) {
  const float rS = __shfl_xor_sync(0xffffffffu, S, off), rC = __shfl_xor_sync(0xffffffffu, C, off);
  const float s = S + rS;
  const float bb = s - S;
  const float e = (S - (s - bb)) + (rS - bb);
  S = s;
  C = C + rC + e;
}

template <int MODE, bool TAB>
__global__ void __launch_bounds__(kThreads, TAB ? kTabBlocks : 2) legendre_df_kernel(const LegArgs A, const LegDfArgs D) {
  extern __shared__ double2 dsm[];
  __shared__ double red[kThreads / 32][32];
  __shared__ double mred[kThreads / 32][3];
  __shared__ int tab_tmin[kTabTiles];  // table form: first evaluated l of each tile of the chunk
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
  const size_t base = alm_idx_d(lmax, m, m);
  if (m > L) {
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
  const int Lp = Lm + kLB;
  // shared: tl [Lp] double2 | sA [Lp] float2 | ss [Lp] float4 (synthesis coefficients g_l s_lm);
  // table form: tl | ss (no sA)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2 *tl = dsm;
  float2 *sA = reinterpret_cast<float2 *>(dsm + Lp);
  float4 *ss = TAB ? reinterpret_cast<float4 *>(dsm + Lp) : reinterpret_cast<float4 *>(sA + Lp + (Lp & 1));
  for (int i = threadIdx.x; i < Lp; i += blockDim.x) {
    if (!TAB) sA[i] = (i < Lm) ? D.A[base + i] : make_float2(0.f, 0.f);
    tl[i] = make_double2(0.0, 0.0);
  }
  const int npr = (lmax - m + 2) >> 1;  // table form: rows of m
  const int rlast = (L - m) >> 1;       // table form: last row needed
  const float4 *tm = TAB ? D.tab + (size_t)D.poff[m] * ((RP + 31) >> 5) * 32 : nullptr;
  __syncthreads();

  if (MODE == LEG_ANALYSIS || MODE == LEG_ITER) {
    // per ring pair state in shared memory: the thread's sums then cover all of
    // its ring pairs of a chunk before one reduction per block of kLB values of
    // l; chunks of kAnaChunk ring pairs run one after another (one chunk up to
    // Nside 512), each adding its share to t_l
    if (TAB) {
      // lane (rho, sigma) = (lane / 8, lane % 8) sums row 4 rg + rho of the warp's row group
      // over the columns sigma + 8 j of every tile
      const int rho = lane >> 3, sig = lane & 7;
      for (int k0 = 0; k0 < RP; k0 += kAnaChunk) {
        const int nk = min(kAnaChunk, RP - k0);
        const int ntile = (nk + 31) >> 5;
        float4 *stE = ss, *stO = ss + nk;
        for (int kk = threadIdx.x; kk < nk; kk += blockDim.x) {
          const double4_32a t = A.FT[(size_t)m * RP + k0 + kk];
          const dfl er = df_from(t.x + t.z), ei = df_from(t.y + t.w);
          const dfl orr = df_from(t.x - t.z), oi = df_from(t.y - t.w);
          stE[kk] = make_float4(er.h, er.l, ei.h, ei.l);
          stO[kk] = make_float4(orr.h, orr.l, oi.h, oi.l);
        }
        for (int t = warp; t < ntile; t += kWarps) {
          const int kk = 32 * t + lane;
          const int mn = __reduce_min_sync(0xffffffffu, kk < nk ? D.ls[(size_t)m * RP + k0 + kk] : kNoStartD);
          if (lane == 0) tab_tmin[t] = mn;
        }
        __syncthreads();
        const float4 *tc0 = tm + (size_t)(k0 >> 5) * npr * 32;  // the chunk's first tile
        for (int rg = warp; 4 * rg <= rlast; rg += kWarps) {
          const int r = 4 * rg + rho;
          const int lhi = m + 8 * rg + 7;  // last l of the row group
          auto next_tile = [&](int t) {    // the next tile holding a term of the row group
            while (t < ntile && tab_tmin[t] > lhi) ++t;
            return t;
          };
          auto load = [&](int t, float4 (&v)[4]) {
            const float4 *src = tc0 + ((size_t)t * npr + r) * 32 + sig;
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = (r <= rlast) ? __ldcs(src + 8 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
          };
          float aS[4] = {0.f, 0.f, 0.f, 0.f}, aC[4] = {0.f, 0.f, 0.f, 0.f};
          float4 cur[4], nxt[4];
          int t = next_tile(0);
          if (t < ntile) load(t, cur);
          while (t < ntile) {
            const int tn = next_tile(t + 1);
            if (tn < ntile) load(tn, nxt);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int kk = 32 * t + sig + 8 * j;
              if (kk < nk) {
                const float4 e4 = stE[kk], o4 = stO[kk];
                const dfl le{cur[j].x, cur[j].y}, lo{cur[j].z, cur[j].w};
                dot2_acc(aS[0], aC[0], le, dfl{e4.x, e4.y});
                dot2_acc(aS[1], aC[1], le, dfl{e4.z, e4.w});
                dot2_acc(aS[2], aC[2], lo, dfl{o4.x, o4.y});
                dot2_acc(aS[3], aC[3], lo, dfl{o4.z, o4.w});
              }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) cur[j] = nxt[j];
            t = tn;
          }
#pragma unroll
          for (int off = 1; off < 8; off <<= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) df_xor_sum(aS[q], aC[q], off);
          if (sig == 0 && r <= rlast) {  // l = m + 2 r (even part) and m + 2 r + 1 (odd part)
            tl[2 * r].x += (double)aS[0] + (double)aC[0];
            tl[2 * r].y += (double)aS[1] + (double)aC[1];
            tl[2 * r + 1].x += (double)aS[2] + (double)aC[2];
            tl[2 * r + 1].y += (double)aS[3] + (double)aC[3];
          }
        }
        __syncthreads();
      }
    } else
    for (int k0 = 0; k0 < RP; k0 += kAnaChunk) {
      const int nk = min(kAnaChunk, RP - k0);
      float4 *stE = ss;                            // (Er, Ei) as hi/lo
      float4 *stO = stE + nk;                      // (Or, Oi)
      float4 *stP = stO + nk;                      // (p1, p2)
      float2 *stX = reinterpret_cast<float2 *>(stP + nk);  // x as double-float
      for (int kk = threadIdx.x; kk < nk; kk += blockDim.x) {
        const int k = k0 + kk;
        const double4_32a t = A.FT[(size_t)m * RP + k];
        const dfl er = df_from(t.x + t.z), ei = df_from(t.y + t.w);
        const dfl orr = df_from(t.x - t.z), oi = df_from(t.y - t.w);
        stE[kk] = make_float4(er.h, er.l, ei.h, ei.l);
        stO[kk] = make_float4(orr.h, orr.l, oi.h, oi.l);
        stP[kk] = make_float4(0.f, 0.f, 0.f, 0.f);
        const dfl xk = df_from(A.x[k]);
        stX[kk] = make_float2(xk.h, xk.l);
      }
      __syncthreads();
      for (int l0 = m; l0 <= L; l0 += kLB) {
        float S[32], C[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) { S[j] = 0.f; C[j] = 0.f; }
        for (int kk = threadIdx.x; kk < nk; kk += blockDim.x) {
          const size_t mk = (size_t)m * RP + k0 + kk;
          const int ls = D.ls[mk];
          if (ls >= l0 + kLB) continue;            // no evaluated term yet in this block
          const float2 x2 = stX[kk];
          const dfl x = dfl{x2.x, x2.y};
          const float4 e4 = stE[kk], o4 = stO[kk], q4 = stP[kk];
          dfl p1 = dfl{q4.x, q4.y}, p2 = dfl{q4.z, q4.w};
          if (ls + 1 >= l0) {                      // a start value falls in this block
            const float4 s4 = D.sv[mk];
            analysis_block<true>(l0, m, sA, x, p1, p2, ls, dfl{s4.x, s4.y}, dfl{s4.z, s4.w}, dfl{e4.x, e4.y},
                                 dfl{e4.z, e4.w}, dfl{o4.x, o4.y}, dfl{o4.z, o4.w}, S, C);
          } else {
            analysis_block<false>(l0, m, sA, x, p1, p2, ls, dfl{0.f, 0.f}, dfl{0.f, 0.f}, dfl{e4.x, e4.y},
                                  dfl{e4.z, e4.w}, dfl{o4.x, o4.y}, dfl{o4.z, o4.w}, S, C);
          }
          stP[kk] = make_float4(p1.h, p1.l, p2.h, p2.l);
        }
        const double s = warp_transpose_sum_df(S, C);
        red[warp][lane] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
          double t = 0.0;
#pragma unroll
          for (int w = 0; w < kThreads / 32; ++w) t += red[w][threadIdx.x];
          double *dst = reinterpret_cast<double *>(&tl[l0 - m + (threadIdx.x >> 1)]);
          dst[threadIdx.x & 1] += t;
        }
        __syncthreads();
      }
    }
    // undo the rescaling: lambda = g mu (the table holds lambda itself)
    for (int l = m + threadIdx.x; l <= L && !TAB; l += blockDim.x) {
      const double gl = D.g[base + (l - m)];
      tl[l - m].x *= gl;
      tl[l - m].y *= gl;
    }
    __syncthreads();
  }

  if (MODE == LEG_ANALYSIS) {
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x)
      A.alm[base + (l - m)] = (l <= L) ? tl[l - m] : make_double2(0.0, 0.0);
    return;
  }

  if (MODE == LEG_ITER) {
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
      if (l <= L) {
        const double gl = TAB ? 1.0 : D.g[base + (l - m)];
        const dfl re = df_from(gl * sn.x), im = df_from(gl * sn.y);
        ss[l - m] = make_float4(re.h, re.l, im.h, im.l);
      }
    }
    if (TAB && threadIdx.x < 2) ss[Lm + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
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
    if (TAB && threadIdx.x < 2) ss[Lm + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
      const double gl = TAB ? 1.0 : D.g[base + (l - m)];
      const double2 s = A.alm_in[base + (l - m)];
      const dfl re = df_from(gl * s.x), im = df_from(gl * s.y);
      ss[l - m] = make_float4(re.h, re.l, im.h, im.l);
    }
    __syncthreads();
  }

  // ---- synthesis onto every ring pair (one ring pair per thread at a time)
  if constexpr (TAB) {
    // each warp takes tiles of 32 ring pairs (lane = ring pair) and walks the rows
    // from the first any of them needs; rows below a ring pair's cut hold zeros
    for (int cg = warp; 32 * cg < RP; cg += kWarps) {
      const int k = 32 * cg + lane;
      const int lw = __reduce_min_sync(0xffffffffu, k < RP ? D.ls[(size_t)m * RP + k] : kNoStartD);
      float ERs = 0.f, ERc = 0.f, EIs = 0.f, EIc = 0.f, ORs = 0.f, ORc = 0.f, OIs = 0.f, OIc = 0.f;
      if (lw <= L) {
        const float4 *src = tm + (size_t)cg * npr * 32 + lane;
        auto load = [&](int r, float4 (&v)[kSynRows]) {
#pragma unroll
          for (int i = 0; i < kSynRows; ++i)
            v[i] = (r + i <= rlast) ? __ldcs(src + (size_t)(r + i) * 32) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        float4 cur[kSynRows], nxt[kSynRows];
        int r = (lw - m) >> 1;
        load(r, cur);
        for (; r <= rlast; r += kSynRows) {
          if (r + kSynRows <= rlast) load(r + kSynRows, nxt);
#pragma unroll
          for (int i = 0; i < kSynRows; ++i) {
            if (r + i <= rlast) {
              const float4 ce = ss[2 * (r + i)], co = ss[2 * (r + i) + 1];
              const dfl le{cur[i].x, cur[i].y}, lo{cur[i].z, cur[i].w};
              dot2_acc(ERs, ERc, le, dfl{ce.x, ce.y});
              dot2_acc(EIs, EIc, le, dfl{ce.z, ce.w});
              dot2_acc(ORs, ORc, lo, dfl{co.x, co.y});
              dot2_acc(OIs, OIc, lo, dfl{co.z, co.w});
            }
          }
#pragma unroll
          for (int i = 0; i < kSynRows; ++i) cur[i] = nxt[i];
        }
      }
      if (k < RP) {
        const double er = (double)ERs + (double)ERc, ei = (double)EIs + (double)EIc;
        const double orr = (double)ORs + (double)ORc, oi = (double)OIs + (double)OIc;
        A.FS[(size_t)m * RP + k] = make_double4_32a(er + orr, ei + oi, er - orr, ei - oi);
      }
    }
    return;
  } else {
    for (int k = threadIdx.x; k < RP; k += blockDim.x) {
      const size_t mk = (size_t)m * RP + k;
      const int ls = D.ls[mk];
      float ERs = 0.f, ERc = 0.f, EIs = 0.f, EIc = 0.f, ORs = 0.f, ORc = 0.f, OIs = 0.f, OIc = 0.f;
      if (ls <= L) {
        const dfl x = df_from(A.x[k]);
        const float4 s4 = D.sv[mk];
        dfl p2 = dfl{s4.x, s4.y};
        dfl p1 = dfl{s4.z, s4.w};
        int l = ls;
        {
          const float4 c = ss[l - m];
          if (((l - m) & 1) == 0) { dot2_acc(ERs, ERc, p2, dfl{c.x, c.y}); dot2_acc(EIs, EIc, p2, dfl{c.z, c.w}); }
          else { dot2_acc(ORs, ORc, p2, dfl{c.x, c.y}); dot2_acc(OIs, OIc, p2, dfl{c.z, c.w}); }
        }
        if (l + 1 <= L) {
          const float4 c = ss[l + 1 - m];
          if (((l + 1 - m) & 1) == 0) { dot2_acc(ERs, ERc, p1, dfl{c.x, c.y}); dot2_acc(EIs, EIc, p1, dfl{c.z, c.w}); }
          else { dot2_acc(ORs, ORc, p1, dfl{c.x, c.y}); dot2_acc(OIs, OIc, p1, dfl{c.z, c.w}); }
        }
        l += 2;
        if (((l - m) & 1) == 1 && l <= L) {
          const float2 a2 = sA[l - m];
          const dfl mu = df_step(dfl{a2.x, a2.y}, x, p1, p2);
          p2 = p1; p1 = mu;
          const float4 c = ss[l - m];
          dot2_acc(ORs, ORc, mu, dfl{c.x, c.y});
          dot2_acc(OIs, OIc, mu, dfl{c.z, c.w});
          ++l;
        }
        for (; l + 1 <= L; l += 2) {
          const float2 a0 = sA[l - m], a1 = sA[l + 1 - m];
          const dfl me = df_step(dfl{a0.x, a0.y}, x, p1, p2);
          const dfl mo = df_step(dfl{a1.x, a1.y}, x, me, p1);
          p2 = me; p1 = mo;
          const float4 ce = ss[l - m], co = ss[l + 1 - m];
          dot2_acc(ERs, ERc, me, dfl{ce.x, ce.y});
          dot2_acc(EIs, EIc, me, dfl{ce.z, ce.w});
          dot2_acc(ORs, ORc, mo, dfl{co.x, co.y});
          dot2_acc(OIs, OIc, mo, dfl{co.z, co.w});
        }
        if (l <= L) {
          const float2 a0 = sA[l - m];
          const dfl me = df_step(dfl{a0.x, a0.y}, x, p1, p2);
          const float4 ce = ss[l - m];
          dot2_acc(ERs, ERc, me, dfl{ce.x, ce.y});
          dot2_acc(EIs, EIc, me, dfl{ce.z, ce.w});
        }
      }
      const double er = (double)ERs + (double)ERc, ei = (double)EIs + (double)EIc;
      const double orr = (double)ORs + (double)ORc, oi = (double)OIs + (double)OIc;
      A.FS[mk] = make_double4_32a(er + orr, ei + oi, er - orr, ei - oi);
    }
  }
}

// tl [Lp] double2 | sA [Lp (+1)] float2 | max(Lp, 3.5 chunk) float4 (synthesis
// coefficients, or the per-ring-pair analysis state of one chunk)
static size_t leg_df_smem(int lmax, int RP) {
  const size_t Lp = (size_t)lmax + 1 + kLB;
  const size_t nk = RP < kAnaChunk ? (size_t)RP : (size_t)kAnaChunk;
  const size_t st = 3 * nk + (nk + 1) / 2;
  const size_t q = Lp > st ? Lp : st;
  return Lp * sizeof(double2) + (Lp + 1) * sizeof(float2) + q * sizeof(float4) + 16;
}

// table form: tl [Lp] double2 | max(Lp, 2 chunk) float4
size_t leg_tab_smem(int lmax, int RP) {
  const size_t Lp = (size_t)lmax + 1 + kLB;
  const size_t nk = RP < kAnaChunk ? (size_t)RP : (size_t)kAnaChunk;
  const size_t q = Lp > 2 * nk ? Lp : 2 * nk;
  return Lp * sizeof(double2) + q * sizeof(float4);
}

template <bool TAB>
static void launch_leg_df(const LegArgs &a, const LegDfArgs &d, cudaStream_t s, int mode, size_t sm, int grid) {
  switch (mode) {
    case LEG_SYNTH:
      raise_smem_cap(reinterpret_cast<const void *>(legendre_df_kernel<LEG_SYNTH, TAB>));
      legendre_df_kernel<LEG_SYNTH, TAB><<<grid, kThreads, sm, s>>>(a, d);
      break;
    case LEG_ANALYSIS:
      raise_smem_cap(reinterpret_cast<const void *>(legendre_df_kernel<LEG_ANALYSIS, TAB>));
      legendre_df_kernel<LEG_ANALYSIS, TAB><<<grid, kThreads, sm, s>>>(a, d);
      break;
    default:
      raise_smem_cap(reinterpret_cast<const void *>(legendre_df_kernel<LEG_ITER, TAB>));
      legendre_df_kernel<LEG_ITER, TAB><<<grid, kThreads, sm, s>>>(a, d);
      break;
  }
}

void launch_legendre_df(const LegArgs &a, const LegDfArgs &d, cudaStream_t s, int mode) {
  const int grid = a.lmax + 1;
  if (d.tab) launch_leg_df<true>(a, d, s, mode, leg_tab_smem(a.lmax, a.RP), grid);
  else launch_leg_df<false>(a, d, s, mode, leg_df_smem(a.lmax, a.RP), grid);
}

size_t lam_table_rows(int lmax) {
  size_t rows = 0;
  for (int m = 0; m <= lmax; ++m) rows += (size_t)(lmax - m + 2) / 2;
  return rows;
}

void launch_lam_table(const double *x, const double2 *rec, const int *ls64, const double2 *sv64, const int *ls_df,
                      const long long *poff, int lmax, int RP, float4 *tab, cudaStream_t s) {
  const long long n = (long long)(lmax + 1) * RP;
  lam_table_kernel<<<(int)((n + 127) / 128), 128, 0, s>>>(x, rec, ls64, sv64, ls_df, poff, lmax, RP, tab);
}

void launch_df_tables(const double *x, const double2 *rec, int lmax, int RP, double *g, float2 *A, int *ls,
                      float4 *sv, cudaStream_t s) {
  rescale_coeffs_kernel<<<lmax + 1, 32, 0, s>>>(rec, lmax, g, A);
  const long long n = (long long)(lmax + 1) * RP;
  start_values_df_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(x, rec, g, lmax, RP, ls, sv);
}

}  // namespace wfk
