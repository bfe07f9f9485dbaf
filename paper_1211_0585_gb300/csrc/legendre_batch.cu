// Legendre stage of one messenger iteration for NB right-hand sides at once,
// double-float, table form (the FP64 path's batched solves).
//
// The single-map table kernel (legendre_df.cu) reads the lambda table twice per
// iteration and issues instructions about half of its time. Here one CTA per m
// reads each table row once for NB maps that share the shape (their own data,
// state, C_l, lambda and band limit): the analysis lanes apply one table value
// to NB maps' Fourier sums, the synthesis lanes to NB maps' coefficients, so
// the table traffic per map falls by NB; the compensated products (13 FP32
// instructions each) then bound it. Measured on whole solves at Nside 512:
// 2.15 solves/s in pairs against 1.97 one by one; groups of four were no
// faster per map than single solves (one CTA per SM by registers and shared
// memory), so groups are of two.
// The arithmetic per map is exactly the single kernel's: the same compensated
// dot products in the same order (lane (rho, sigma) sums row 4 g + rho over
// columns sigma + 8 j of every tile, the 8 sigma lanes combine by xor steps;
// synthesis lanes are ring pairs walking the rows upwards), the same Eq. 4 and
// partial sums, so a batched map's iterates equal its single solve's bit for
// bit (the analysis takes its ring pairs in chunks of kBatchChunk, as the
// single kernel does).
// MODE LEG_SYNTH and LEG_ANALYSIS are the single kernel's transforms for NB
// maps (several messenger fields: one synthesis and one analysis per map and
// iteration, the maps' Eq. 4 joint): the synthesis reads each map's
// coefficients from Bm.alm, the analysis writes each map's t_l there.
#include <cuda_runtime.h>

#include "df.cuh"
#include "wf_internal.h"

namespace wfk {
namespace {

constexpr int kBatchChunkMax = 1024;
constexpr int kBTiles = kBatchChunkMax / 32;
constexpr int kNoStartB = 1 << 30;

__device__ __forceinline__ size_t aidx_b(int lmax, int l, int m) { return (size_t)m * (2 * lmax + 1 - m) / 2 + l; }

__device__ __forceinline__ void xor_sum_b(float &S, float &C, int off) {
  const float rS = __shfl_xor_sync(0xffffffffu, S, off), rC = __shfl_xor_sync(0xffffffffu, C, off);
  const float s = S + rS;
  const float bb = s - S;
  const float e = (S - (s - bb)) + (rS - bb);
  S = s;
  C = C + rC + e;
}

template <int NB, int kBThreads, int kBatchChunk, int kMinBlocks, int MODE>
__global__ void __launch_bounds__(kBThreads, kMinBlocks) legendre_batch_kernel(const LegArgs A, const LegDfArgs D,
                                                                                const LegBatchMaps Bm) {
  constexpr int kBWarps = kBThreads / 32;
  extern __shared__ double2 bsm[];
  __shared__ int tab_tmin[kBTiles];
  __shared__ double mred[kBWarps][3];
  const int m = blockIdx.x;
  const int lmax = A.lmax, RP = A.RP;
  int Lb[NB];
  double lam[NB];
  bool on[NB];
  int Lmax = -1;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    on[b] = b < Bm.n && !Bm.ctl[b]->done;
    Lb[b] = on[b] ? Bm.ctl[b]->lsht : -1;
    lam[b] = on[b] ? Bm.ctl[b]->lambda : 1.0;
    Lmax = max(Lmax, Lb[b]);
  }
  if (Lmax < 0) return;
  const size_t base = aidx_b(lmax, m, m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double wgt = (m == 0) ? 1.0 : 2.0;

  // a map whose band limit is below m: zero its state and F, record its state's partials
  auto outside = [&](int b) {
    double c2 = 0.0, inc = 0.0;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const double2 so = Bm.alm[b][base + (l - m)];
      const double a2 = so.x * so.x + so.y * so.y;
      if (Bm.cl[b][l] > 0.0) c2 += wgt * a2 / Bm.cl[b][l];
      inc += wgt * a2;
      Bm.alm[b][base + (l - m)] = make_double2(0.0, 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) {
      c2 += __shfl_xor_sync(0xffffffffu, c2, o);
      inc += __shfl_xor_sync(0xffffffffu, inc, o);
    }
    if (lane == 0) { mred[warp][0] = c2; mred[warp][1] = inc; }
    for (int k = threadIdx.x; k < RP; k += blockDim.x)
      Bm.FS[b][(size_t)m * RP + k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int w = 0; w < kBWarps; ++w) { a += mred[w][0]; c += mred[w][1]; }
      Bm.m_part[b][3 * m] = a;
      Bm.m_part[b][3 * m + 1] = c;
      Bm.m_part[b][3 * m + 2] = 0.0;
    }
    __syncthreads();
  };
  if (m > Lmax) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!on[b]) continue;
      if (MODE == LEG_ITER) {
        outside(b);
      } else if (MODE == LEG_ANALYSIS) {
        for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) Bm.alm[b][base + (l - m)] = make_double2(0.0, 0.0);
      } else {
        for (int k = threadIdx.x; k < RP; k += blockDim.x)
          Bm.FS[b][(size_t)m * RP + k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      }
    }
    return;
  }
  const int L = Lmax;
  const int Lm = L - m + 1;
  const int Lpm = lmax + 1 + kLB;
  const int nkm = RP < kBatchChunk ? RP : kBatchChunk;
  // shared: tl [NB][Lpm] double2 | region [max(NB Lpm, 2 NB chunk)] float4: the maps' synthesis
  // coefficients, or during the analysis their staged E and O sums
  double2 *tl = bsm;
  float4 *reg = reinterpret_cast<float4 *>(bsm + (size_t)NB * Lpm);
  for (int i = threadIdx.x; i < NB * Lpm; i += blockDim.x) tl[i] = make_double2(0.0, 0.0);
  const int npr = (lmax - m + 2) >> 1;
  const int rlast = (L - m) >> 1;
  const float4 *tm = D.tab + (size_t)D.poff[m] * ((RP + 31) >> 5) * 32;
  __syncthreads();

  // ---- analysis
  if (MODE != LEG_SYNTH) {
    const int rho = lane >> 3, sig = lane & 7;
    for (int k0 = 0; k0 < RP; k0 += kBatchChunk) {
      const int nk = min(kBatchChunk, RP - k0);
      const int ntile = (nk + 31) >> 5;
      for (int i = threadIdx.x; i < NB * nk; i += blockDim.x) {
        const int b = i / nk, kk = i % nk;
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f), o = e;
        if (b < Bm.n && Lb[b] >= m) {
          const double4_32a t = Bm.FT[b][(size_t)m * RP + k0 + kk];
          const dfl er = df_from(t.x + t.z), ei = df_from(t.y + t.w);
          const dfl orr = df_from(t.x - t.z), oi = df_from(t.y - t.w);
          e = make_float4(er.h, er.l, ei.h, ei.l);
          o = make_float4(orr.h, orr.l, oi.h, oi.l);
        }
        reg[(size_t)(2 * b) * nkm + kk] = e;
        reg[(size_t)(2 * b + 1) * nkm + kk] = o;
      }
      for (int t = warp; t < ntile; t += kBWarps) {
        const int kk = 32 * t + lane;
        const int mn = __reduce_min_sync(0xffffffffu, kk < nk ? D.ls[(size_t)m * RP + k0 + kk] : kNoStartB);
        if (lane == 0) tab_tmin[t] = mn;
      }
      __syncthreads();
      const float4 *tc0 = tm + (size_t)(k0 >> 5) * npr * 32;
      for (int rg = warp; 4 * rg <= rlast; rg += kBWarps) {
        const int r = 4 * rg + rho;
        const int lhi = m + 8 * rg + 7;
        auto next_tile = [&](int t) {
          while (t < ntile && tab_tmin[t] > lhi) ++t;
          return t;
        };
        auto load = [&](int t, float4 (&v)[4]) {
          const float4 *src = tc0 + ((size_t)t * npr + r) * 32 + sig;
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] = (r <= rlast) ? __ldcs(src + 8 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        float aS[NB][4], aC[NB][4];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int q = 0; q < 4; ++q) { aS[b][q] = 0.f; aC[b][q] = 0.f; }
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
              const dfl le{cur[j].x, cur[j].y}, lo{cur[j].z, cur[j].w};
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                const float4 e4 = reg[(size_t)(2 * b) * nkm + kk], o4 = reg[(size_t)(2 * b + 1) * nkm + kk];
                dot2_acc(aS[b][0], aC[b][0], le, dfl{e4.x, e4.y});
                dot2_acc(aS[b][1], aC[b][1], le, dfl{e4.z, e4.w});
                dot2_acc(aS[b][2], aC[b][2], lo, dfl{o4.x, o4.y});
                dot2_acc(aS[b][3], aC[b][3], lo, dfl{o4.z, o4.w});
              }
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) cur[j] = nxt[j];
          t = tn;
        }
#pragma unroll
        for (int off = 1; off < 8; off <<= 1)
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) xor_sum_b(aS[b][q], aC[b][q], off);
        if (sig == 0 && r <= rlast) {
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            double2 *tb = tl + (size_t)b * Lpm;
            tb[2 * r].x += (double)aS[b][0] + (double)aC[b][0];
            tb[2 * r].y += (double)aS[b][1] + (double)aC[b][1];
            tb[2 * r + 1].x += (double)aS[b][2] + (double)aC[b][2];
            tb[2 * r + 1].y += (double)aS[b][3] + (double)aC[b][3];
          }
        }
      }
      __syncthreads();
    }
  }

  if (MODE == LEG_ANALYSIS) {   // t_l of every map, zero above its band limit
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!on[b]) continue;
      const double2 *tb = tl + (size_t)b * Lpm;
      for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x)
        Bm.alm[b][base + (l - m)] = (l <= Lb[b]) ? tb[l - m] : make_double2(0.0, 0.0);
    }
    return;
  }

  // ---- Eq. 4, the prior chi^2 / increment / norm partials and the synthesis coefficients, map by map
  // (synthesis alone: the coefficients are the maps' a_lm)
  float4 *ss = reg;   // [NB][Lpm]
  if (MODE == LEG_SYNTH) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      float4 *sb = ss + (size_t)b * Lpm;
      const bool use = on[b] && m <= Lb[b];
      for (int i = threadIdx.x; i < Lm + 2; i += blockDim.x) {
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (use && i < Lm && m + i <= Lb[b]) {
          const double2 v = Bm.alm[b][base + i];
          const dfl re = df_from(v.x), im = df_from(v.y);
          c = make_float4(re.h, re.l, im.h, im.l);
        }
        sb[i] = c;
      }
      if (on[b] && m > Lb[b])
        for (int k = threadIdx.x; k < RP; k += blockDim.x)
          Bm.FS[b][(size_t)m * RP + k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < NB && MODE == LEG_ITER; ++b) {
    float4 *sb = ss + (size_t)b * Lpm;
    if (!on[b] || m > Lb[b]) {
      // the synthesis reads rows up to L: coefficients 0 .. Lm + 1 (Lm + 2 <= Lpm)
      for (int i = threadIdx.x; i < Lm + 2; i += blockDim.x) sb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (on[b]) outside(b);
      continue;
    }
    const int Lbb = Lb[b];
    double c2 = 0.0, inc = 0.0, nrm = 0.0;
    const double lto = lam[b] * Bm.tau[b] * A.omega;
    const double2 *tb = tl + (size_t)b * Lpm;
    double2 *ab = Bm.alm[b];
    const double *clb = Bm.cl[b];
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const double2 so = ab[base + (l - m)];
      const double c = clb[l];
      double2 sn = make_double2(0.0, 0.0);
      if (l <= Lbb && c > 0.0) {
        const double f = c / (c + lto);
        const double2 t = tb[l - m];
        sn = make_double2(f * (so.x + t.x), f * (so.y + t.y));
      }
      if (c > 0.0) c2 += wgt * (so.x * so.x + so.y * so.y) / c;
      const double dx = sn.x - so.x, dy = sn.y - so.y;
      inc += wgt * (dx * dx + dy * dy);
      nrm += wgt * (sn.x * sn.x + sn.y * sn.y);
      ab[base + (l - m)] = sn;
      if (l <= L) {
        const dfl re = df_from(sn.x), im = df_from(sn.y);
        sb[l - m] = make_float4(re.h, re.l, im.h, im.l);
      }
    }
    if (threadIdx.x < 2) sb[Lm + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int o = 16; o > 0; o >>= 1) {
      c2 += __shfl_xor_sync(0xffffffffu, c2, o);
      inc += __shfl_xor_sync(0xffffffffu, inc, o);
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    if (lane == 0) { mred[warp][0] = c2; mred[warp][1] = inc; mred[warp][2] = nrm; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0, e = 0.0;
      for (int w = 0; w < kBWarps; ++w) { a += mred[w][0]; c += mred[w][1]; e += mred[w][2]; }
      Bm.m_part[b][3 * m] = a;
      Bm.m_part[b][3 * m + 1] = c;
      Bm.m_part[b][3 * m + 2] = e;
    }
    __syncthreads();
  }

  // ---- synthesis: lanes are ring pairs, rows walked upwards, one table load for every map
  for (int cg = warp; 32 * cg < RP; cg += kBWarps) {
    const int k = 32 * cg + lane;
    const int lw = __reduce_min_sync(0xffffffffu, k < RP ? D.ls[(size_t)m * RP + k] : kNoStartB);
    float acc[NB][8];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[b][q] = 0.f;
    if (lw <= L) {
      const float4 *src = tm + (size_t)cg * npr * 32 + lane;
      auto load = [&](int r, float4 (&v)[kSynRowsB]) {
#pragma unroll
        for (int i = 0; i < kSynRowsB; ++i)
          v[i] = (r + i <= rlast) ? __ldcs(src + (size_t)(r + i) * 32) : make_float4(0.f, 0.f, 0.f, 0.f);
      };
      float4 cur[kSynRowsB], nxt[kSynRowsB];
      int r = (lw - m) >> 1;
      load(r, cur);
      for (; r <= rlast; r += kSynRowsB) {
        if (r + kSynRowsB <= rlast) load(r + kSynRowsB, nxt);
#pragma unroll
        for (int i = 0; i < kSynRowsB; ++i) {
          if (r + i <= rlast) {
            const dfl le{cur[i].x, cur[i].y}, lo{cur[i].z, cur[i].w};
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float4 ce = ss[(size_t)b * Lpm + 2 * (r + i)], co = ss[(size_t)b * Lpm + 2 * (r + i) + 1];
              dot2_acc(acc[b][0], acc[b][1], le, dfl{ce.x, ce.y});
              dot2_acc(acc[b][2], acc[b][3], le, dfl{ce.z, ce.w});
              dot2_acc(acc[b][4], acc[b][5], lo, dfl{co.x, co.y});
              dot2_acc(acc[b][6], acc[b][7], lo, dfl{co.z, co.w});
            }
          }
        }
#pragma unroll
        for (int i = 0; i < kSynRowsB; ++i) cur[i] = nxt[i];
      }
    }
    if (k < RP) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (!on[b] || m > Lb[b]) continue;
        const double er = (double)acc[b][0] + (double)acc[b][1], ei = (double)acc[b][2] + (double)acc[b][3];
        const double orr = (double)acc[b][4] + (double)acc[b][5], oi = (double)acc[b][6] + (double)acc[b][7];
        Bm.FS[b][(size_t)m * RP + k] = make_double4_32a(er + orr, ei + oi, er - orr, ei - oi);
      }
    }
  }
}

}  // namespace

// tl [NB][Lpm] double2 | max(NB Lpm, 2 NB chunk) float4
static size_t batch_smem(int nb, int chunk, int lmax, int RP) {
  const size_t Lpm = (size_t)lmax + 1 + kLB;
  const size_t nk = RP < chunk ? (size_t)RP : (size_t)chunk;
  const size_t q = (size_t)nb * Lpm > 2 * (size_t)nb * nk ? (size_t)nb * Lpm : 2 * (size_t)nb * nk;
  return (size_t)nb * Lpm * sizeof(double2) + q * sizeof(float4);
}

size_t leg_batch_smem(int nb, int lmax, int RP) { return batch_smem(nb, 1024, lmax, RP); }

template <int MODE>
static void launch_lb(const LegArgs &a, const LegDfArgs &d, const LegBatchMaps &bm, cudaStream_t s) {
  raise_smem_cap(reinterpret_cast<const void *>(legendre_batch_kernel<2, 256, 1024, 1, MODE>));
  legendre_batch_kernel<2, 256, 1024, 1, MODE><<<a.lmax + 1, 256, batch_smem(2, 1024, a.lmax, a.RP), s>>>(a, d, bm);
}

void launch_legendre_batch(const LegArgs &a, const LegDfArgs &d, const LegBatchMaps &bm, int nb, cudaStream_t s,
                           int mode) {
  (void)nb;   // groups of kLegBatchMax = 2 maps (four were measured no faster per map)
  if (mode == LEG_SYNTH) launch_lb<LEG_SYNTH>(a, d, bm, s);
  else if (mode == LEG_ANALYSIS) launch_lb<LEG_ANALYSIS>(a, d, bm, s);
  else launch_lb<LEG_ITER>(a, d, bm, s);
}

}  // namespace wfk
