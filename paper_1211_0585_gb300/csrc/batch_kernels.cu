// Batched messenger iteration: B independent solves of one HEALPix shape
// (nside, lmax) advance together, one kernel per stage for all of them.
// Each slot has its own data, noise, mask, C_l, lambda schedule and band
// limit; the Legendre functions depend on the shape only, so the Legendre
// stage is a pair of real GEMMs per m over a precomputed table
// Lambda_m[l][k] = lambda_lm(x_k) (FP32, built once from the double-float
// recurrence):
//   analysis   t_{l,b} = sum_k Lambda_m[l][k] X_{k,b},  X = E (l-m even) or O (l-m odd)
//   synthesis  E_{k,b} = sum_{l-m even} Lambda_m[l][k] s_{l,b},  O likewise
// Mixed precision: the ring FFTs and both contractions run in FP32 (FP32
// accumulation over k-chunks of 32 rings, chunk sums added in double), the
// state s_lm, the Eq. 3 / Eq. 4 updates, the chi^2 reductions and the
// controller run in double.
#include <cuda_runtime.h>

#include <algorithm>

#include "ctl.cuh"
#include "df.cuh"
#include "fft.cuh"
#include "wf_internal.h"

namespace wfk {

namespace {

__device__ __forceinline__ size_t aidx(int lmax, int l, int m) { return (size_t)m * (2 * lmax + 1 - m) / 2 + l; }

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 f2conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.x, v.z); }  // hi parts of a df complex

}  // namespace

// Lambda table: one thread per (m, k) runs the double-float recurrence from
// its start values and writes lambda_lm(x_k) for every l (0 below l_start).
__global__ void lam_table_kernel(const double *xk, const LegDfArgs D, int lmax, int RP, float *lam) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(lmax + 1) * RP) return;
  const int m = (int)(id / RP), k = (int)(id % RP);
  const size_t mk = (size_t)m * RP + k;
  const int ls = D.ls[mk];
  const float4 s4 = D.sv[mk];
  const dfl x = df_from(xk[k]);
  const size_t base = aidx(lmax, m, m);
  dfl p1 = {0.f, 0.f}, p2 = {0.f, 0.f};
  for (int l = m; l <= lmax; ++l) {
    float v = 0.f;
    if (l >= ls) {
      dfl mu;
      if (l == ls) mu = dfl{s4.x, s4.y};
      else if (l == ls + 1) mu = dfl{s4.z, s4.w};
      else {
        const float2 a2 = D.A[base + (l - m)];
        mu = df_step(dfl{a2.x, a2.y}, x, p1, p2);
      }
      p2 = p1;
      p1 = mu;
      v = (float)(D.g[base + (l - m)] * df_to(mu));
    }
    lam[(base + (l - m)) * (size_t)RP + k] = v;
  }
}

// ---------------------------------------------------------------- ring stage
// One CTA per (ring, group of G slots). The ring values of every slot are
// real, so two slots a, b share one complex FFT: the inverse transform of
// Z = G_a + i G_b gives f_a + i f_b, and the forward transform of u_a + i u_b
// gives Z with U_a = (Z_q + conj Z_{n-q}) / 2 and U_b = (Z_q - conj Z_{n-q}) / 2i.
// The G / 2 packed arrays share every twiddle load, the pixel pass updates
// them in place (the inverse transform's output order is the forward
// transform's input order), and the G slots read their Fourier coefficients
// as one contiguous run of G float4. Four CTAs of 128 threads per SM, so that
// the FFT passes of one CTA overlap the global loads and stores of another.
constexpr int kBringThreads = 128;
template <int G>
__global__ void __launch_bounds__(kBringThreads, 4) bring_kernel(const BatchArgs A) {
  static_assert(G % 2 == 0, "slots are packed in pairs");
  constexpr int P = G / 2;
  extern __shared__ float2 bsm[];
  const int r = A.order[A.first + blockIdx.x], b0 = blockIdx.y * G;
  const int B = A.B;
  // slots of this group that iterate (the group's live mask is uniform per CTA)
  bool on[G];
  bool any = false;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int b = b0 + g;
    on[g] = b < B && A.active[b] && !A.ctl[b].done;
    any |= on[g];
  }
  if (!any) return;
  const RingDev rg = A.rings[r];
  const int n = rg.n, M = 1 << rg.logM;
  float2 *buf = bsm;                                          // [P][M] (swizzled, px)
  __shared__ double red[kBringThreads / 32][2 * G];
  const float4 *hs = A.hsf + rg.hs_off;
  const float4 *ch = A.chf + rg.ch_off;
  const float2 *Bf = A.Bf2 + rg.B_off;
  const int k = rg.pair, slot = rg.side;
  int Lg[G];
  float lt[G], l1t[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (on[g]) {
      const Ctl &c = A.ctl[b0 + g];
      Lg[g] = c.lsht;
      lt[g] = (float)(c.lambda * c.tau);
      l1t[g] = (float)((c.lambda - 1.0) * c.tau);
    } else {
      Lg[g] = -1; lt[g] = 0.f; l1t[g] = 0.f;
    }
  }
  int Lmax = -1;
#pragma unroll
  for (int g = 0; g < G; ++g) Lmax = max(Lmax, Lg[g]);

  // fold F_m onto residues q for the G slots, packed in pairs
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    float2 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float2(0.f, 0.f);
    int j = 0;
    for (int m = q; m <= Lmax; m += n, ++j) {
      const float4 *src = A.FS + ((size_t)m * A.RP + k) * B + b0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (m > Lg[g]) continue;
        const float4 f4 = __ldg(src + g);
        float2 f = slot ? make_float2(f4.z, f4.w) : make_float2(f4.x, f4.y);
        if (rg.shifted && (j & 1)) { f.x = -f.x; f.y = -f.y; }
        acc[g] = f2add(acc[g], f);
      }
    }
    j = 1;
    for (int m = (q == 0 ? n : n - q); m <= Lmax; m += n, ++j) {
      const float4 *src = A.FS + ((size_t)m * A.RP + k) * B + b0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (m > Lg[g]) continue;
        const float4 f4 = __ldg(src + g);
        float2 f = slot ? make_float2(f4.z, -f4.w) : make_float2(f4.x, -f4.y);
        if (rg.shifted && (j & 1)) { f.x = -f.x; f.y = -f.y; }
        acc[g] = f2add(acc[g], f);
      }
    }
    const float2 h = hi2(hs[q]), cq = rg.blue ? hi2(ch[q]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int pp = 0; pp < P; ++pp) {
      float2 va = acc[2 * pp], vb = acc[2 * pp + 1];
      if (rg.shifted) { va = f2mul(va, h); vb = f2mul(vb, h); }
      const float2 z = make_float2(va.x - vb.y, va.y + vb.x);    // G_a + i G_b
      buf[pp * M + px<OpsF32>(q)] = rg.blue ? f2mul(f2conj(z), cq) : z;
    }
  }
  if (rg.blue)
    for (int q = n + threadIdx.x; q < M; q += blockDim.x)
#pragma unroll
      for (int pp = 0; pp < P; ++pp) buf[pp * M + px<OpsF32>(q)] = make_float2(0.f, 0.f);
  __syncthreads();
  if (rg.blue) bluestein4<OpsF32, P>(buf, M, M, rg.logM, Bf, A.tw2, A.logMmax);
  else fft_dif4<OpsF32, P>(buf, M, M, rg.logM, +1, A.tw2, A.logMmax);

  // Eq. 3 per pixel (in place: s_a + i s_b -> u_a + i u_b) and the chi^2
  // partials in FP32 (per-thread sums, warp sums by shuffles), the sum over
  // warps in double
  float c2n[G], c2l[G];
#pragma unroll
  for (int g = 0; g < G; ++g) { c2n[g] = 0.f; c2l[g] = 0.f; }
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const float2 cp = rg.blue ? hi2(ch[p]) : make_float2(0.f, 0.f);
    const int br = px<OpsF32>(rg.blue ? p : digitrev(p, rg.logM));
#pragma unroll
    for (int pp = 0; pp < P; ++pp) {
      const float2 z = buf[pp * M + br];
      float sv[2];
      if (rg.blue) {   // the inverse DFT came out conjugated (conj of the DFT of conj Z)
        const float2 R = f2mul(cp, z);
        sv[0] = R.x; sv[1] = -R.y;
      } else {
        sv[0] = z.x; sv[1] = z.y;
      }
      float u[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int g = 2 * pp + e;
        u[e] = 0.f;
        if (!on[g]) continue;
        const size_t pix = (size_t)(b0 + g) * A.npix + rg.off + p;
        const float2 dw = __ldg(A.dw32 + pix);
        const float wp = dw.y;
        const float res = dw.x - sv[e];
        const float gg = __fdividef(wp, fmaf(l1t[g], wp, 1.f));
        c2n[g] = fmaf(wp * res, res, c2n[g]);
        c2l[g] = fmaf(gg * res, res, c2l[g]);
        u[e] = lt[g] * gg * res;
      }
      const float2 uz = make_float2(u[0], u[1]);
      buf[pp * M + br] = rg.blue ? f2mul(uz, cp) : uz;
    }
  }
  if (rg.blue)
    for (int p = n + threadIdx.x; p < M; p += blockDim.x)
#pragma unroll
      for (int pp = 0; pp < P; ++pp) buf[pp * M + px<OpsF32>(p)] = make_float2(0.f, 0.f);
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      float a = c2n[g], bsum = c2l[g];   // warp sums in FP32, the per-warp partials in double
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
      }
      if (lane == 0) { red[warp][2 * g] = a; red[warp][2 * g + 1] = bsum; }
    }
    __syncthreads();   // also orders the pixel pass before the forward transform
    if (threadIdx.x < G && on[threadIdx.x]) {
      const int g = threadIdx.x;
      double sa = 0.0, sb = 0.0;
      for (int w2 = 0; w2 < kBringThreads / 32; ++w2) { sa += red[w2][2 * g]; sb += red[w2][2 * g + 1]; }
      A.ring_part[((size_t)(b0 + g) * A.R + r) * 2] = sa;
      A.ring_part[((size_t)(b0 + g) * A.R + r) * 2 + 1] = sb;
    }
  }
  // forward DFT of u_a + i u_b
  if (rg.blue) bluestein4<OpsF32, P>(buf, M, M, rg.logM, Bf, A.tw2, A.logMmax);
  else fft_dit4<OpsF32, P>(buf, M, M, rg.logM, -1, A.tw2, A.logMmax);
  // unpack U_a, U_b and unfold to m = 0 .. Lmax
  const float om = (float)A.omega;
  for (int m = threadIdx.x; m <= Lmax; m += blockDim.x) {
    const int q = m % n, j = m / n, q2 = q == 0 ? 0 : n - q;
    const float2 cq = rg.blue ? hi2(ch[q]) : make_float2(0.f, 0.f);
    const float2 cq2 = rg.blue ? hi2(ch[q2]) : make_float2(0.f, 0.f);
    const float2 hq = f2conj(hi2(hs[q]));
    float4 *dst4 = A.FT + ((size_t)m * A.RP + k) * B + b0;
#pragma unroll
    for (int pp = 0; pp < P; ++pp) {
      float2 Z1 = buf[pp * M + px<OpsF32>(q)], Z2 = buf[pp * M + px<OpsF32>(q2)];
      if (rg.blue) { Z1 = f2mul(cq, Z1); Z2 = f2mul(cq2, Z2); }
      float2 U[2];
      U[0] = make_float2(0.5f * (Z1.x + Z2.x), 0.5f * (Z1.y - Z2.y));   // (Z_q + conj Z_{n-q}) / 2
      U[1] = make_float2(0.5f * (Z1.y + Z2.y), 0.5f * (Z2.x - Z1.x));   // (Z_q - conj Z_{n-q}) / 2i
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int g = 2 * pp + e;
        if (m > Lg[g]) continue;
        float2 V = U[e];
        if (rg.shifted) {
          V = f2mul(V, hq);
          if (j & 1) { V.x = -V.x; V.y = -V.y; }
        }
        float *dst = reinterpret_cast<float *>(dst4 + g) + 2 * slot;
        dst[0] = om * V.x;
        dst[1] = om * V.y;
      }
    }
  }
}

// ---------------------------------------------------------------- analysis GEMM + Eq. 4
// Tile: 64 values of l (32 of each parity of l - m) x all slots, reduced over
// every ring pair in chunks of 32. Thread (par, rg, cg): rows par + 2 (4 rg + i),
// i < 4, columns 8 cg .. 8 cg + 7 of the 2 B (re, im) columns.
constexpr int kAT = 64, kKC = 32;

__global__ void __launch_bounds__(256) bana_kernel(const BatchArgs A) {
  __shared__ __align__(16) float Lt[kKC][2][32];           // [k][parity][row]
  __shared__ __align__(16) float XEO[2][kKC][2 * kBatchMax];  // E / O: [k][2 b + re/im]
  float(*XE)[2 * kBatchMax] = XEO[0];
  float(*XO)[2 * kBatchMax] = XEO[1];
  // after the k loop the X tiles are dead; the epilogue partials reuse them
  double(*part)[16][3] = reinterpret_cast<double(*)[16][3]>(&XEO[0][0][0]);
  const int2 tile = A.tiles[blockIdx.x];
  const int m = tile.x, l0 = tile.y;
  const int Lact = A.bstate[0];
  const int B = A.B, RP = A.RP, lmax = A.lmax;
  const int t = threadIdx.x;
  const int cg = t & 15, rgp = t >> 4;          // column group, row group (0..15)
  const int par = rgp & 1, rg = rgp >> 1;       // parity, row group within parity (0..7)
  const bool live = m <= Lact && l0 <= Lact;
  // chunk sums folded into double-float accumulators (two_sum on the FP32 pipe)
  float ah[4][8], al[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) { ah[i][j] = 0.f; al[i][j] = 0.f; }
  if (live) {
    const size_t base = aidx(lmax, m, m);
    for (int k0 = 0; k0 < RP; k0 += kKC) {
      for (int e = t; e < kAT * kKC; e += 256) {
        const int row = e / kKC, kk = e % kKC;
        const int l = l0 + row, k = k0 + kk;
        float v = 0.f;
        if (l <= lmax && l <= Lact && k < RP) v = A.lam[(base + (l - m)) * (size_t)RP + k];
        Lt[kk][row & 1][row >> 1] = v;
      }
      for (int e = t; e < kKC * B; e += 256) {
        const int kk = e / B, bb = e % B, k = k0 + kk;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < RP) f = A.FT[((size_t)m * RP + k) * B + bb];
        XE[kk][2 * bb] = f.x + f.z;
        XE[kk][2 * bb + 1] = f.y + f.w;
        XO[kk][2 * bb] = f.x - f.z;
        XO[kk][2 * bb + 1] = f.y - f.w;
      }
      __syncthreads();
      if (8 * cg < 2 * B) {
        float pa[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) pa[i][j] = 0.f;
        const float(*X)[2 * kBatchMax] = par ? XO : XE;
#pragma unroll 8
        for (int kk = 0; kk < kKC; ++kk) {
          const float4 a = *reinterpret_cast<const float4 *>(&Lt[kk][par][4 * rg]);
          const float4 x0 = *reinterpret_cast<const float4 *>(&X[kk][8 * cg]);
          const float4 x1 = *reinterpret_cast<const float4 *>(&X[kk][8 * cg + 4]);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) pa[i][j] = fmaf(av[i], xv[j], pa[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float s = ah[i][j] + pa[i][j];
            const float bb = s - ah[i][j];
            al[i][j] += (ah[i][j] - (s - bb)) + (pa[i][j] - bb);
            ah[i][j] = s;
          }
      }
      __syncthreads();
    }
  }
  // epilogue: Eq. 4 per (l, slot) on the double-float state (f_l from the
  // per-iteration table, 0 above the slot's band limit and where C_l = 0),
  // prior chi^2 / increment / norm partials in FP32 (all on the FP32 pipe)
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int bb = 4 * cg + jj;      // slot of columns 8 cg + 2 jj, + 1
    float c2 = 0.f, inc = 0.f, nrm = 0.f;
    if (bb < B && A.active[bb] && !A.ctl[bb].done) {
      const float2 *fb = A.fdf + (size_t)bb * (lmax + 1);
      const float *ib = A.icl + (size_t)bb * (lmax + 1);
      float4 *sb = A.sdf + (size_t)bb * A.nalm;
      const float wgt = (m == 0) ? 1.f : 2.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int l = l0 + par + 2 * (4 * rg + i);
        if (l > lmax) continue;
        const size_t idx = aidx(lmax, l, m);
        const float4 so = sb[idx];
        float4 sn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live) {
          const float2 f2 = fb[l];
          const dfl f = dfl{f2.x, f2.y};
          const dfl re = df_mul(f, df_add(dfl{so.x, so.y}, dfl{ah[i][2 * jj], al[i][2 * jj]}));
          const dfl im = df_mul(f, df_add(dfl{so.z, so.w}, dfl{ah[i][2 * jj + 1], al[i][2 * jj + 1]}));
          sn = make_float4(re.h, re.l, im.h, im.l);
        }
        c2 += wgt * (so.x * so.x + so.z * so.z) * ib[l];
        const float dx = (sn.x - so.x) + (sn.y - so.y), dy = (sn.z - so.z) + (sn.w - so.w);
        inc += wgt * (dx * dx + dy * dy);
        nrm += wgt * (sn.x * sn.x + sn.z * sn.z);
        sb[idx] = sn;
        A.SP[idx * B + bb] = make_float2(sn.x, sn.z);
      }
    }
    if (bb < kBatchMax) {
      part[bb][rgp][0] = c2;
      part[bb][rgp][1] = inc;
      part[bb][rgp][2] = nrm;
    }
  }
  __syncthreads();
  for (int bb = t; bb < B; bb += 256) {
    double a = 0.0, bsum = 0.0, cs = 0.0;
    for (int q = 0; q < 16; ++q) { a += part[bb][q][0]; bsum += part[bb][q][1]; cs += part[bb][q][2]; }
    double *dst = A.m_part + ((size_t)bb * A.ntiles + blockIdx.x) * 3;
    dst[0] = a;
    dst[1] = bsum;
    dst[2] = cs;
  }
}

// ---------------------------------------------------------------- synthesis GEMM
// Tile: 32 ring pairs x all slots; E (l - m even) and O (odd) accumulated by
// separate thread halves over l = m .. Lact in chunks of 32.
constexpr int kST = 32, kLC = 32;

__global__ void __launch_bounds__(256) bsyn_kernel(const BatchArgs A) {
  __shared__ __align__(16) float Ls[kLC][kST];              // [l][k]
  __shared__ __align__(16) float Ss[kLC][2 * kBatchMax];    // [l][2 b + re/im]
  __shared__ __align__(16) float OutE[kST][2 * kBatchMax];  // E sums, read by the O half
  const int2 tile = A.stiles[blockIdx.x];
  const int m = tile.x, k0 = tile.y;
  const int Lact = A.bstate[0];
  const int B = A.B, RP = A.RP, lmax = A.lmax;
  const int t = threadIdx.x;
  if (m > Lact) {
    for (int e = t; e < kST * B; e += 256) {
      const int kk = e / B, bb = e % B, k = k0 + kk;
      if (k < RP) A.FS[((size_t)m * RP + k) * B + bb] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;
  }
  const int eo = t >> 7;                  // 0: E (even l - m), 1: O
  const int tt = t & 127;
  const int cg = tt & 15, kg = tt >> 4;   // column group (8 columns), ring group (4 rings)
  const size_t base = aidx(lmax, m, m);
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int lc = m; lc <= Lact; lc += kLC) {
    for (int e = t; e < kLC * kST; e += 256) {
      const int ll = e / kST, kk = e % kST;
      const int l = lc + ll, k = k0 + kk;
      float v = 0.f;
      if (l <= Lact && k < RP) v = A.lam[(base + (l - m)) * (size_t)RP + k];
      Ls[ll][kk] = v;
    }
    for (int e = t; e < kLC * B; e += 256) {
      const int ll = e / B, bb = e % B, l = lc + ll;
      float2 v = make_float2(0.f, 0.f);
      if (l <= Lact) v = A.SP[(base + (l - m)) * B + bb];
      Ss[ll][2 * bb] = v.x;
      Ss[ll][2 * bb + 1] = v.y;
    }
    __syncthreads();
    if (8 * cg < 2 * B) {
#pragma unroll 4
      for (int ll = eo; ll < kLC; ll += 2) {
        const float4 a = *reinterpret_cast<const float4 *>(&Ls[ll][4 * kg]);
        const float4 x0 = *reinterpret_cast<const float4 *>(&Ss[ll][8 * cg]);
        const float4 x1 = *reinterpret_cast<const float4 *>(&Ss[ll][8 * cg + 4]);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  if (eo == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) OutE[4 * kg + i][8 * cg + j] = acc[i][j];
  }
  __syncthreads();
  if (eo == 1 && 8 * cg < 2 * B) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + 4 * kg + i;
      if (k >= RP) continue;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int bb = 4 * cg + jj;
        if (bb >= B) continue;
        const float er = OutE[4 * kg + i][2 * bb], ei = OutE[4 * kg + i][2 * bb + 1];
        const float orr = acc[i][2 * jj], oi = acc[i][2 * jj + 1];
        A.FS[((size_t)m * RP + k) * B + bb] = make_float4(er + orr, ei + oi, er - orr, ei - oi);
      }
    }
  }
}

// ---------------------------------------------------------------- control
__global__ void __launch_bounds__(256) bctl_kernel(const BatchArgs A) {
  __shared__ double sh[5][256];
  const int b = blockIdx.x;
  if (!A.active[b] || A.ctl[b].done) return;
  double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
  for (int i = threadIdx.x; i < A.R; i += blockDim.x) {
    a0 += A.ring_part[((size_t)b * A.R + i) * 2];
    a1 += A.ring_part[((size_t)b * A.R + i) * 2 + 1];
  }
  for (int i = threadIdx.x; i < A.ntiles; i += blockDim.x) {
    const double *p = A.m_part + ((size_t)b * A.ntiles + i) * 3;
    b0 += p[0]; b1 += p[1]; b2 += p[2];
  }
  sh[0][threadIdx.x] = a0; sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = b0; sh[3][threadIdx.x] = b1; sh[4][threadIdx.x] = b2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    ctl_advance(A.ctl + b, A.cl + (size_t)b * (A.lmax + 1), sh[2][0], sh[0][0], sh[1][0], sh[3][0], sh[4][0],
                nullptr, 0, A.last + b);
}

// largest band limit and number of slots still iterating
__global__ void bstate_kernel(const BatchArgs A, int *bstate) {
  __shared__ int lmx[kBatchMax], nact[kBatchMax];
  const int b = threadIdx.x;
  int l = -1, a = 0;
  if (b < A.B && A.active[b] && !A.ctl[b].done) { l = A.ctl[b].lsht; a = 1; }
  lmx[b] = l;
  nact[b] = a;
  __syncthreads();
  if (b == 0) {
    int L = -1, n = 0;
    for (int i = 0; i < kBatchMax; ++i) { L = max(L, lmx[i]); n += nact[i]; }
    bstate[0] = L;
    bstate[1] = n;
  }
}

// reset slot b: zero its state and its synthesis coefficients
__global__ void bzero_slot_kernel(const BatchArgs A, int b) {
  const long long nF = (long long)(A.lmax + 1) * A.RP;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += (long long)gridDim.x * blockDim.x)
    A.FS[i * A.B + b] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nalm; i += (long long)gridDim.x * blockDim.x)
    A.sdf[(size_t)b * A.nalm + i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// the double-float state of slot b as double a_lm (export of a finished solve)
__global__ void bexport_slot_kernel(const BatchArgs A, int b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nalm; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = A.sdf[(size_t)b * A.nalm + i];
    A.s[(size_t)b * A.nalm + i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}

// per-iteration filter table f_l(lambda_b) = C_l / (C_l + lambda tau Omega)
// (0 above the slot's band limit or where C_l = 0) and 1 / C_l (0 where C_l = 0)
__global__ void bfilter_kernel(const BatchArgs A) {
  const int b = blockIdx.x;
  if (!A.active[b] || A.ctl[b].done) return;
  const Ctl &c = A.ctl[b];
  const double lto = c.lambda * c.tau * c.omega;
  const double *clb = A.cl + (size_t)b * (A.lmax + 1);
  for (int l = threadIdx.x; l <= A.lmax; l += blockDim.x) {
    const double cl = clb[l];
    const double f = (cl > 0.0 && l <= c.lsht) ? cl / (cl + lto) : 0.0;
    const dfl fd = df_from(f);
    A.fdf[(size_t)b * (A.lmax + 1) + l] = make_float2(fd.h, fd.l);
    A.icl[(size_t)b * (A.lmax + 1) + l] = cl > 0.0 ? (float)(1.0 / cl) : 0.f;
  }
}

// hi parts of a double-float complex table (the FP32 twiddle and Bluestein tables)
__global__ void hi_table_kernel(const float4 *src, float2 *dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = hi2(src[i]);
}

void launch_hi_table(const float4 *src, float2 *dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  hi_table_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(src, dst, n);
}

void launch_batch_export_slot(const BatchArgs &a, int b, cudaStream_t s) {
  bexport_slot_kernel<<<256, 256, 0, s>>>(a, b);
}

void launch_lam_table(const double *x, const LegDfArgs &D, int lmax, int RP, float *lam, cudaStream_t s) {
  const long long n = (long long)(lmax + 1) * RP;
  lam_table_kernel<<<(int)((n + 127) / 128), 128, 0, s>>>(x, D, lmax, RP, lam);
}

// FP32 copies of slot b's data and inverse noise for the ring stage
__global__ void bconvert_slot_kernel(const BatchArgs A, int b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.npix; i += (long long)gridDim.x * blockDim.x) {
    A.dw32[(size_t)b * A.npix + i] = make_float2((float)A.d[(size_t)b * A.npix + i], (float)A.w[(size_t)b * A.npix + i]);
  }
}

void launch_batch_convert_slot(const BatchArgs &a, int b, cudaStream_t s) {
  bconvert_slot_kernel<<<512, 256, 0, s>>>(a, b);
}

// shared memory of one packed pair of slots of a class
static size_t bring_smem_per_pair(int logM) { return ((size_t)1 << logM) * sizeof(float2); }

// slots per ring-stage CTA of a class: 8, 4 or 2 (pairs share one FFT),
// within a quarter of an SM's shared memory so that four CTAs share each SM
static int batch_ring_group(int logM, int B) {
  int G = 8;
  while (G > 2 && ((G / 2) * bring_smem_per_pair(logM) > 56 * 1024 || G >= 2 * B)) G >>= 1;
  return G;
}

template <int G>
static void launch_bring(const BatchArgs &a, const RingClass &c, cudaStream_t s) {
  const size_t sm = (size_t)(G / 2) * bring_smem_per_pair(c.logM);
  BatchArgs ac = a;
  ac.first = c.first;
  bring_kernel<G><<<dim3(c.count, (a.B + G - 1) / G), kBringThreads, sm, s>>>(ac);
}

void launch_batch_iteration(const BatchArgs &a, const RingClass *cls, int ncls, int n_stiles, int *bstate,
                            cudaStream_t s) {
  raise_smem_cap(reinterpret_cast<const void *>(bring_kernel<2>));
  raise_smem_cap(reinterpret_cast<const void *>(bring_kernel<4>));
  raise_smem_cap(reinterpret_cast<const void *>(bring_kernel<8>));
  for (int c = 0; c < ncls; ++c) {
    if (cls[c].count <= 0) continue;
    const int G = batch_ring_group(cls[c].logM, a.B);
    if (G == 8) launch_bring<8>(a, cls[c], s);
    else if (G == 4) launch_bring<4>(a, cls[c], s);
    else launch_bring<2>(a, cls[c], s);
  }
  bfilter_kernel<<<a.B, 256, 0, s>>>(a);
  bana_kernel<<<a.ntiles, 256, 0, s>>>(a);
  bsyn_kernel<<<n_stiles, 256, 0, s>>>(a);
  bctl_kernel<<<a.B, 256, 0, s>>>(a);
  bstate_kernel<<<1, kBatchMax, 0, s>>>(a, bstate);
}

void launch_batch_state(const BatchArgs &a, int *bstate, cudaStream_t s) {
  bstate_kernel<<<1, kBatchMax, 0, s>>>(a, bstate);
}

void launch_batch_zero_slot(const BatchArgs &a, int b, cudaStream_t s) {
  bzero_slot_kernel<<<512, 256, 0, s>>>(a, b);
}

}  // namespace wfk
