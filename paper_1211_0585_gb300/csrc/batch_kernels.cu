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

#include "batch_engine.h"
#include "ctl.cuh"
#include "df.cuh"
#include "fft.cuh"
#include "wf_internal.h"

namespace wfk {

namespace {

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 f2conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.x, v.z); }  // hi parts of a df complex
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}

}  // namespace

// ---------------------------------------------------------------- ring stage
// One CTA per (ring, group of G slots). The ring values of every slot are
// real, so two slots a, b share one complex FFT: the inverse transform of
// Z = G_a + i G_b gives f_a + i f_b, and the forward transform of u_a + i u_b
// gives Z with U_a = (Z_q + conj Z_{n-q}) / 2 and U_b = (Z_q - conj Z_{n-q}) / 2i.
// The G / 2 packed arrays share every twiddle load, the pixel pass updates
// them in place (the inverse transform's output order is the forward
// transform's input order), and the G slots read their Fourier coefficients
// as one contiguous run of G float4. Four CTAs of 256 threads per SM (64
// registers), so that the FFT passes of one CTA overlap the global loads and
// stores of the others.
constexpr int kBringThreads = 256;
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
  // alias partial sums of rings shorter than the block: [kBringThreads][G] after
  // the FFT buffers (present in the classes whose rings can be that short)
  float2(*fpart)[G] = reinterpret_cast<float2(*)[G]>(bsm + P * M);
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
  // Every global line this CTA reads goes to L2 first, all requests at once:
  // the Fourier coefficients of the G slots (one run of G float4 per m) and
  // the slots' (d, w) on the ring. The fold's and the pixel pass's loads then
  // wait on L2, not on HBM, one after another.
  for (int m = threadIdx.x; m <= Lmax; m += blockDim.x) prefetch_l2(A.FS + ((size_t)m * A.RP + k) * B + b0);
  {
    constexpr int kLine = 128 / sizeof(float2);   // pixels per line
    const int nl = (n + kLine - 1) / kLine + 1;     // the ring's run may straddle one more line
    for (int e = threadIdx.x; e < G * nl; e += blockDim.x) {
      const int g = e / nl, li = e % nl;
      if (on[g]) prefetch_l2(A.dw32 + (size_t)(b0 + g) * A.npix + rg.off + min(li * kLine, n - 1));
    }
  }

  // fold F_m onto residues q for the G slots (m-aliasing), packed in pairs;
  // on rings shorter than the block each residue's alias series is split over
  // several threads (partial sums added in a fixed order)
  auto alias_sum = [&](int q, int j0, int dj, float2 (&acc)[G]) {
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float2(0.f, 0.f);
    for (int j = j0, m = q + n * j0; m <= Lmax; j += dj, m += n * dj) {
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
    for (int j = 1 + j0, m = n * (1 + j0) - q; m <= Lmax; j += dj, m += n * dj) {
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
  };
  auto store_residue = [&](int q, const float2 (&acc)[G]) {
    const float2 h = rg.shifted ? hi2(hs[q]) : make_float2(0.f, 0.f), cq = rg.blue ? hi2(ch[q]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int pp = 0; pp < P; ++pp) {
      float2 va = acc[2 * pp], vb = acc[2 * pp + 1];
      if (rg.shifted) { va = f2mul(va, h); vb = f2mul(vb, h); }
      const float2 z = make_float2(va.x - vb.y, va.y + vb.x);    // G_a + i G_b
      buf[pp * M + px<OpsF32>(q)] = rg.blue ? f2mul(f2conj(z), cq) : z;
    }
  };
  if (n >= kBringThreads) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      float2 acc[G];
      alias_sum(q, 0, 1, acc);
      store_residue(q, acc);
    }
  } else {
    const int nj = kBringThreads / n, t = threadIdx.x;
    if (t < n * nj) {
      float2 acc[G];
      alias_sum(t % n, t / n, nj, acc);
#pragma unroll
      for (int g = 0; g < G; ++g) fpart[t][g] = acc[g];
    }
    __syncthreads();
    if (t < n) {
      float2 acc[G];
#pragma unroll
      for (int g = 0; g < G; ++g) acc[g] = make_float2(0.f, 0.f);
      for (int jg = 0; jg < nj; ++jg)
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = f2add(acc[g], fpart[jg * n + t][g]);
      store_residue(t, acc);
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
  // kPix pixels per thread at a time: their (d, w) loads are issued together
  constexpr int kPix = G <= 2 ? 8 : 16 / G;
  for (int p0 = threadIdx.x; p0 < n; p0 += kPix * blockDim.x) {
    float2 dw[kPix][G];
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      const int p = p0 + k * blockDim.x;
#pragma unroll
      for (int g = 0; g < G; ++g)
        dw[k][g] = (p < n && on[g]) ? __ldg(A.dw32 + (size_t)(b0 + g) * A.npix + rg.off + p) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      const int p = p0 + k * blockDim.x;
      if (p >= n) break;
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
          const float wp = dw[k][g].y;
          const float res = dw[k][g].x - sv[e];
          const float gg = __fdividef(wp, fmaf(l1t[g], wp, 1.f));
          c2n[g] = fmaf(wp * res, res, c2n[g]);
          c2l[g] = fmaf(gg * res, res, c2l[g]);
          u[e] = lt[g] * gg * res;
        }
        const float2 uz = make_float2(u[0], u[1]);
        buf[pp * M + br] = rg.blue ? f2mul(uz, cp) : uz;
      }
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
        reinterpret_cast<float2 *>(dst4 + g)[slot] = make_float2(om * V.x, om * V.y);
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

// reset slot b: zero its state, its Fourier coefficients and its columns of
// the synthesis operand (2 b, 2 b + 1 of every part of every 32-wide chunk)
__global__ void bzero_slot_kernel(const BatchArgs A, const TcArgs T, long long nchunks, int b) {
  const long long nF = (long long)(A.lmax + 1) * A.RP;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += stride)
    A.FS[i * A.B + b] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nalm; i += stride)
    A.sdf[(size_t)b * A.nalm + i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nchunks * 3 * 64; i += stride) {
    const long long q = i >> 6, e = i & 63;   // (chunk, part), (column 2 b or 2 b + 1, i within the chunk)
    T.SPT[(q * T.Nc + 2 * b + (e >> 5)) * 32 + (e & 31)] = 0.f;
  }
}

// the double-float state of slot b as double a_lm (export of a finished solve)
__global__ void bexport_slot_kernel(const BatchArgs A, int b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nalm; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = A.sdf[(size_t)b * A.nalm + i];
    A.s[(size_t)b * A.nalm + A.alm_of_row[i]] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
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
    A.fdf[(size_t)l * A.B + b] = make_float2(fd.h, fd.l);
    A.icl[(size_t)l * A.B + b] = cl > 0.0 ? (float)(1.0 / cl) : 0.f;
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


// FP32 copies of slot b's data and inverse noise for the ring stage
__global__ void bconvert_slot_kernel(const BatchArgs A, int b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.npix; i += (long long)gridDim.x * blockDim.x) {
    A.dw32[(size_t)b * A.npix + i] = make_float2((float)A.d[i], (float)A.w[i]);   // d, w: one staging slot
  }
}

void launch_batch_convert_slot(const BatchArgs &a, int b, cudaStream_t s) {
  bconvert_slot_kernel<<<512, 256, 0, s>>>(a, b);
}

// shared memory of one packed pair of slots of a class
static size_t bring_smem_per_pair(int logM) { return ((size_t)1 << logM) * sizeof(float2); }

// shared memory of a CTA of G slots: the packed FFT buffers, plus the alias
// partial sums when the class can hold rings shorter than the block
static size_t bring_smem(int logM, int G) {
  const size_t part = ((size_t)1 << logM) <= 2 * kBringThreads ? (size_t)kBringThreads * G * sizeof(float2) : 0;
  return (size_t)(G / 2) * bring_smem_per_pair(logM) + part;
}


// default slots per ring-stage CTA of a class (before autotuning): 8, 4 or 2
// (pairs share one FFT), within a quarter of an SM's shared memory so that four
// CTAs share each SM
static int batch_ring_group(int logM, int B) {
  int G = 8;
  while (G > 2 && (bring_smem(logM, G) > 54 * 1024 || G >= 2 * B)) G >>= 1;
  return G;
}

template <int G>
static void launch_bring(const BatchArgs &a, const RingClass &c, cudaStream_t s) {
  const size_t sm = bring_smem(c.logM, G);
  BatchArgs ac = a;
  ac.first = c.first;
  bring_kernel<G><<<dim3(c.count, (a.B + G - 1) / G), kBringThreads, sm, s>>>(ac);
}

// slots per CTA that a ring class may use: even, at most 8, the packed FFT
// buffers within the shared memory of one CTA
bool batch_ring_group_ok(int logM, int G) {
  return (G == 2 || G == 4 || G == 8) && bring_smem(logM, G) <= 200 * 1024;
}

void launch_batch_ring_class(const BatchArgs &a, const RingClass &c, int G, cudaStream_t s) {
  raise_smem_cap(reinterpret_cast<const void *>(bring_kernel<2>));
  raise_smem_cap(reinterpret_cast<const void *>(bring_kernel<4>));
  raise_smem_cap(reinterpret_cast<const void *>(bring_kernel<8>));
  if (c.count <= 0) return;
  if (G <= 0 || !batch_ring_group_ok(c.logM, G)) G = batch_ring_group(c.logM, a.B);
  if (G == 8) launch_bring<8>(a, c, s);
  else if (G == 4) launch_bring<4>(a, c, s);
  else launch_bring<2>(a, c, s);
}

void launch_batch_iteration(const BatchArgs &a, const TcArgs &t, const TcMaps &maps, const RingClass *cls, int ncls,
                            const int *groups, int *bstate, cudaStream_t s, const SynBand *bands, int nbands) {
  for (int c = 0; c < ncls; ++c) launch_batch_ring_class(a, cls[c], groups ? groups[c] : 0, s);
  bfilter_kernel<<<a.B, 256, 0, s>>>(a);
  launch_batch_gemms_tc(a, t, maps, s, 0, bands, nbands);   // FT -> XT, analysis GEMM, Eq. 4
  launch_batch_gemms_tc(a, t, maps, s, 1, bands, nbands);   // synthesis GEMM
  bctl_kernel<<<a.B, 256, 0, s>>>(a);
  bstate_kernel<<<1, kBatchMax, 0, s>>>(a, bstate);
}

void launch_batch_state(const BatchArgs &a, int *bstate, cudaStream_t s) {
  bstate_kernel<<<1, kBatchMax, 0, s>>>(a, bstate);
}

void launch_batch_zero_slot(const BatchArgs &a, const TcArgs &t, long long nchunks, int b, cudaStream_t s) {
  bzero_slot_kernel<<<512, 256, 0, s>>>(a, t, nchunks, b);
}

}  // namespace wfk
