// Ring stage in double-float arithmetic (FP64-accurate FFTs on the FP32 pipe).
//
// Same algorithm and data flow as ring.cu (fold F_m onto residues with the
// half-pixel shift, inverse DFT, Eq. 3 per pixel with the chi^2 partials,
// forward DFT, unfold), but every FFT value is a pair of floats per real
// component and every butterfly is built from error-free transformations
// (two_sum, two_prod), because GB300's FP64 pipe is 1/63 of its FP32 pipe.
// The per-pixel Eq. 3 update and the chi^2 partials stay in double (one pass
// over the ring's pixels). Tables (twiddles, half-shift, chirp, Bluestein
// filter) are stored as double-float pairs, converted once from the double
// tables when the plan is built.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "fold.cuh"
#include "wf_internal.h"

namespace wfk {

namespace {

struct dd { float h, l; };

__device__ __forceinline__ dd mk(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double todbl(dd a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ dd dadd(dd a, dd b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float r = s + e;
  return {r, e - (r - s)};
}
__device__ __forceinline__ dd dneg(dd a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dd dmul(dd a, dd b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  const float r = p + e;
  return {r, e - (r - p)};
}

// complex double-float held as float4 (re.h, re.l, im.h, im.l)
__device__ __forceinline__ float4 pack(dd re, dd im) { return make_float4(re.h, re.l, im.h, im.l); }
__device__ __forceinline__ dd RE(float4 v) { return {v.x, v.y}; }
__device__ __forceinline__ dd IM(float4 v) { return {v.z, v.w}; }
__device__ __forceinline__ float4 cmul(float4 a, float4 b) {
  const dd re = dadd(dmul(RE(a), RE(b)), dneg(dmul(IM(a), IM(b))));
  const dd im = dadd(dmul(RE(a), IM(b)), dmul(IM(a), RE(b)));
  return pack(re, im);
}
__device__ __forceinline__ float4 cconj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 cneg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

__device__ void block_sum2(double &a, double &b, double *red) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[2 * warp] = a; red[2 * warp + 1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) { sa += red[2 * w2]; sb += red[2 * w2 + 1]; }
    a = sa; b = sb;
  }
}

}  // namespace

// One CTA per ring pair: the two rings of a pair have the same length,
// half-pixel shift and tables, and real pixel values, so they share one
// complex transform (Sect. 2 basis change, both directions):
//   synthesis  IDFT(G_N + i G_S) = f_N + i f_S
//   analysis   Z = DFT(u_N + i u_S): U_N(q) = (Z_q + conj Z_{n-q}) / 2,
//                                    U_S(q) = (Z_q - conj Z_{n-q}) / (2 i)
// which halves the FFT work against one transform per ring. The equator is a
// pair of one ring (its south half stays zero). Eq. 3 runs in place on the
// inverse transform's output, which is the forward transform's input order.
// 256 threads and three CTAs per SM (up to 64 KB of FFT buffer each at Nside
// 512), so that one pair's barriers and global loads overlap another's work.
constexpr int kRingDfThreads = 256;
template <int MODE>
__global__ void __launch_bounds__(kRingDfThreads, 3) ring_df_kernel(const RingArgs A, const RingDfArgs T) {
  extern __shared__ float4 rsm[];
  const int2 pr = A.porder[A.first + blockIdx.x];  // (north ring, south ring or -1)
  const RingDev rg = A.rings[pr.x];
  const bool two = pr.y >= 0;
  const long long offS = two ? A.rings[pr.y].off : 0;
  const int n = rg.n;
  const int M = 1 << rg.logM;
  const int Mp = M;
  // [Mp] (swizzled, px): shared memory, or this CTA's part of the global scratch
  float4 *buf = A.scratch ? reinterpret_cast<float4 *>(A.scratch) + (size_t)blockIdx.x * M : rsm;
  __shared__ double red[64];
  __shared__ double4_16a fold_part[kRingDfThreads];

  int L = A.lsht;
  double lam = 1.0;
  if (MODE != RING_ITER && A.gate && A.gate->done) return;
  if (MODE == RING_ITER) {
    if (A.ctl->done) return;
    L = A.ctl->lsht;
    lam = A.ctl->lambda;
  }
  const float4 *hs = T.hs + rg.hs_off;
  const float4 *ch = T.chirp + rg.ch_off;
  const float4 *Bf = T.B + rg.B_off;
  const int k = rg.pair;

  if (MODE == RING_SYNTH || MODE == RING_ITER) {
    // folding is a handful of additions: done in double; Z = G_N + i G_S
    fold_ring2(A.FS, A.RP, k, rg.shifted, n, L, fold_part, [&](int q, double2 gN, double2 gS) {
      float4 acc = pack(mk(gN.x - gS.y), mk(gN.y + gS.x));
      if (rg.shifted) acc = cmul(acc, hs[q]);
      buf[px<OpsDF>(q)] = rg.blue ? cmul(cconj(acc), ch[q]) : acc;
    });
    if (rg.blue) {
      for (int q = n + threadIdx.x; q < M; q += blockDim.x) buf[px<OpsDF>(q)] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (rg.blue) bluestein4<OpsDF, 1>(buf, Mp, M, rg.logM, Bf, T.tw, A.logMmax);
    else fft_dif4<OpsDF, 1>(buf, Mp, M, rg.logM, +1, T.tw, A.logMmax);
  }
  // pixel p of both rings: z = f_N + i f_S at buf[loc(p)] (Bluestein: conj of ch[p] buf[p])
  auto loc = [&](int p) { return rg.blue ? px<OpsDF>(p) : px<OpsDF>(digitrev(p, rg.logM)); };
  auto pixel = [&](int p) {
    const float4 v = buf[loc(p)];
    return rg.blue ? cconj(cmul(ch[p], v)) : v;
  };
  if (MODE == RING_SYNTH) {
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const float4 z = pixel(p);
      A.map_out[rg.off + p] = todbl(RE(z));
      if (two) A.map_out[offS + p] = todbl(IM(z));
    }
    return;
  }
  if (MODE == RING_ITER) {
    // Eq. 3 and the chi^2 partials in double-float (the FP64 pipe is 1/63 of the
    // FP32 one); the per-thread partials become doubles for the block sums
    dd cnN{0.f, 0.f}, clN{0.f, 0.f}, cnS{0.f, 0.f}, clS{0.f, 0.f};
    const bool fresh = T.gainlam[pr.x] == lam;   // gains of this pair already at this lambda
    const dd ltd = mk(lam * A.tau);
    const double l1t = (lam - 1.0) * A.tau;
    auto update = [&](long long at, dd s, dd &cn, dd &cl) {  // Eq. 3, returns u
      const float2 d2 = T.d[at], w2 = T.w[at];
      const dd dv{d2.x, d2.y}, wv{w2.x, w2.y};
      dd g;
      if (fresh) {
        const float2 g2 = T.gain[at];
        g = dd{g2.x, g2.y};
      } else {  // the first pass at a new lambda: the gain from w in double
        const double w = A.w[at];
        g = mk(w / (1.0 + l1t * w));
        T.gain[at] = make_float2(g.h, g.l);
      }
      const dd res = dadd(dv, dneg(s));
      const dd r2 = dmul(res, res);
      cn = dadd(cn, dmul(wv, r2));
      cl = dadd(cl, dmul(g, r2));
      return dmul(dmul(ltd, g), res);
    };
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const float4 z = pixel(p);
      const dd uN = update(rg.off + p, RE(z), cnN, clN);
      const dd uS = two ? update(offS + p, IM(z), cnS, clS) : dd{0.f, 0.f};
      const float4 u = pack(uN, uS);
      buf[loc(p)] = rg.blue ? cmul(u, ch[p]) : u;
    }
    double c2n = todbl(cnN), c2l = todbl(clN), c2nS = todbl(cnS), c2lS = todbl(clS);
    if (rg.blue) {
      for (int q = n + threadIdx.x; q < M; q += blockDim.x) buf[px<OpsDF>(q)] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    block_sum2(c2n, c2l, red);
    if (threadIdx.x == 0) {
      A.ring_part[2 * pr.x] = c2n;
      A.ring_part[2 * pr.x + 1] = c2l;
    }
    __syncthreads();
    if (two) {
      block_sum2(c2nS, c2lS, red);
      if (threadIdx.x == 0) {
        A.ring_part[2 * pr.y] = c2nS;
        A.ring_part[2 * pr.y + 1] = c2lS;
      }
    }
    if (threadIdx.x == 0 && !fresh) {  // after block_sum2's barrier: every gain of the pair is written
      T.gainlam[pr.x] = lam;
      if (two) T.gainlam[pr.y] = lam;
    }
    __syncthreads();
  } else {  // RING_ANALYSIS: u = the input maps
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
      if (p < n) {
        const float4 u = pack(mk(A.map_in[rg.off + p]), mk(two ? A.map_in[offS + p] : 0.0));
        buf[loc(p)] = rg.blue ? cmul(u, ch[p]) : u;
      } else if (rg.blue) {
        buf[px<OpsDF>(p)] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
  }

  if (rg.blue) bluestein4<OpsDF, 1>(buf, Mp, M, rg.logM, Bf, T.tw, A.logMmax);
  else fft_dit4<OpsDF, 1>(buf, Mp, M, rg.logM, -1, T.tw, A.logMmax);
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const int q = m % n, j = m / n, qn = q ? n - q : 0;
    const float4 Zq = rg.blue ? cmul(ch[q], buf[px<OpsDF>(q)]) : buf[px<OpsDF>(q)];
    const float4 Zn = rg.blue ? cmul(ch[qn], buf[px<OpsDF>(qn)]) : buf[px<OpsDF>(qn)];
    // U_N = (Z_q + conj Z_{n-q}) / 2, U_S = (Z_q - conj Z_{n-q}) / (2 i)
    float4 UN = pack(dadd(RE(Zq), RE(Zn)), dadd(IM(Zq), dneg(IM(Zn))));
    float4 US = pack(dadd(IM(Zq), IM(Zn)), dadd(RE(Zn), dneg(RE(Zq))));
    UN = make_float4(0.5f * UN.x, 0.5f * UN.y, 0.5f * UN.z, 0.5f * UN.w);
    US = make_float4(0.5f * US.x, 0.5f * US.y, 0.5f * US.z, 0.5f * US.w);
    if (rg.shifted) {
      UN = cmul(UN, cconj(hs[q]));
      US = cmul(US, cconj(hs[q]));
      if (j & 1) { UN = cneg(UN); US = cneg(US); }
    }
    const double om = A.omega;
    A.FT[(size_t)m * A.RP + k] = two ? make_double4_32a(om * todbl(RE(UN)), om * todbl(IM(UN)), om * todbl(RE(US)),
                                                      om * todbl(IM(US)))
                                     : make_double4_32a(om * todbl(RE(UN)), om * todbl(IM(UN)), 0.0, 0.0);
  }
}

// double -> double-float (hi, lo) per element
__global__ void to_df2_kernel(const double *src, float2 *dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dd v = mk(src[i]);
    dst[i] = make_float2(v.h, v.l);
  }
}

void launch_to_df2(const double *src, float2 *dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  to_df2_kernel<<<(int)blocks, 256, 0, s>>>(src, dst, n);
}

// double -> double-float table conversion
__global__ void to_df_kernel(const double2 *src, float4 *dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = pack(mk(v.x), mk(v.y));
  }
}

void launch_to_df(const double2 *src, float4 *dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  to_df_kernel<<<(int)blocks, 256, 0, s>>>(src, dst, n);
}

template <int MODE>
static void launch_ring_df_mode(const RingArgs &a, const RingDfArgs &t, const RingClass *cls, int ncls,
                                cudaStream_t s) {
  auto smem = [](const RingClass &c) { return c.global ? (size_t)16 : ((size_t)1 << c.logM) * sizeof(float4); };
  raise_smem_cap(reinterpret_cast<const void *>(ring_df_kernel<MODE>));
  for (int c = 0; c < ncls; ++c) {
    if (cls[c].count <= 0) continue;
    const size_t sm = smem(cls[c]);
    RingArgs ac = a;
    ac.first = cls[c].first;
    ac.scratch = cls[c].global ? a.scratch : nullptr;
    ring_df_kernel<MODE><<<cls[c].count, kRingDfThreads, sm, s>>>(ac, t);
  }
}

void launch_ring_df(const RingArgs &a, const RingDfArgs &t, const RingClass *cls, int ncls, cudaStream_t s,
                    int mode) {
  switch (mode) {
    case RING_SYNTH: launch_ring_df_mode<RING_SYNTH>(a, t, cls, ncls, s); break;
    case RING_ANALYSIS: launch_ring_df_mode<RING_ANALYSIS>(a, t, cls, ncls, s); break;
    default: launch_ring_df_mode<RING_ITER>(a, t, cls, ncls, s); break;
  }
}

}  // namespace wfk
