// In-place power-of-two FFTs in shared memory, shared by the ring kernels of
// every precision.
//
//   dif: natural order in, digit-reversed order out (radix-4 stages from the
//        full length down, then one radix-2 stage when log2 M is odd);
//   dit: digit-reversed order in, natural order out (the mirror image).
// sign < 0 computes sum_j x_j e^{-2 pi i jk/M}, sign > 0 the e^{+...} sum
// (unnormalised). dit(+1)(dif(-1)(a) * dif(-1)(b)) = M * (a circularly
// convolved with b), which is how the Bluestein convolution uses them.
//
// Policies with kR16 run two consecutive radix-4 stages per shared-memory
// pass (a radix-16 pass: 16 values in registers per thread), which halves the
// passes and barriers; the stage arithmetic and the output order are those of
// the radix-4 stages it replaces.
//
// Shared-memory layout: element e of an array sits at px(e) = e XOR f(e),
// where f folds every higher group of kSw bits of e onto the low kSw bits
// (2^kSw elements fill the 128 bytes of the 32 banks: 16 of 8 bytes, 8 of
// 16 bytes). The map is a bijection, linear over XOR, and it spreads both
// the strided accesses of every butterfly stage (down to the stride-1 stage
// where a thread owns consecutive elements) and the digit-reversed accesses
// of the pixel pass over distinct banks. G arrays of length M lie one after
// another (stride Mp) and share every twiddle load.
// tw[k] = e^{-2 pi i k / Mmax}, k < Mmax.
#pragma once

#include <cuda_runtime.h>

namespace wfk {

// position of frequency (or time index) k in the digit-reversed order
__device__ __forceinline__ int digitrev(int k, int logM) {
  int pos = 0, rem = logM;
  for (int s = 0; s < (logM >> 1); ++s) {
    rem -= 2;
    pos |= (k & 3) << rem;
    k >>= 2;
  }
  if (logM & 1) pos |= (k & 1) << (rem - 1);
  return pos;
}

// Arithmetic policies: complex type T, twiddle table type W, swizzle width kSw.
struct OpsF64 {
  using T = double2;
  using W = double2;
  static constexpr int kSw = 3;
  static constexpr bool kR16 = false;
  static __device__ __forceinline__ T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ T sub(T a, T b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ T mul(T a, T b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ T muli(T a, int sign) {  // a * (sign i)
    return sign < 0 ? make_double2(a.y, -a.x) : make_double2(-a.y, a.x);
  }
  static __device__ __forceinline__ T tw(const W *t, int idx, int sign) {
    double2 w = t[idx];
    if (sign > 0) w.y = -w.y;
    return w;
  }
};

struct OpsF32 {  // float complex; twiddles from a float table
  using T = float2;
  using W = float2;
  static constexpr int kSw = 4;
  static constexpr bool kR16 = true;
  static __device__ __forceinline__ T add(T a, T b) { return make_float2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ T sub(T a, T b) { return make_float2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ T mul(T a, T b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ T muli(T a, int sign) {
    return sign < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  }
  static __device__ __forceinline__ T tw(const W *t, int idx, int sign) {
    const float2 w = t[idx];
    return make_float2(w.x, sign > 0 ? -w.y : w.y);
  }
  // e^{sign 2 pi i m / 16}, m = 0 .. 15 (m a compile-time constant after unrolling)
  static __device__ __forceinline__ T w16(int m, int sign) {
    constexpr float c[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                             0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
    const float sn = c[(m + 12) & 15];   // sin(2 pi m / 16) = cos(2 pi (m - 4) / 16)
    return make_float2(c[m & 15], sign < 0 ? -sn : sn);
  }
};

struct OpsDF {  // double-float complex: float4 (re hi, re lo, im hi, im lo)
  using T = float4;
  using W = float4;
  static constexpr int kSw = 3;
  static constexpr bool kR16 = false;
  static __device__ __forceinline__ float2 dadd(float ah, float al, float bh, float bl) {
    const float s = ah + bh;
    const float bb = s - ah;
    float e = (ah - (s - bb)) + (bh - bb);
    e += al + bl;
    const float r = s + e;
    return make_float2(r, e - (r - s));
  }
  static __device__ __forceinline__ float2 dmul(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    const float r = p + e;
    return make_float2(r, e - (r - p));
  }
  static __device__ __forceinline__ T add(T a, T b) {
    const float2 re = dadd(a.x, a.y, b.x, b.y), im = dadd(a.z, a.w, b.z, b.w);
    return make_float4(re.x, re.y, im.x, im.y);
  }
  static __device__ __forceinline__ T sub(T a, T b) {
    const float2 re = dadd(a.x, a.y, -b.x, -b.y), im = dadd(a.z, a.w, -b.z, -b.w);
    return make_float4(re.x, re.y, im.x, im.y);
  }
  static __device__ __forceinline__ T mul(T a, T b) {
    const float2 rr = dmul(a.x, a.y, b.x, b.y), ii = dmul(a.z, a.w, b.z, b.w);
    const float2 ri = dmul(a.x, a.y, b.z, b.w), ir = dmul(a.z, a.w, b.x, b.y);
    const float2 re = dadd(rr.x, rr.y, -ii.x, -ii.y), im = dadd(ri.x, ri.y, ir.x, ir.y);
    return make_float4(re.x, re.y, im.x, im.y);
  }
  static __device__ __forceinline__ T muli(T a, int sign) {
    return sign < 0 ? make_float4(a.z, a.w, -a.x, -a.y) : make_float4(-a.z, -a.w, a.x, a.y);
  }
  static __device__ __forceinline__ T tw(const W *t, int idx, int sign) {
    const float4 w = t[idx];
    return sign > 0 ? make_float4(w.x, w.y, -w.z, -w.w) : w;
  }
};

// swizzled position of element e (e < 2^15)
template <class O>
__device__ __forceinline__ int px(int e) {
  constexpr int k = O::kSw, m = (1 << k) - 1;
  int f = (e >> k) ^ (e >> (2 * k)) ^ (e >> (3 * k));
  if (k < 4) f ^= e >> (4 * k);
  return e ^ (f & m);
}

// radix-4 butterfly: (a0, a1, a2, a3) <- (t0 + t2, t1 + t3, t0 - t2, t1 - t3)
template <class O>
__device__ __forceinline__ void bfly4(typename O::T &a0, typename O::T &a1, typename O::T &a2, typename O::T &a3,
                                      int sign) {
  using T = typename O::T;
  const T t0 = O::add(a0, a2), t1 = O::sub(a0, a2);
  const T t2 = O::add(a1, a3), t3 = O::muli(O::sub(a1, a3), sign);
  a0 = O::add(t0, t2);
  a1 = O::add(t1, t3);
  a2 = O::sub(t0, t2);
  a3 = O::sub(t1, t3);
}

// one radix-4 DIF (DIT) stage on sub-transforms of size 2^s, every array
template <class O, int G, bool DIT>
__device__ void stage4(typename O::T *buf, int Mp, int M, int s, int sign, const typename O::W *tw, int logMmax) {
  using T = typename O::T;
  const int qsh = s - 2, Q = 1 << qsh;
  const int tsh = logMmax - s;
  for (int t = threadIdx.x; t < (M >> 2); t += blockDim.x) {
    const int i = t & (Q - 1);
    const int base = ((t >> qsh) << s) + i;
    const T w1 = O::tw(tw, i << tsh, sign);
    const T w2 = O::tw(tw, (2 * i) << tsh, sign);
    const T w3 = O::tw(tw, (3 * i) << tsh, sign);
    // base and j Q have disjoint bits, so px(base + j Q) = px(base) ^ px(j Q)
    const int p0 = px<O>(base), q1 = px<O>(Q), q2 = px<O>(2 * Q);
    const int p1 = p0 ^ q1, p2 = p0 ^ q2, p3 = p0 ^ q1 ^ q2;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      T *x = buf + g * Mp;
      T a0 = x[p0], a1 = x[p1], a2 = x[p2], a3 = x[p3];
      if (DIT) { a1 = O::mul(a1, w1); a2 = O::mul(a2, w2); a3 = O::mul(a3, w3); }
      bfly4<O>(a0, a1, a2, a3, sign);
      if (!DIT) { a1 = O::mul(a1, w1); a2 = O::mul(a2, w2); a3 = O::mul(a3, w3); }
      x[p0] = a0; x[p1] = a1; x[p2] = a2; x[p3] = a3;
    }
  }
  __syncthreads();
}

// radix-2 stage on adjacent pairs (the odd stage of an odd log2 M)
template <class O, int G>
__device__ void stage2(typename O::T *buf, int Mp, int M) {
  using T = typename O::T;
  for (int t = threadIdx.x; t < (M >> 1); t += blockDim.x) {
    const int p0 = px<O>(2 * t), p1 = px<O>(2 * t + 1);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      T *x = buf + g * Mp;
      const T a = x[p0], b = x[p1];
      x[p0] = O::add(a, b);
      x[p1] = O::sub(a, b);
    }
  }
  __syncthreads();
}

// Radix-16 pass: the radix-4 stages at sizes 2^s (stride 4Q, "A") and 2^(s-2)
// (stride Q, "B") on 16 values v[j] = x[base + j Q] held in registers.
// Stage A pairs v[r + 4c] (c = 0..3) at position r Q + i of its 4Q block, with
// twiddles W_{16Q}^{(rQ + i) c} = W_{16Q}^{i c} W_16^{r c}; stage B pairs
// v[4c + j] (j = 0..3) at position i, with twiddles W_{4Q}^{i j}. DIF runs A
// then B (twiddles after the butterflies), DIT runs B then A (before).
template <class O, bool DIT>
__device__ __forceinline__ void pass16_body(typename O::T (&v)[16], int i, int s, int sign, const typename O::W *tw,
                                            int logMmax) {
  using T = typename O::T;
  const int tshA = logMmax - s, tshB = tshA + 2;
  T a[4], b[4];
#pragma unroll
  for (int c = 1; c < 4; ++c) {
    a[c] = O::tw(tw, (i * c) << tshA, sign);
    b[c] = O::tw(tw, (i * c) << tshB, sign);
  }
  auto stageA = [&](bool pre) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      T w[4];
#pragma unroll
      for (int c = 1; c < 4; ++c) w[c] = r == 0 ? a[c] : O::mul(a[c], O::w16(r * c, sign));
      if (pre) {
#pragma unroll
        for (int c = 1; c < 4; ++c) v[r + 4 * c] = O::mul(v[r + 4 * c], w[c]);
      }
      bfly4<O>(v[r], v[r + 4], v[r + 8], v[r + 12], sign);
      if (!pre) {
#pragma unroll
        for (int c = 1; c < 4; ++c) v[r + 4 * c] = O::mul(v[r + 4 * c], w[c]);
      }
    }
  };
  auto stageB = [&](bool pre) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (pre) {
#pragma unroll
        for (int j = 1; j < 4; ++j) v[4 * c + j] = O::mul(v[4 * c + j], b[j]);
      }
      bfly4<O>(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3], sign);
      if (!pre) {
#pragma unroll
        for (int j = 1; j < 4; ++j) v[4 * c + j] = O::mul(v[4 * c + j], b[j]);
      }
    }
  };
  if (!DIT) { stageA(false); stageB(false); }
  else { stageB(true); stageA(true); }
}

template <class O, int G, bool DIT>
__device__ void pass16(typename O::T *buf, int Mp, int M, int logM, int s, int sign, const typename O::W *tw,
                       int logMmax) {
  using T = typename O::T;
  const int qsh = s - 4, Q = 1 << qsh;
  const int ngrp = M >> 4;
  for (int t = threadIdx.x; t < G * ngrp; t += blockDim.x) {
    const int g = t >> (logM - 4), tt = t & (ngrp - 1);
    const int i = tt & (Q - 1);
    const int base = ((tt >> qsh) << s) + i;
    T *x = buf + g * Mp;
    // base and j Q have disjoint bits: px(base + j Q) = px(base) ^ (XOR of px(2^b Q) over the bits b of j)
    const int pb = px<O>(base);
    int qb[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) qb[b] = px<O>(Q << b);
    int pj[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      pj[j] = pb ^ ((j & 1) ? qb[0] : 0) ^ ((j & 2) ? qb[1] : 0) ^ ((j & 4) ? qb[2] : 0) ^ ((j & 8) ? qb[3] : 0);
    T v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = x[pj[j]];
    pass16_body<O, DIT>(v, i, s, sign, tw, logMmax);
#pragma unroll
    for (int j = 0; j < 16; ++j) x[pj[j]] = v[j];
  }
  __syncthreads();
}

// Radix-8 pass: the radix-4 stage at size 8 (stride 2; twiddles W_8^{ik},
// constants) and the radix-2 stage on 8 consecutive values in registers (the
// last two stages of an odd log2 M). DIF runs the radix-4 stage first.
template <class O, int G, bool DIT>
__device__ void pass8(typename O::T *buf, int Mp, int M, int logM, int sign) {
  using T = typename O::T;
  const int ngrp = M >> 3;
  for (int t = threadIdx.x; t < G * ngrp; t += blockDim.x) {
    const int g = t >> (logM - 3), tt = t & (ngrp - 1);
    T *x = buf + g * Mp;
    const int pb = px<O>(tt << 3);   // tt << 3 and j < 8 have disjoint bits
    int pj[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) pj[j] = pb ^ px<O>(j);
    T v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = x[pj[j]];
    auto radix2 = [&]() {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T a0 = v[2 * c], a1 = v[2 * c + 1];
        v[2 * c] = O::add(a0, a1);
        v[2 * c + 1] = O::sub(a0, a1);
      }
    };
    auto radix4 = [&](bool pre) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (pre && i == 1) {
#pragma unroll
          for (int k = 1; k < 4; ++k) v[i + 2 * k] = O::mul(v[i + 2 * k], O::w16(2 * k, sign));
        }
        bfly4<O>(v[i], v[i + 2], v[i + 4], v[i + 6], sign);
        if (!pre && i == 1) {
#pragma unroll
          for (int k = 1; k < 4; ++k) v[i + 2 * k] = O::mul(v[i + 2 * k], O::w16(2 * k, sign));
        }
      }
    };
    if (!DIT) { radix4(false); radix2(); }
    else { radix2(); radix4(true); }
#pragma unroll
    for (int j = 0; j < 8; ++j) x[pj[j]] = v[j];
  }
  __syncthreads();
}

template <class O, int G>
__device__ void fft_dif4(typename O::T *buf, int Mp, int M, int logM, int sign, const typename O::W *tw,
                         int logMmax) {
  int s = logM;
  if constexpr (O::kR16) {
    for (; s >= 4; s -= 4) pass16<O, G, false>(buf, Mp, M, logM, s, sign, tw, logMmax);
    if (s == 3) { pass8<O, G, false>(buf, Mp, M, logM, sign); return; }
  }
  for (; s >= 2; s -= 2) stage4<O, G, false>(buf, Mp, M, s, sign, tw, logMmax);
  if (s == 1) stage2<O, G>(buf, Mp, M);
}

template <class O, int G>
__device__ void fft_dit4(typename O::T *buf, int Mp, int M, int logM, int sign, const typename O::W *tw,
                         int logMmax) {
  // the mirror of fft_dif4: the passes it ran last run first
  if constexpr (O::kR16) {
    int s = logM & 3;                                  // stages below the radix-16 passes
    if (s == 3) pass8<O, G, true>(buf, Mp, M, logM, sign);
    else if (s == 2) stage4<O, G, true>(buf, Mp, M, 2, sign, tw, logMmax);
    else if (s == 1) stage2<O, G>(buf, Mp, M);
    for (s += 4; s <= logM; s += 4) pass16<O, G, true>(buf, Mp, M, logM, s, sign, tw, logMmax);
  } else {
    int s = 0;
    if (logM & 1) { stage2<O, G>(buf, Mp, M); s = 1; }
    for (s += 2; s <= logM; s += 2) stage4<O, G, true>(buf, Mp, M, s, sign, tw, logMmax);
  }
}

// Bluestein core for G arrays: on entry buf holds x_j c_j (zero-padded to M);
// on exit buf[k] (natural order) = M^-1-scaled circular convolution with the
// chirp filter whose dif(-1) spectrum (digit-reversed, / M) is Bf.
template <class O, int G>
__device__ void bluestein4(typename O::T *buf, int Mp, int M, int logM, const typename O::W *Bf,
                           const typename O::W *tw, int logMmax) {
  fft_dif4<O, G>(buf, Mp, M, logM, -1, tw, logMmax);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const typename O::T f = O::tw(Bf, i, -1);
    const int p = px<O>(i);
#pragma unroll
    for (int g = 0; g < G; ++g) buf[g * Mp + p] = O::mul(buf[g * Mp + p], f);
  }
  __syncthreads();
  fft_dit4<O, G>(buf, Mp, M, logM, +1, tw, logMmax);
}

}  // namespace wfk
