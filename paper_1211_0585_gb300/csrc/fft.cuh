// In-place mixed radix-4 / radix-2 FFTs in shared memory, shared by the ring
// kernels of every precision.
//
//   dif: natural order in, digit-reversed order out (radix 4 stages from the
//        full length down, then one radix-2 stage when log2 M is odd);
//   dit: digit-reversed order in, natural order out (the mirror image).
// sign < 0 computes sum_j x_j e^{-2 pi i jk/M}, sign > 0 the e^{+...} sum
// (unnormalised). dit(+1)(dif(-1)(a) * dif(-1)(b)) = M * (a circularly
// convolved with b), which is how the Bluestein convolution uses them.
//
// G arrays of length M laid out one after another share every twiddle load
// (G slots of the batched engine); tw[k] = e^{-2 pi i k / Mmax}, k < Mmax.
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

// Arithmetic policies: complex type T, twiddle table type W.
struct OpsF64 {
  using T = double2;
  using W = double2;
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

struct OpsF32 {  // float complex; twiddles read from a double-float table (hi parts)
  using T = float2;
  using W = float4;
  static __device__ __forceinline__ T add(T a, T b) { return make_float2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ T sub(T a, T b) { return make_float2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ T mul(T a, T b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ T muli(T a, int sign) {
    return sign < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  }
  static __device__ __forceinline__ T tw(const W *t, int idx, int sign) {
    const float4 w = t[idx];
    return make_float2(w.x, sign > 0 ? -w.z : w.z);
  }
};

struct OpsDF {  // double-float complex: float4 (re hi, re lo, im hi, im lo)
  using T = float4;
  using W = float4;
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

template <class O, int G>
__device__ void fft_dif4(typename O::T *buf, int M, int logM, int sign, const typename O::W *tw, int logMmax) {
  using T = typename O::T;
  int s = logM;
  for (; s >= 2; s -= 2) {
    const int qsh = s - 2, Q = 1 << qsh;
    const int tsh = logMmax - s;
    for (int t = threadIdx.x; t < (M >> 2); t += blockDim.x) {
      const int i = t & (Q - 1);
      const int base = ((t >> qsh) << s) + i;
      const T w1 = O::tw(tw, i << tsh, sign);
      const T w2 = O::tw(tw, (2 * i) << tsh, sign);
      const T w3 = O::tw(tw, (3 * i) << tsh, sign);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        T *x = buf + g * M + base;
        const T a0 = x[0], a1 = x[Q], a2 = x[2 * Q], a3 = x[3 * Q];
        const T t0 = O::add(a0, a2), t1 = O::sub(a0, a2);
        const T t2 = O::add(a1, a3), t3 = O::muli(O::sub(a1, a3), sign);
        x[0] = O::add(t0, t2);
        x[Q] = O::mul(O::add(t1, t3), w1);
        x[2 * Q] = O::mul(O::sub(t0, t2), w2);
        x[3 * Q] = O::mul(O::sub(t1, t3), w3);
      }
    }
    __syncthreads();
  }
  if (s == 1) {
    for (int t = threadIdx.x; t < (M >> 1); t += blockDim.x) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        T *x = buf + g * M + 2 * t;
        const T a = x[0], b = x[1];
        x[0] = O::add(a, b);
        x[1] = O::sub(a, b);
      }
    }
    __syncthreads();
  }
}

template <class O, int G>
__device__ void fft_dit4(typename O::T *buf, int M, int logM, int sign, const typename O::W *tw, int logMmax) {
  using T = typename O::T;
  int s = 0;
  if (logM & 1) {
    for (int t = threadIdx.x; t < (M >> 1); t += blockDim.x) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        T *x = buf + g * M + 2 * t;
        const T a = x[0], b = x[1];
        x[0] = O::add(a, b);
        x[1] = O::sub(a, b);
      }
    }
    __syncthreads();
    s = 1;
  }
  for (s += 2; s <= logM; s += 2) {
    const int qsh = s - 2, Q = 1 << qsh;
    const int tsh = logMmax - s;
    for (int t = threadIdx.x; t < (M >> 2); t += blockDim.x) {
      const int i = t & (Q - 1);
      const int base = ((t >> qsh) << s) + i;
      const T w1 = O::tw(tw, i << tsh, sign);
      const T w2 = O::tw(tw, (2 * i) << tsh, sign);
      const T w3 = O::tw(tw, (3 * i) << tsh, sign);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        T *x = buf + g * M + base;
        const T a0 = x[0], a1 = O::mul(x[Q], w1), a2 = O::mul(x[2 * Q], w2), a3 = O::mul(x[3 * Q], w3);
        const T t0 = O::add(a0, a2), t1 = O::sub(a0, a2);
        const T t2 = O::add(a1, a3), t3 = O::muli(O::sub(a1, a3), sign);
        x[0] = O::add(t0, t2);
        x[Q] = O::add(t1, t3);
        x[2 * Q] = O::sub(t0, t2);
        x[3 * Q] = O::sub(t1, t3);
      }
    }
    __syncthreads();
  }
}

// Bluestein core for G arrays: on entry buf holds x_j c_j (zero-padded to M);
// on exit buf[k] (natural order) = M^-1-scaled circular convolution with the
// chirp filter whose dif(-1) spectrum (digit-reversed, / M) is Bf.
template <class O, int G>
__device__ void bluestein4(typename O::T *buf, int M, int logM, const typename O::W *Bf, const typename O::W *tw,
                           int logMmax) {
  fft_dif4<O, G>(buf, M, logM, -1, tw, logMmax);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const typename O::T f = O::tw(Bf, i, -1);
#pragma unroll
    for (int g = 0; g < G; ++g) buf[g * M + i] = O::mul(buf[g * M + i], f);
  }
  __syncthreads();
  fft_dit4<O, G>(buf, M, logM, +1, tw, logMmax);
}

}  // namespace wfk
