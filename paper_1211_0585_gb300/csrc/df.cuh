// Double-float arithmetic helpers shared by the FP64-accurate kernels: a value
// is the unevaluated sum hi + lo of two floats (48 significant bits), and
// every operation is built from error-free transformations (two_sum,
// two_prod via fma).
#pragma once

#include <cuda_runtime.h>

namespace wfk {

struct dfl { float h, l; };

__device__ __forceinline__ dfl df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to(dfl a) { return (double)a.h + (double)a.l; }

// a + b (two_sum of the high parts, low parts added, renormalised)
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float r = s + e;
  return {r, e - (r - s)};
}

// a * b (two_prod of the high parts plus the cross terms, renormalised)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  const float r = p + e;
  return {r, e - (r - p)};
}

// S + C += a * b: compensated dot-product step (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005)
__device__ __forceinline__ void dot2_acc(float &S, float &C, dfl a, dfl b) {
  const float ph = a.h * b.h;
  const float pe = fmaf(a.h, b.h, -ph);
  const float pc = fmaf(a.h, b.l, a.l * b.h);
  const float s = S + ph;
  const float bb = s - S;
  const float e = (S - (s - bb)) + (ph - bb);
  S = s;
  C += e + (pe + pc);
}

// mu_l = (A x) mu1 - mu2 in double-float: one step of the rescaled Legendre
// recurrence mu_l = A_l x mu_{l-1} - mu_{l-2}
__device__ __forceinline__ dfl df_step(dfl A, dfl x, dfl mu1, dfl mu2) {
  const float ch = A.h * x.h;
  float ce = fmaf(A.h, x.h, -ch);
  ce = fmaf(A.h, x.l, fmaf(A.l, x.h, ce));
  const float qh = ch * mu1.h;
  float qe = fmaf(ch, mu1.h, -qh);
  qe = fmaf(ch, mu1.l, fmaf(ce, mu1.h, qe));
  const float sh = qh - mu2.h;
  const float bb = sh - qh;
  float e = (qh - (sh - bb)) + (-mu2.h - bb);
  e += qe - mu2.l;
  const float rh = sh + e;
  return {rh, e - (rh - sh)};
}

}  // namespace wfk
