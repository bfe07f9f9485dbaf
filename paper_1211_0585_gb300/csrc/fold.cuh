// Folding of a ring's azimuthal Fourier coefficients onto the residues of its
// DFT (m-aliasing): for a ring of n pixels,
//   G_q = sum_{j >= 0} s^j F_{q + n j} + sum_{j >= 1} s^j conj(F_{n j - q}),
// m <= L, with s = -1 on rings whose first pixel sits half a pixel off
// (the phase e^{i m phi0} changes sign with each alias) and s = 1 otherwise.
// On rings shorter than the thread block, each residue's alias series is split
// over several threads and their partial sums are added in a fixed order.
#pragma once

#include <cuda_runtime.h>

#include "wf_internal.h"

namespace wfk {

// The share j = j0, j0 + dj, ... of residue q's series, from F stored as
// double4_32a (north re, north im, south re, south im) at [m RP + k].
__device__ __forceinline__ double2 fold_alias_sum(const double4_32a *FS, int RP, int k, int slot, int shifted,
                                                  int n, int q, int L, int j0, int dj) {
  double ar = 0.0, ai = 0.0;
  for (int j = j0, m = q + n * j0; m <= L; j += dj, m += n * dj) {
    const double4_32a f4 = FS[(size_t)m * RP + k];
    double fr = slot ? f4.z : f4.x, fi = slot ? f4.w : f4.y;
    if (shifted && (j & 1)) { fr = -fr; fi = -fi; }
    ar += fr; ai += fi;
  }
  for (int j = 1 + j0, m = n * (1 + j0) - q; m <= L; j += dj, m += n * dj) {
    const double4_32a f4 = FS[(size_t)m * RP + k];
    double fr = slot ? f4.z : f4.x, fi = slot ? -f4.w : -f4.y;
    if (shifted && (j & 1)) { fr = -fr; fi = -fi; }
    ar += fr; ai += fi;
  }
  return make_double2(ar, ai);
}

// Both slots' shares at once (north in .x/.y, south in .z/.w), each F record
// read once.
__device__ __forceinline__ double4_16a fold_alias_sum2(const double4_32a *FS, int RP, int k, int shifted, int n, int q,
                                                   int L, int j0, int dj) {
  double4_16a a = make_double4_16a(0.0, 0.0, 0.0, 0.0);
  for (int j = j0, m = q + n * j0; m <= L; j += dj, m += n * dj) {
    const double4_32a f4 = FS[(size_t)m * RP + k];
    const double sg = (shifted && (j & 1)) ? -1.0 : 1.0;
    a.x += sg * f4.x; a.y += sg * f4.y; a.z += sg * f4.z; a.w += sg * f4.w;
  }
  for (int j = 1 + j0, m = n * (1 + j0) - q; m <= L; j += dj, m += n * dj) {
    const double4_32a f4 = FS[(size_t)m * RP + k];
    const double sg = (shifted && (j & 1)) ? -1.0 : 1.0;
    a.x += sg * f4.x; a.y -= sg * f4.y; a.z += sg * f4.z; a.w -= sg * f4.w;
  }
  return a;
}

// fold_ring for both rings of a pair: store(q, G_q north, G_q south).
// part: shared scratch of blockDim.x double4_16a.
template <class Store>
__device__ __forceinline__ void fold_ring2(const double4_32a *FS, int RP, int k, int shifted, int n, int L,
                                           double4_16a *part, Store store) {
  const int nt = blockDim.x;
  if (n >= nt) {
    for (int q = threadIdx.x; q < n; q += nt) {
      const double4_16a g = fold_alias_sum2(FS, RP, k, shifted, n, q, L, 0, 1);
      store(q, make_double2(g.x, g.y), make_double2(g.z, g.w));
    }
    return;
  }
  const int nj = nt / n, t = threadIdx.x;
  if (t < n * nj) part[t] = fold_alias_sum2(FS, RP, k, shifted, n, t % n, L, t / n, nj);
  __syncthreads();
  if (t < n) {
    double4_16a g = make_double4_16a(0.0, 0.0, 0.0, 0.0);
    for (int jg = 0; jg < nj; ++jg) {
      const double4_16a p = part[jg * n + t];
      g.x += p.x; g.y += p.y; g.z += p.z; g.w += p.w;
    }
    store(t, make_double2(g.x, g.y), make_double2(g.z, g.w));
  }
}

// G_q for every residue, passed to store(q, G_q) by one thread each.
// part: shared scratch of blockDim.x double2. Contains a __syncthreads when
// the ring is shorter than the block (uniform over the CTA).
template <class Store>
__device__ __forceinline__ void fold_ring(const double4_32a *FS, int RP, int k, int slot, int shifted, int n, int L,
                                          double2 *part, Store store) {
  const int nt = blockDim.x;
  if (n >= nt) {
    for (int q = threadIdx.x; q < n; q += nt) store(q, fold_alias_sum(FS, RP, k, slot, shifted, n, q, L, 0, 1));
    return;
  }
  const int nj = nt / n, t = threadIdx.x;
  if (t < n * nj) part[t] = fold_alias_sum(FS, RP, k, slot, shifted, n, t % n, L, t / n, nj);
  __syncthreads();
  if (t < n) {
    double2 g = make_double2(0.0, 0.0);
    for (int jg = 0; jg < nj; ++jg) {
      g.x += part[jg * n + t].x;
      g.y += part[jg * n + t].y;
    }
    store(t, g);
  }
}

}  // namespace wfk
