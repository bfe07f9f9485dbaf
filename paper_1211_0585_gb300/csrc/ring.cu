// Ring stage of the HEALPix spherical harmonic transform pair, FP64.
//
// One CTA per ring. A ring of n pixels at azimuths phi_j = phi0 + 2 pi j / n
// (phi0 = pi / n for shifted rings, 0 otherwise) carries the Fourier
// coefficients F_m, m = 0 .. lsht, of the Legendre stage. Synthesis folds every
// frequency -lsht .. lsht onto its residue q = m mod n (m-aliasing on rings
// shorter than 2 lsht + 1) and applies an inverse DFT of length n; analysis is
// the forward DFT followed by the same unfolding:
//     f_j  = sum_q G_q e^{+2 pi i j q / n},  G_q = e^{i q phi0} sum_{m = q mod n} (-1)^{(m-q)/n [shifted]} F_m
//     T_m  = Omega e^{-i m phi0} sum_j u_j e^{-2 pi i j m / n}
// (Sect. 2: the basis change between pixel space and harmonic space, here its
// azimuthal half.) Power-of-two n use the in-place radix-4/2 FFT of fft.cuh
// in shared memory; other n (polar rings, n = 4i) use Bluestein's chirp-z
// convolution with a power-of-two size M >= 2n - 1, whose filter spectrum is
// precomputed per ring length.
//
// RING_ITER fuses the pixel-space half of one messenger iteration between the
// two transforms: s_p = f_p, r_p = d_p - s_p, the chi^2 partials of Sect. 3
// (sum w r^2 and sum w r^2 / (1 + (lambda - 1) tau w)) and the Eq. 3 increment
// u_p = t_p - s_p = a_p r_p with a_p = lambda tau w_p / (1 + (lambda - 1) tau w_p).
#include <cuda_runtime.h>

#include "fft.cuh"
#include "fold.cuh"
#include "wf_internal.h"

namespace wfk {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

// Deterministic block sum of two doubles (fixed tree); result valid in thread 0.
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

template <int MODE>
__global__ void __launch_bounds__(kRingThreads) ring_kernel(const RingArgs A) {
  extern __shared__ double2 smem[];
  const int r = A.order ? A.order[A.first + blockIdx.x] : A.first + blockIdx.x;
  const RingDev rg = A.rings[r];
  const int n = rg.n;
  const int M = 1 << rg.logM;
  const int Mp = M;
  // [Mp] (swizzled, px): shared memory, or this CTA's part of the global scratch
  double2 *buf = A.scratch ? reinterpret_cast<double2 *>(A.scratch) + (size_t)blockIdx.x * M : smem;
  double *ureal = reinterpret_cast<double *>(A.scratch ? smem : smem + Mp);  // [n]
  __shared__ double red[64];
  __shared__ double2 fold_part[kRingThreads];

  int L = A.lsht;
  double lam = 1.0;
  if (MODE != RING_ITER && A.gate && A.gate->done) return;
  if (MODE == RING_ITER) {
    if (A.ctl->done) return;
    L = A.ctl->lsht;
    lam = A.ctl->lambda;
  }
  const double2 *hs = A.hs + rg.hs_off;
  const double2 *ch = A.chirp + rg.ch_off;
  const double2 *Bf = A.B + rg.B_off;
  const int k = rg.pair;
  const int slot = rg.side;

  if (MODE == RING_SYNTH || MODE == RING_ITER) {
    // ---- fold F_m onto residues q (m-aliasing) with the half-pixel shift
    fold_ring(A.FS, A.RP, k, slot, rg.shifted, n, L, fold_part, [&](int q, double2 acc) {
      if (rg.shifted) acc = cmul(acc, hs[q]);
      // Bluestein: the inverse DFT via conj(DFT(conj(G)))
      buf[px<OpsF64>(q)] = rg.blue ? cmul(conjd(acc), ch[q]) : acc;
    });
    if (rg.blue) {
      for (int q = n + threadIdx.x; q < M; q += blockDim.x) buf[px<OpsF64>(q)] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (rg.blue) {
      bluestein4<OpsF64, 1>(buf, Mp, M, rg.logM, Bf, A.tw, A.logMmax);
    } else {
      fft_dif4<OpsF64, 1>(buf, Mp, M, rg.logM, +1, A.tw, A.logMmax);
    }
    // pixel values: Re of the inverse DFT
    if (MODE == RING_SYNTH) {
      for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const double f = rg.blue ? cmul(ch[p], buf[px<OpsF64>(p)]).x : buf[px<OpsF64>(digitrev(p, rg.logM))].x;
        A.map_out[rg.off + p] = f;
      }
      return;
    }
    // ---- RING_ITER: Eq. 3 per pixel and the chi^2 partials
    double c2n = 0.0, c2l = 0.0;
    const double lt = lam * A.tau, l1t = (lam - 1.0) * A.tau;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const double s = rg.blue ? cmul(ch[p], buf[px<OpsF64>(p)]).x : buf[px<OpsF64>(digitrev(p, rg.logM))].x;
      const double w = A.w[rg.off + p];
      const double res = A.d[rg.off + p] - s;
      const double wr2 = w * res * res;
      const double g = w / (1.0 + l1t * w);   // 1 / (sigma^2 + (lambda - 1) tau), 0 if masked
      c2n += wr2;
      c2l += g * res * res;
      ureal[p] = lt * g * res;                 // a_p (d_p - s_p)
    }
    block_sum2(c2n, c2l, red);
    if (threadIdx.x == 0) {
      A.ring_part[2 * r] = c2n;
      A.ring_part[2 * r + 1] = c2l;
    }
    __syncthreads();
  } else {
    for (int p = threadIdx.x; p < n; p += blockDim.x) ureal[p] = A.map_in[rg.off + p];
    __syncthreads();
  }

  // ---- forward DFT of the real ring values
  if (rg.blue) {
    for (int p = threadIdx.x; p < M; p += blockDim.x)
      buf[px<OpsF64>(p)] = p < n ? make_double2(ureal[p] * ch[p].x, ureal[p] * ch[p].y) : make_double2(0.0, 0.0);
    __syncthreads();
    bluestein4<OpsF64, 1>(buf, Mp, M, rg.logM, Bf, A.tw, A.logMmax);
  } else {
    for (int p = threadIdx.x; p < n; p += blockDim.x)
      buf[px<OpsF64>(digitrev(p, rg.logM))] = make_double2(ureal[p], 0.0);
    __syncthreads();
    fft_dit4<OpsF64, 1>(buf, Mp, M, rg.logM, -1, A.tw, A.logMmax);
  }
  // ---- unfold residues to m = 0 .. L, apply e^{-i m phi0} and Omega
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const int q = m % n, j = m / n;
    double2 U = rg.blue ? cmul(ch[q], buf[px<OpsF64>(q)]) : buf[px<OpsF64>(q)];
    if (rg.shifted) {
      U = cmul(U, conjd(hs[q]));
      if (j & 1) { U.x = -U.x; U.y = -U.y; }
    }
    double *dst = reinterpret_cast<double *>(A.FT + (size_t)m * A.RP + k) + 2 * slot;
    dst[0] = A.omega * U.x;
    dst[1] = A.omega * U.y;
  }
}

// Bluestein filter spectrum per ring length: b_q = conj(c_q) for |q| < n
// (wrapped into [0, M)), transformed by the DIF FFT (so stored digit-reversed)
// and scaled by 1/M. One CTA per ring of a class; only the first ring of each
// length (the north ring of a polar pair) writes. Classes whose buffers do not
// fit shared memory work in the global scratch, as the ring kernels do.
__global__ void __launch_bounds__(kRingThreads) bluestein_setup_kernel(const RingDev *rings, const int *order,
                                                                   int first, double2 *scratch,
                                                                   const double2 *tw, int logMmax,
                                                                   const double2 *chirp, double2 *B) {
  extern __shared__ double2 smem[];
  const RingDev rg = rings[order ? order[first + blockIdx.x] : first + blockIdx.x];
  if (!rg.blue || rg.side != 0) return;
  const int n = rg.n, M = 1 << rg.logM;
  double2 *buf = scratch ? scratch + (size_t)blockIdx.x * M : smem;
  const double2 *ch = chirp + rg.ch_off;
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (q < n) v = conjd(ch[q]);
    else if (q > M - n) v = conjd(ch[M - q]);
    buf[px<OpsF64>(q)] = v;
  }
  __syncthreads();
  fft_dif4<OpsF64, 1>(buf, M, M, rg.logM, -1, tw, logMmax);
  const double inv = 1.0 / (double)M;
  for (int q = threadIdx.x; q < M; q += blockDim.x)
    B[rg.B_off + q] = make_double2(buf[px<OpsF64>(q)].x * inv, buf[px<OpsF64>(q)].y * inv);
}

// Shared memory of a class: the FFT buffer plus the real ring values (n <= M).
static size_t ring_smem(const RingClass &c) {
  return (c.global ? 0 : ((size_t)1 << c.logM) * sizeof(double2)) + ((size_t)1 << c.logM) * sizeof(double);
}

template <int MODE>
static void launch_ring_mode(const RingArgs &a, const RingClass *cls, int ncls, cudaStream_t s) {
  raise_smem_cap(reinterpret_cast<const void *>(ring_kernel<MODE>));
  for (int c = 0; c < ncls; ++c) {
    if (cls[c].count <= 0) continue;
    const size_t sm = ring_smem(cls[c]);
    RingArgs ac = a;
    ac.first = cls[c].first;
    ac.scratch = cls[c].global ? a.scratch : nullptr;
    ring_kernel<MODE><<<cls[c].count, kRingThreads, sm, s>>>(ac);
  }
}

void launch_ring(const RingArgs &a, const RingClass *cls, int ncls, cudaStream_t s, int mode) {
  switch (mode) {
    case RING_SYNTH: launch_ring_mode<RING_SYNTH>(a, cls, ncls, s); break;
    case RING_ANALYSIS: launch_ring_mode<RING_ANALYSIS>(a, cls, ncls, s); break;
    default: launch_ring_mode<RING_ITER>(a, cls, ncls, s); break;
  }
}

void launch_bluestein_setup(const RingDev *rings, const int *order, const RingClass *cls, int ncls, void *scratch,
                            const double2 *tw, int logMmax, const double2 *chirp, double2 *B, cudaStream_t s) {
  raise_smem_cap(reinterpret_cast<const void *>(bluestein_setup_kernel));
  for (int c = 0; c < ncls; ++c) {
    if (cls[c].count <= 0) continue;
    const size_t sm = cls[c].global ? 0 : ((size_t)1 << cls[c].logM) * sizeof(double2);
    bluestein_setup_kernel<<<cls[c].count, kRingThreads, sm, s>>>(
        rings, order, cls[c].first, cls[c].global ? reinterpret_cast<double2 *>(scratch) : nullptr, tw, logMmax,
        chirp, B);
  }
}

}  // namespace wfk
