// Constrained realisations (Sect. 3, WMAP analysis: a Wiener-filter map plus
// a fluctuation map is a constrained realisation with the correct signal
// variance; the power-spectra figure).
//
//   s_CR,i = s_WF(d) + xi_i - s_WF(Y xi_i + n_i),   i = 0 .. nreal - 1,
//
// with xi_i ~ N(0, S) drawn as a_lm and n_i ~ N(0, N) drawn per observed
// pixel, both on the device. The nreal + 1 Wiener filters (d and the nreal
// fluctuation maps) run as one wf_solve_batch in the plan's precision, so on a
// mixed-precision plan they share the batched engine's steps.
//
// Random numbers: Philox4x64-10, the counter-based generator of Salmon,
// Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3",
// SC 2011): ten rounds on a 256-bit counter under a 128-bit key, each round
// two 64 x 64 -> 128-bit products (multipliers M0, M1) whose halves are
// mixed with the other words and the key, the key advanced by the Weyl
// constants W0, W1 between rounds. Every normal is a function of its index
// alone (no generator state), so any thread draws any entry:
//   key (seed, 0), counter (block j, kind, realisation i, 0);
//   kind 0: a_lm entry q takes the normals 2q (real part) and 2q + 1
//   (imaginary part), kind 1: pixel p takes normal p; normal 4j + w of a
//   block comes from its words by Box and Muller's transform,
//   u = ((x >> 11) + 1/2) 2^-53, r = sqrt(-2 ln u_{2t}), normals 4j + 2t and
//   4j + 2t + 1 = r cos(2 pi u_{2t+1}), r sin(2 pi u_{2t+1}).
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "wf_internal.h"
#include "wf_plan.h"

namespace wfk {
namespace {

constexpr unsigned long long kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
constexpr unsigned long long kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;

struct Block4 { unsigned long long x[4]; };

__device__ __forceinline__ Block4 philox4x64_10(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                                unsigned long long c3, unsigned long long k0, unsigned long long k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
    const unsigned long long hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  return Block4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ double uniform53(unsigned long long x) {
  return ((double)(x >> 11) + 0.5) * 0x1p-53;
}

// the Box-Muller pair t (0 or 1) of a block: (r cos, r sin)
__device__ __forceinline__ double2 box_muller(const Block4 &b, int t) {
  const double r = sqrt(-2.0 * log(uniform53(b.x[2 * t])));
  double sn, cs;
  sincospi(2.0 * uniform53(b.x[2 * t + 1]), &sn, &cs);
  return make_double2(r * cs, r * sn);
}

// xi ~ N(0, S): a_l0 = sqrt(C_l) z_re, a_lm = sqrt(C_l / 2) (z_re + i z_im) for m > 0; one CTA per m
__global__ void cr_signal_kernel(unsigned long long seed, int real_i, int lmax, const double *cl, double2 *xi) {
  const int m = blockIdx.x;
  const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const unsigned long long q = base + l;
    const Block4 b = philox4x64_10(q >> 1, 0ull, (unsigned long long)real_i, 0ull, seed, 0ull);
    const double2 z = box_muller(b, (int)(q & 1));
    const double c = cl[l] > 0.0 ? cl[l] : 0.0;
    xi[q] = (m == 0) ? make_double2(sqrt(c) * z.x, 0.0) : make_double2(sqrt(0.5 * c) * z.x, sqrt(0.5 * c) * z.y);
  }
}

// map += n, n_p = sigma_p z_p on observed pixels (w_p = 1 / sigma_p^2 > 0), 0 where masked; one thread per block
__global__ void cr_noise_kernel(unsigned long long seed, int real_i, long long npix, const double *w, double *map) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * j >= npix) return;
  const Block4 b = philox4x64_10((unsigned long long)j, 1ull, (unsigned long long)real_i, 0ull, seed, 0ull);
  const double2 z01 = box_muller(b, 0), z23 = box_muller(b, 1);
  const double z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long long p = 4 * j + k;
    if (p < npix && w[p] > 0.0) map[p] += z[k] / sqrt(w[p]);
  }
}

// cr_i = wf + xi_i - sol_i
__global__ void cr_combine_kernel(long long nalm, int nreal, const double2 *wf, const double2 *xi, const double2 *sol,
                                  double2 *cr) {
  const long long n = nalm * nreal;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long q = t % nalm;
    const double2 a = wf[q], x = xi[t], s = sol[t];
    cr[t] = make_double2(a.x + x.x - s.x, a.y + x.y - s.y);
  }
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace
}  // namespace wfk

using namespace wfk;

#define CR_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

extern "C" wf_status wf_constrained_realisations(wf_plan_t plan, int nreal, uint64_t seed, const double *d,
                                                 int d_on_device, double *cr_out, int out_on_device,
                                                 double *wf_out, wf_stats *stats) {
  if (!plan || !d || !cr_out || nreal < 1) {
    set_error("wf_constrained_realisations: NULL argument or nreal < 1");
    return WF_EINVAL;
  }
  Plan *P = static_cast<Plan *>(plan);
  const long long npix = P->npix, nalm = P->nalm;
  const int lmax = P->lmax;
  cudaStream_t s = P->run_stream();
  DevBuf D, X, SOL, OUT;
  CR_CUDA(cudaMalloc(&D.p, sizeof(double) * npix * (nreal + 1)));
  CR_CUDA(cudaMalloc(&X.p, sizeof(double2) * nalm * nreal));
  CR_CUDA(cudaMalloc(&SOL.p, sizeof(double2) * nalm * (nreal + 1)));
  CR_CUDA(cudaMalloc(&OUT.p, sizeof(double2) * nalm * nreal));
  double *dd = static_cast<double *>(D.p);
  double2 *xi = static_cast<double2 *>(X.p), *sol = static_cast<double2 *>(SOL.p), *cr = static_cast<double2 *>(OUT.p);
  CR_CUDA(cudaMemcpyAsync(dd, d, sizeof(double) * npix, d_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s));
  // the fluctuation data Y xi_i + n_i
  for (int i = 0; i < nreal; ++i) {
    cr_signal_kernel<<<lmax + 1, 128, 0, s>>>((unsigned long long)seed, i, lmax, P->d_cl, xi + (size_t)i * nalm);
    wf_status st = wf_alm2map(plan, lmax, reinterpret_cast<const double *>(xi + (size_t)i * nalm),
                              dd + (size_t)(i + 1) * npix);
    if (st) return st;
    const long long nblk = (npix + 3) / 4;
    cr_noise_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>((unsigned long long)seed, i, npix, P->d_w,
                                                                  dd + (size_t)(i + 1) * npix);
  }
  CR_CUDA(cudaGetLastError());
  // every Wiener filter in one batch: d first, then the fluctuation maps
  const wf_status sst = wf_solve_batch(plan, nreal + 1, dd, 1, reinterpret_cast<double *>(sol), 1, stats);
  if (sst != WF_OK && sst != WF_ENOTCONVERGED) return sst;
  cr_combine_kernel<<<1024, 256, 0, s>>>(nalm, nreal, sol, xi, sol + nalm, cr);
  CR_CUDA(cudaGetLastError());
  const auto kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CR_CUDA(cudaMemcpyAsync(cr_out, cr, sizeof(double2) * nalm * nreal, kind, s));
  if (wf_out) CR_CUDA(cudaMemcpyAsync(wf_out, sol, sizeof(double2) * nalm, kind, s));
  CR_CUDA(cudaStreamSynchronize(s));
  return sst;
}
