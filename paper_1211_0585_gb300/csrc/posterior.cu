// Posterior gradient of a solution (a diagnostic reported beside the
// iteration's own stop rule).
//
// The messenger iteration converges to the Wiener filter of the discretised
// problem only up to the quadrature error of the HEALPix analysis (the basis
// change of Sect. 2 is exact only for an orthogonal transform). How far a
// solution a is from the posterior mean (S^-1 + N^-1) s = N^-1 d (Eq. 2) on
// the grid is measured by the residual of its normal equations, with
// Y = synthesis, Y^T = map2alm / Omega and W = N^-1 (0 where masked):
//   r_lm = [Y^T W (d - Y a)]_lm - a_lm / C_l        (modes with C_l > 0)
//   b_lm = [Y^T W d]_lm
// reported as ||r|| / ||b|| with the m > 0 modes counted twice (real degrees
// of freedom), summed per m and then over m in a fixed order.
#include <cuda_runtime.h>

#include "wf_internal.h"

namespace wfk {

// ya: Y a on input, W (d - Y a) on output; wd: W d
__global__ void posterior_maps_kernel(const double *d, const double *w, double *ya, double *wd, long long npix) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const double wp = w[p];
    ya[p] = wp * (d[p] - ya[p]);
    wd[p] = wp * d[p];
  }
}

// part[2 m] = sum_l wgt |r_lm|^2, part[2 m + 1] = sum_l wgt |b_lm|^2 (one CTA per m)
__global__ void __launch_bounds__(256) posterior_norms_kernel(const double2 *a, const double2 *ta, const double2 *tb,
                                                              const double *cl, int lmax, double inv_omega,
                                                              double *part) {
  __shared__ double sh[2][256];
  const int m = blockIdx.x;
  const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
  const double wgt = m == 0 ? 1.0 : 2.0;
  double rr = 0.0, bb = 0.0;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    if (!(cl[l] > 0.0)) continue;
    const double2 av = a[base + l], t = ta[base + l], u = tb[base + l];
    const double rx = t.x * inv_omega - av.x / cl[l], ry = t.y * inv_omega - av.y / cl[l];
    const double bx = u.x * inv_omega, by = u.y * inv_omega;
    rr += wgt * (rx * rx + ry * ry);
    bb += wgt * (bx * bx + by * by);
  }
  sh[0][threadIdx.x] = rr;
  sh[1][threadIdx.x] = bb;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * m] = sh[0][0];
    part[2 * m + 1] = sh[1][0];
  }
}

void launch_posterior_maps(const double *d, const double *w, double *ya, double *wd, long long npix, cudaStream_t s) {
  long long blocks = (npix + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  posterior_maps_kernel<<<(int)blocks, 256, 0, s>>>(d, w, ya, wd, npix);
}

void launch_posterior_norms(const double2 *a, const double2 *ta, const double2 *tb, const double *cl, int lmax,
                            double inv_omega, double *part, cudaStream_t s) {
  posterior_norms_kernel<<<lmax + 1, 256, 0, s>>>(a, ta, tb, cl, lmax, inv_omega, part);
}

}  // namespace wfk
