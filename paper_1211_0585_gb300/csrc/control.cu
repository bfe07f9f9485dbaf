// Device-resident iteration controller (Sect. 3 of the paper).
//
// Runs as the last kernel of every iteration: reduces the per-ring and per-m
// partial sums in a fixed order (bitwise reproducible), writes the
// iteration's record, and advances the schedule:
//   chi^2 = s^+ S^-1 s + (d - s)^+ N^-1 (d - s) of the iteration's input state;
//   while lambda > 1: after a chi^2 plateau (|chi2_k - chi2_{k-1}| below
//     plateau_eps * sigma_chi2, sigma_chi2 = sqrt(2 n_obs), both iterates of the
//     same level) double l_iter and lower lambda to C_{l_iter} / (tau Omega)
//     (clamped to >= 1; 1 once l_iter > lmax), band limit
//     lmax_SHT = min(lmax, l_iter + margin);
//   at lambda = 1 (band limit lmax): stop when the relative increment
//     ||s_k - s_{k-1}|| / ||s_k|| <= tol, or, if enabled, when
//     |Delta chi^2| < final_dchi2 * sigma_chi2 (the paper's rule, 1e-4).
// Keeping the controller on the device lets a whole block of iterations run
// as one CUDA graph with no host round trip.
#include <cuda_runtime.h>

#include "ctl.cuh"
#include "wf_internal.h"

namespace wfk {

__global__ void __launch_bounds__(256) control_kernel(Ctl *c, const double *ring_part, int R,
                                                      const double *m_part, int lmax, const double *cl,
                                                      wf_iter_record *hist, int hist_cap) {
  __shared__ double sh[5][256];
  if (c->done) return;
  double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
  for (int i = threadIdx.x; i < R; i += blockDim.x) {
    a0 += ring_part[2 * i];
    a1 += ring_part[2 * i + 1];
  }
  for (int i = threadIdx.x; i <= lmax; i += blockDim.x) {
    b0 += m_part[3 * i];
    b1 += m_part[3 * i + 1];
    b2 += m_part[3 * i + 2];
  }
  sh[0][threadIdx.x] = a0; sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = b0; sh[3][threadIdx.x] = b1; sh[4][threadIdx.x] = b2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
#pragma unroll
      for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;

  ctl_advance(c, cl, sh[2][0], sh[0][0], sh[1][0], sh[3][0], sh[4][0], hist, hist_cap, nullptr);
}

void launch_control(Ctl *ctl, const double *ring_part, int R, const double *m_part, int lmax, const double *cl,
                    wf_iter_record *hist, int hist_cap, cudaStream_t s) {
  control_kernel<<<1, 256, 0, s>>>(ctl, ring_part, R, m_part, lmax, cl, hist, hist_cap);
}

}  // namespace wfk
