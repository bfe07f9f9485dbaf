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

#include "wf_internal.h"

namespace wfk {

__device__ double lambda_for(const Ctl *c, const double *cl, int l_iter) {
  if (l_iter > c->lmax) return 1.0;
  const double r = cl[l_iter] / (c->tau * c->omega);
  return r > 1.0 ? r : 1.0;
}

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

  const double chi2_noise = sh[0][0], chi2_lnoise = sh[1][0];
  const double chi2_prior = sh[2][0], incr2 = sh[3][0], norm2 = sh[4][0];
  const double chi2 = chi2_prior + chi2_noise;
  if (c->iter < hist_cap) {
    wf_iter_record rec;
    rec.chi2_prior = chi2_prior;
    rec.chi2_noise = chi2_noise;
    rec.chi2_lambda = chi2_prior + chi2_lnoise;
    rec.incr2 = incr2;
    rec.norm2 = norm2;
    rec.lambda = c->lambda;
    rec.lmax_sht = c->lsht;
    rec.level = c->level;
    hist[c->iter] = rec;
  }
  c->iter += 1;
  c->last_rel = norm2 > 0.0 ? sqrt(incr2 / norm2) : 0.0;
  if (!isfinite(chi2) || !isfinite(norm2)) {
    c->numeric = 1;
    c->done = 1;
    return;
  }
  if (c->mode == 0) {
    if (c->iter >= c->n_fixed) c->done = 1;
    return;
  }
  c->level_iters += 1;
  const bool have_d = c->have_prev && c->level_iters >= 3;
  const double dchi2 = have_d ? fabs(chi2 - c->prev_chi2) : 0.0;
  c->prev_chi2 = chi2;
  c->have_prev = 1;
  if (c->lambda > 1.0) {
    const bool plateau = have_d && dchi2 < c->plateau_eps * c->sigma_chi2 && c->level_iters >= c->min_level_iters;
    if (plateau || c->level_iters >= c->max_level_iters) {
      c->l_iter *= 2;
      const double ln = lambda_for(c, cl, c->l_iter);
      c->lambda = ln < c->lambda ? ln : c->lambda;
      c->level += 1;
      c->level_iters = 0;
      c->have_prev = 0;
      const int lb = c->l_iter + c->margin;
      c->lsht = (c->lambda <= 1.0 || !c->band_limit) ? c->lmax : (lb < c->lmax ? lb : c->lmax);
    }
  } else {
    if (c->level_iters >= 2 && c->last_rel <= c->tol) {
      c->converged = 1;
      c->done = 1;
    } else if (c->final_dchi2 > 0.0 && have_d && dchi2 < c->final_dchi2 * c->sigma_chi2) {
      c->converged = 1;
      c->done = 1;
    }
  }
  if (c->iter >= c->max_iter) c->done = 1;
}

void launch_control(Ctl *ctl, const double *ring_part, int R, const double *m_part, int lmax, const double *cl,
                    wf_iter_record *hist, int hist_cap, cudaStream_t s) {
  control_kernel<<<1, 256, 0, s>>>(ctl, ring_part, R, m_part, lmax, cl, hist, hist_cap);
}

}  // namespace wfk
