// One step of the Sect. 3 schedule on a controller state, shared by the
// single-map controller (control.cu) and the per-slot batched controller.
#pragma once

#include "wf_internal.h"

namespace wfk {

__device__ __forceinline__ double ctl_lambda_for(const Ctl *c, const double *cl, int l_iter) {
  if (l_iter > c->lmax) return 1.0;
  const double r = cl[l_iter] / (c->tau * c->omega);
  return r > 1.0 ? r : 1.0;
}

// Record the iteration (when hist != nullptr and room remains) and advance
// the schedule: plateau -> next level (Sect. 3), stop rule at lambda = 1.
__device__ __forceinline__ void ctl_advance(Ctl *c, const double *cl, double chi2_prior, double chi2_noise,
                                            double chi2_lnoise, double incr2, double norm2, wf_iter_record *hist,
                                            int hist_cap, wf_iter_record *last) {
  const double chi2 = chi2_prior + chi2_noise;
  wf_iter_record rec;
  rec.chi2_prior = chi2_prior;
  rec.chi2_noise = chi2_noise;
  rec.chi2_lambda = chi2_prior + chi2_lnoise;
  rec.incr2 = incr2;
  rec.norm2 = norm2;
  rec.lambda = c->lambda;
  rec.lmax_sht = c->lsht;
  rec.level = c->level;
  if (hist && c->iter < hist_cap) hist[c->iter] = rec;
  if (last) *last = rec;
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
      const double ln = ctl_lambda_for(c, cl, c->l_iter);
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

}  // namespace wfk
