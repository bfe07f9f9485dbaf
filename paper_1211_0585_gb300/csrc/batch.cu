// Multiple right-hand sides sharing one plan (C_l, noise, mask).
#include <cuda_runtime.h>

#include "wf_internal.h"
#include "wf_plan.h"

using namespace wfk;

extern "C" wf_status wf_solve_batch(wf_plan_t plan, int nrhs, const double *d, int d_on_device, double *alm_out,
                                    int alm_on_device, wf_stats *stats) {
  if (!plan || !d || !alm_out || nrhs < 0) { set_error("wf_solve_batch: bad argument"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  wf_status worst = WF_OK;
  for (int i = 0; i < nrhs; ++i) {
    const wf_status st = wf_solve(plan, d + (size_t)i * P->npix, d_on_device, alm_out + (size_t)i * 2 * P->nalm,
                                  alm_on_device, nullptr, stats ? stats + i : nullptr);
    if (st != WF_OK && st != WF_ENOTCONVERGED) return st;
    if (st != WF_OK) worst = st;
  }
  return worst;
}
