// Batched FP64 solves: wf_solve_batch on a WF_PREC_FP64 plan with a lambda
// table. Right-hand sides go in groups of up to kLegBatchMax maps that
// iterate together: each map runs its own ring stage (Eq. 3 with its own data
// and cached gains) and its own controller (Sect. 3 schedule and stop rule),
// and one launch of legendre_batch_kernel does every map's Legendre stage,
// reading each table row once for the group. A map that has stopped is skipped
// by every kernel until the group's last map stops. The first map of a group
// uses the plan's own buffers; the others use plans of the same shape that
// hold no lambda table (created on first use, re-pointed at the plan's C_l
// and noise), whose buffers the group's kernels read and write. Each map's
// iterates equal its single solve's bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "wf_internal.h"
#include "wf_plan.h"

namespace wfk {

struct F64Batch {
  int nb = 0;
  std::vector<Plan *> sub;          // maps 1 .. nb-1
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  std::vector<const void *> graph_hist;   // the record buffers the graph writes (rebuilt if any moves)
  Ctl *h_ctl = nullptr;             // pinned [nb]
  ~F64Batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (h_ctl) cudaFreeHost(h_ctl);
    for (Plan *p : sub) wf_plan_destroy(p);
  }
};

void destroy_f64_batch(F64Batch *b) { delete b; }

namespace {

#define FB_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

wf_status make_batch(Plan *P, int nb) {
  if (P->f64batch && P->f64batch->nb == nb) return WF_OK;
  destroy_f64_batch(P->f64batch);
  P->f64batch = nullptr;
  F64Batch *F = new (std::nothrow) F64Batch();
  if (!F) { set_error("out of host memory"); return WF_ENOMEM; }
  F->nb = nb;
  std::vector<double> w(P->npix), unit(P->npix, 1.0);
  cudaError_t e = cudaStreamSynchronize(P->run_stream());
  if (e == cudaSuccess) e = cudaMemcpy(w.data(), P->d_w, sizeof(double) * P->npix, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&F->h_ctl, sizeof(Ctl) * nb);
  if (e != cudaSuccess) { delete F; return cuda_status(e, "batched FP64 set-up"); }
  for (int b = 1; b < nb; ++b) {
    wf_options o = P->opt;
    o.legendre_table_bytes = 0;   // the plan's table serves every map
    wf_plan_t q = nullptr;
    wf_status st = wf_plan_create(P->nside, P->lmax, P->h_cl.data(), unit.data(), nullptr, &o, &q);
    if (!st) st = plan_rebind(static_cast<Plan *>(q), P->h_cl.data(), w.data(), P->tau, P->n_obs);
    if (st) { if (q) wf_plan_destroy(q); delete F; return st; }
    F->sub.push_back(static_cast<Plan *>(q));
  }
  P->f64batch = F;
  return WF_OK;
}

}  // namespace

wf_status solve_fp64_batch(Plan *P, int nrhs, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                           wf_stats *stats) {
  if (!P->d_tab || nrhs < 2 || P->opt.precision != WF_PREC_FP64) {
    wf_status worst = WF_OK;
    for (int i = 0; i < nrhs; ++i) {
      const wf_status st = wf_solve(P, d + (size_t)i * P->npix, d_on_device, alm_out + (size_t)i * 2 * P->nalm,
                                    alm_on_device, nullptr, stats ? stats + i : nullptr);
      if (st != WF_OK && st != WF_ENOTCONVERGED) return st;
      if (st != WF_OK) worst = st;
    }
    return worst;
  }
  cudaStream_t s = P->run_stream();
  const int nb = kLegBatchMax;
  wf_status st = make_batch(P, nb);
  if (st) return st;
  F64Batch *F = P->f64batch;
  std::vector<Plan *> M(nb);
  M[0] = P;
  for (int b = 1; b < nb; ++b) {
    M[b] = F->sub[b - 1];
    if ((st = M[b]->ensure_hist(P->opt.max_iter + 1))) return st;
  }
  LegBatchMaps bm{};
  bm.n = nb;
  for (int b = 0; b < nb; ++b) {
    bm.FT[b] = M[b]->d_FT;
    bm.FS[b] = M[b]->d_FS;
    bm.alm[b] = M[b]->d_s;
    bm.m_part[b] = M[b]->d_m_part;
    bm.ctl[b] = M[b]->d_ctl;
    bm.cl[b] = M[b]->d_cl;
    bm.tau[b] = M[b]->tau;
  }
  const int gi = P->opt.graph_iters;
  std::vector<const void *> hist(nb);
  for (int b = 0; b < nb; ++b) hist[b] = M[b]->d_hist;
  if (!F->graph || F->graph_iters != gi || F->graph_hist != hist) {
    if (F->graph) cudaGraphExecDestroy(F->graph);
    F->graph = nullptr;
    cudaGraph_t g;
    FB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < gi; ++i) {
      for (int b = 0; b < nb; ++b) M[b]->launch_rng(M[b]->ring_args(), s, RING_ITER);
      launch_legendre_batch(P->leg_args(), P->legdf_args(), bm, nb, s);
      for (int b = 0; b < nb; ++b)
        launch_control(M[b]->d_ctl, M[b]->d_ring_part, M[b]->R, M[b]->d_m_part, M[b]->lmax, M[b]->d_cl,
                       M[b]->d_hist, M[b]->hist_cap, s);
    }
    FB_CUDA(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&F->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate (batched FP64)");
    F->graph_iters = gi;
    F->graph_hist = hist;
  }
  const double lam0 = P->opt.cooling ? P->lambda_of(P->opt.l_iter0) : 1.0;
  const int lb = P->opt.l_iter0 + P->opt.lmax_margin;
  const int lsht0 = (lam0 <= 1.0 || !P->opt.band_limit) ? P->lmax : std::min(lb, P->lmax);
  const auto kind_in = d_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const auto kind_out = alm_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  wf_status worst = WF_OK;
  for (int i0 = 0; i0 < nrhs; i0 += nb) {
    const int n = std::min(nb, nrhs - i0);
    FB_CUDA(cudaEventRecord(P->ev0, s));
    for (int b = 0; b < nb; ++b) {
      Ctl c = P->make_ctl(1, lam0, lsht0, 0);
      if (b < n) {
        FB_CUDA(cudaMemcpyAsync(M[b]->d_d, d + (size_t)(i0 + b) * P->npix, sizeof(double) * P->npix, kind_in, s));
        M[b]->stage_data(s);
        FB_CUDA(cudaMemsetAsync(M[b]->d_s, 0, sizeof(double2) * P->nalm, s));
        FB_CUDA(cudaMemsetAsync(M[b]->d_FS, 0, sizeof(double4_32a) * (size_t)(P->lmax + 1) * P->RP, s));
      } else {
        c.done = 1;   // a map of the group with no right-hand side
      }
      F->h_ctl[b] = c;
      FB_CUDA(cudaMemcpyAsync(M[b]->d_ctl, F->h_ctl + b, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    }
    const int max_launch = (P->opt.max_iter + gi - 1) / gi + 1;
    for (int it = 0; it < max_launch; ++it) {
      FB_CUDA(cudaGraphLaunch(F->graph, s));
      for (int b = 0; b < nb; ++b)
        FB_CUDA(cudaMemcpyAsync(F->h_ctl + b, M[b]->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
      FB_CUDA(cudaStreamSynchronize(s));
      bool all = true;
      for (int b = 0; b < nb; ++b) all = all && F->h_ctl[b].done;
      if (all) break;
    }
    FB_CUDA(cudaEventRecord(P->ev1, s));
    for (int b = 0; b < n; ++b)
      FB_CUDA(cudaMemcpyAsync(alm_out + (size_t)(i0 + b) * 2 * P->nalm, M[b]->d_s, sizeof(double2) * P->nalm, kind_out,
                              s));
    std::vector<wf_iter_record> last(n);
    for (int b = 0; b < n; ++b) {
      const Ctl &c = F->h_ctl[b];
      if (c.iter > 0)
        FB_CUDA(cudaMemcpyAsync(&last[b], M[b]->d_hist + (c.iter - 1), sizeof(wf_iter_record), cudaMemcpyDeviceToHost,
                                s));
    }
    FB_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P->ev0, P->ev1);
    for (int b = 0; b < n; ++b) {
      const Ctl &c = F->h_ctl[b];
      M[b]->fs_valid = false;
      double rel_pg = -1.0;
      if (stats && P->opt.posterior_grad)
        if ((st = posterior_grad_plan(M[b], s, &rel_pg))) return st;
      if (stats) {
        wf_stats &o = stats[i0 + b];
        o = wf_stats{};
        o.iters = c.iter;
        o.converged = c.converged;
        o.levels = c.level + 1;
        o.lmax_sht_final = c.lsht;
        o.lambda_final = c.lambda;
        o.chi2_prior = last[b].chi2_prior;
        o.chi2_noise = last[b].chi2_noise;
        o.chi2 = last[b].chi2_prior + last[b].chi2_noise;
        o.chi2_per_dof = o.chi2 / (double)P->n_obs;
        o.rel_increment = c.last_rel;
        o.ms_device = ms;
        o.rel_posterior_grad = rel_pg;
      }
      if (c.numeric) { set_error("batched FP64 solve: chi^2 is not finite"); return WF_ENUMERIC; }
      if (!c.converged) worst = WF_ENOTCONVERGED;
    }
  }
  if (worst == WF_ENOTCONVERGED) set_error("batched FP64 solve: max_iter reached before the stop rule");
  return worst;
}

}  // namespace wfk
