// Plan object behind the opaque wf_plan_t handle.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <vector>

#include "wf_internal.h"

struct wf_plan_s {
  virtual ~wf_plan_s() = default;
};

namespace wfk {

struct Engine;
struct F64Batch;
void destroy_f64_batch(F64Batch *b);

struct Plan : wf_plan_s {
  Engine *engine = nullptr;  // batched engine of this shape (mixed precision), built on first use
  F64Batch *f64batch = nullptr;  // batched FP64 solves (batch_fp64.cu): per-map buffers, built on first use
  int nside = 0, lmax = 0, R = 0, RP = 0;
  long long npix = 0, nalm = 0, n_obs = 0;
  double tau = 0.0, omega = 0.0;
  wf_options opt{};
  std::vector<double> h_cl;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int maxM = 1, logMmax = 0;
  size_t device_bytes = 0;
  std::vector<void *> allocs;

  // geometry and tables
  RingDev *d_rings = nullptr;
  int *d_order = nullptr;               // rings sorted by FFT class (RingClass), largest first
  std::vector<RingClass> rclass;        // the classes (batched ring stage: one launch each)
  std::vector<RingClass> rsingle;       // single-solve ring stage: the classes whose 16-byte FFT buffers
                                        // do not fit shared memory (global scratch), then every other ring
  std::vector<RingClass> psingle;       // the same classes in ring pairs (double-float ring stage)
  int2 *d_porder = nullptr;             // pairs in class order: (north ring, south ring or -1)
  void *d_ring_scratch = nullptr;       // their FFT buffers
  double2 *d_tw = nullptr, *d_hs = nullptr, *d_chirp = nullptr, *d_B = nullptr;
  double *d_x = nullptr;
  double2 *d_rec = nullptr, *d_sv = nullptr;
  int *d_ls = nullptr;
  double *d_cl = nullptr, *d_w = nullptr;
  // double-float ring tables
  float4 *d_twf = nullptr, *d_hsf = nullptr, *d_chf = nullptr, *d_Bf = nullptr;
  long long n_tw = 0, n_hs = 0, n_ch = 0, n_B = 0;
  // double-float Legendre tables
  float2 *d_dfA = nullptr;
  double *d_dfg = nullptr;
  int *d_dfls = nullptr;
  float4 *d_dfsv = nullptr;
  float4 *d_tab = nullptr;              // precomputed lambda (FP64 path, when it fits opt.legendre_table_bytes)
  long long *d_poff = nullptr;
  size_t tab_bytes = 0;
  // working state
  double4_32a *d_FS = nullptr, *d_FT = nullptr;
  double *d_ring_part = nullptr, *d_m_part = nullptr;
  Ctl *d_ctl = nullptr;
  Ctl *h_ctl = nullptr;  // pinned mirror
  wf_iter_record *d_hist = nullptr;
  int hist_cap = 0;
  double *d_d = nullptr;
  double *d_gain = nullptr, *d_gainlam = nullptr;  // cached Eq. 3 gains per pixel, lambda per ring
  // the double-float ring stage's copies: data, inverse noise, cached gains (own lambda cache)
  float2 *d_ddf = nullptr, *d_wdf = nullptr, *d_gdf = nullptr;
  double *d_gainlam_df = nullptr;
  double *d_pmap = nullptr;             // posterior gradient: W (d - Y a) and W d [2][npix]
  double2 *d_palm = nullptr;            // their analyses [2][nalm]
  double *d_ppart = nullptr;            // per-m norms [lmax+1][2]
  double2 *d_s = nullptr;
  bool fs_valid = false;
  int fs_lsht = -1;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_prec = -1;                  // precision whose kernels graph_exec holds
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  const std::atomic<int> *cancel = nullptr;  // set by the server: wf_solve stops between graph launches

  ~Plan() override;
  wf_status dalloc(void **p, size_t bytes);
  wf_status alloc_work();
  wf_status ensure_hist(int cap);
  cudaStream_t run_stream() const;
  RingArgs ring_args() const;
  LegArgs leg_args() const;
  LegDfArgs legdf_args() const { return LegDfArgs{d_dfA, d_dfg, d_dfls, d_dfsv, d_tab, d_poff}; }
  RingDfArgs ringdf_args() const {
    return RingDfArgs{d_twf, d_hsf, d_chf, d_Bf, d_ddf, d_wdf, d_gdf, d_gainlam_df};
  }
  // d_d was (re)written: its double-float copy for the ring stage, in stream order
  void stage_data(cudaStream_t s) const { launch_to_df2(d_d, d_ddf, npix, s); }
  // the ring stage of the plan's precision
  void launch_rng(const RingArgs &a, cudaStream_t s, int mode) const {
    if (opt.precision == WF_PREC_FP64_NATIVE) launch_ring(a, rsingle.data(), (int)rsingle.size(), s, mode);
    else launch_ring_df(a, ringdf_args(), psingle.data(), (int)psingle.size(), s, mode);
  }
  // the Legendre stage of the plan's precision
  void launch_leg(const LegArgs &a, cudaStream_t s, int mode) const {
    if (opt.precision == WF_PREC_FP64_NATIVE) launch_legendre(a, s, mode);
    else launch_legendre_df(a, legdf_args(), s, mode);
  }
  void enqueue_iteration(cudaStream_t s);
  Ctl make_ctl(int mode, double lambda, int lsht, int n_fixed) const;
  double lambda_of(int l_iter) const;
};

// Re-point a plan at another problem of its shape: C_l ([lmax+1]), the inverse
// noise w ([npix], 0 where masked), tau and the observed-pixel count. Every
// table derived from the geometry (FFT, Legendre, lambda table) is kept; the
// cached Eq. 3 gains and the captured iteration graph are dropped. Host
// arrays are read before it returns.
wf_status plan_rebind(Plan *P, const double *cl, const double *w, double tau, long long n_obs);

// FP64 refinement of a mixed result: up to opt.refine_iters double-float
// iterations at lambda = 1 from alm_dev (device a_lm), written to alm_out; the
// refined figures replace those of stats (iterations and time are added).
wf_status refine_fp64(Plan *P, const double *d, int d_on_device, const double *alm_dev, double *alm_out,
                      int alm_on_device, wf_stats *stats);

// rel_posterior_grad of the plan's state d_s against its data d_d (capi.cu).
wf_status posterior_grad_plan(Plan *P, cudaStream_t s, double *rel);

// FP64 solves of nrhs right-hand sides in groups that share the Legendre stage (batch_fp64.cu);
// plans without a lambda table solve them one by one.
wf_status solve_fp64_batch(Plan *P, int nrhs, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                           wf_stats *stats);

// Mixed-precision solves through the plan's batched engine (batch.cu).
wf_status solve_mixed(Plan *P, int nrhs, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                      wf_stats *stats);

}  // namespace wfk
