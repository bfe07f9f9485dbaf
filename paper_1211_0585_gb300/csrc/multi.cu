// Several messenger fields for several observations of one sky (Sect. 4,
// Conclusion: more than one messenger field, e.g. to combine the maps of
// several detectors in one analysis).
//
// K maps on one HEALPix grid, d_k = Y B_k s + n_k, with a beam B_k =
// diag(b_k,l) and noise N_k diagonal in pixel space (masked: N_k^-1 = 0) per
// map. Map k has its own messenger t_k with T_k = tau_k 1, tau_k = min
// diag(N_k), and one iteration is
//   for each k:  Y B_k s                 synthesis of b_k s (Legendre stage, ring FFT)
//                u_k = a_k (d_k - Y B_k s)  Eq. 3 per pixel, the map's own gains a_k(lambda)
//                Y^dagger u_k             analysis (ring FFT, Legendre stage)
//   s_lm = sum_k g_k b_k,l (b_k,l s_lm + (Y^dagger u_k)_lm) / (1 / C_l + sum_k g_k b_k,l^2),
//          g_k = 1 / (lambda tau_k Omega)      Eq. 4 with every messenger
// so that the fixed point at lambda = 1 is the joint Wiener filter
//   (S^-1 + sum_k B_k Y^T N_k^-1 Y B_k) s = sum_k B_k Y^T N_k^-1 d_k.
// The chi^2 monitor sums every map's noise term; the cooling of Sect. 3 sets
// lambda at scale l to C_l sum_k b_k,l^2 / (tau_k Omega) (where the combined
// filter's gain is 1/2). The band limit stays at lmax.
//
// Each map is held by a plan of its own (noise, mask, cached Eq. 3 gains,
// Fourier and ring buffers); the Legendre tables of the first plan serve
// every map's transforms, so only it holds a lambda table. The iterations run
// as CUDA graphs on the first plan's stream with the controller on the device.
#include <cuda_runtime.h>

#include <algorithm>

#include <cmath>
#include <new>
#include <vector>

#include "ctl.cuh"
#include "wf_internal.h"
#include "wf_plan.h"

struct wf_multi_s {
  virtual ~wf_multi_s() = default;
};

namespace wfk {
namespace {

constexpr int kMultiMax = 16;

struct Multi : wf_multi_s {
  int K = 0, nside = 0, lmax = 0, R = 0;
  long long npix = 0, nalm = 0, n_obs = 0;
  double omega = 0.0;
  wf_options opt{};
  std::vector<Plan *> P;
  std::vector<double> h_cl, h_lamcl, taus;
  double *d_beam = nullptr, *d_tau = nullptr, *d_cl = nullptr, *d_lamcl = nullptr;
  double2 *d_s = nullptr, *d_balm = nullptr, *d_ta = nullptr;
  double *d_ring_part = nullptr, *d_m_part = nullptr;
  Ctl *d_ctl = nullptr, *h_ctl = nullptr;
  wf_iter_record *d_hist = nullptr;
  int hist_cap = 0;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void *> allocs;

  ~Multi() override {
    if (graph) cudaGraphExecDestroy(graph);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (h_ctl) cudaFreeHost(h_ctl);
    for (void *p : allocs) cudaFree(p);
    for (Plan *p : P) wf_plan_destroy(p);
  }
  wf_status dalloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) { *p = nullptr; return cuda_status(e, "cudaMalloc (several messenger fields)"); }
    allocs.push_back(*p);
    return WF_OK;
  }
  cudaStream_t stream() const { return P[0]->run_stream(); }
  void enqueue_iteration(cudaStream_t s);
};

__device__ __forceinline__ size_t idx_lm(int lmax, int l, int m) { return (size_t)m * (2 * lmax + 1 - m) / 2 + l; }

// balm = b_k s for every map (one CTA per m)
__global__ void multi_beam_kernel(const Ctl *ctl, int K, int lmax, long long nalm, const double *beam,
                                  const double2 *s, double2 *balm) {
  if (ctl->done) return;
  const int m = blockIdx.x;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const size_t q = idx_lm(lmax, l, m);
    const double2 v = s[q];
    for (int k = 0; k < K; ++k) {
      const double b = beam[(size_t)k * (lmax + 1) + l];
      balm[(size_t)k * nalm + q] = make_double2(b * v.x, b * v.y);
    }
  }
}

// Eq. 4 with K messengers, the prior chi^2 of the input state, the increment
// and norm partials per m (the layout the controller reads)
__global__ void multi_eq4_kernel(const Ctl *ctl, int K, int lmax, long long nalm, double omega, const double *beam,
                                 const double *tau, const double *cl, const double2 *ta, double2 *s,
                                 double *m_part) {
  __shared__ double red[3][32];
  if (ctl->done) return;
  const int m = blockIdx.x;
  const double lam = ctl->lambda;
  const double wgt = (m == 0) ? 1.0 : 2.0;
  double c2 = 0.0, inc = 0.0, nrm = 0.0;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const size_t q = idx_lm(lmax, l, m);
    const double2 so = s[q];
    const double c = cl[l];
    double2 sn = make_double2(0.0, 0.0);
    if (c > 0.0) {
      double nx = 0.0, ny = 0.0, den = 1.0 / c;
      for (int k = 0; k < K; ++k) {
        const double b = beam[(size_t)k * (lmax + 1) + l];
        const double g = 1.0 / (lam * tau[k] * omega);
        const double2 t = ta[(size_t)k * nalm + q];
        nx += g * b * (b * so.x + t.x);
        ny += g * b * (b * so.y + t.y);
        den += g * b * b;
      }
      sn = make_double2(nx / den, ny / den);
      c2 += wgt * (so.x * so.x + so.y * so.y) / c;
    }
    const double dx = sn.x - so.x, dy = sn.y - so.y;
    inc += wgt * (dx * dx + dy * dy);
    nrm += wgt * (sn.x * sn.x + sn.y * sn.y);
    s[q] = sn;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    inc += __shfl_xor_sync(0xffffffffu, inc, o);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][w] = c2; red[1][w] = inc; red[2][w] = nrm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, d = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[0][i]; b += red[1][i]; d += red[2][i]; }
    m_part[3 * m] = a;
    m_part[3 * m + 1] = b;
    m_part[3 * m + 2] = d;
  }
}

void Multi::enqueue_iteration(cudaStream_t s) {
  Plan *P0 = P[0];
  multi_beam_kernel<<<lmax + 1, 128, 0, s>>>(d_ctl, K, lmax, nalm, d_beam, d_s, d_balm);
  if (P0->legdf_args().tab) {
    // table form: the maps' syntheses, and then their analyses, two maps per launch (each table row
    // read once for both; every map's transform bitwise the single kernel's)
    for (int k0 = 0; k0 < K; k0 += kLegBatchMax) {
      const int nb = std::min(kLegBatchMax, K - k0);
      LegBatchMaps syn{}, ana{};
      syn.n = ana.n = nb;
      for (int b = 0; b < nb; ++b) {
        const int k = k0 + b;
        syn.FS[b] = P[k]->d_FS;
        syn.alm[b] = d_balm + (size_t)k * nalm;
        ana.FT[b] = P[k]->d_FT;
        ana.alm[b] = d_ta + (size_t)k * nalm;
        syn.ctl[b] = ana.ctl[b] = d_ctl;
      }
      LegArgs la = P0->leg_args();
      la.lsht = lmax;
      launch_legendre_batch(la, P0->legdf_args(), syn, nb, s, LEG_SYNTH);
      for (int b = 0; b < nb; ++b) {
        const int k = k0 + b;
        RingArgs ra = P[k]->ring_args();   // map k's data, noise, gains and Fourier buffers
        ra.ctl = d_ctl;
        ra.ring_part = d_ring_part + (size_t)k * 2 * R;
        P[k]->launch_rng(ra, s, RING_ITER);
      }
      launch_legendre_batch(la, P0->legdf_args(), ana, nb, s, LEG_ANALYSIS);
    }
    multi_eq4_kernel<<<lmax + 1, 128, 0, s>>>(d_ctl, K, lmax, nalm, omega, d_beam, d_tau, d_cl, d_ta, d_s, d_m_part);
    launch_control(d_ctl, d_ring_part, K * R, d_m_part, lmax, d_lamcl, d_hist, hist_cap, s);
    return;
  }
  for (int k = 0; k < K; ++k) {
    LegArgs ls = P0->leg_args();          // the first plan's Legendre tables, map k's buffers
    ls.lsht = lmax;
    ls.alm_in = d_balm + (size_t)k * nalm;
    ls.FS = P[k]->d_FS;
    ls.gate = d_ctl;
    P0->launch_leg(ls, s, LEG_SYNTH);
    RingArgs ra = P[k]->ring_args();      // map k's data, noise, gains and Fourier buffers
    ra.ctl = d_ctl;
    ra.ring_part = d_ring_part + (size_t)k * 2 * R;
    P[k]->launch_rng(ra, s, RING_ITER);
    LegArgs la = P0->leg_args();
    la.lsht = lmax;
    la.FT = P[k]->d_FT;
    la.alm = d_ta + (size_t)k * nalm;
    la.gate = d_ctl;
    P0->launch_leg(la, s, LEG_ANALYSIS);
  }
  multi_eq4_kernel<<<lmax + 1, 128, 0, s>>>(d_ctl, K, lmax, nalm, omega, d_beam, d_tau, d_cl, d_ta, d_s, d_m_part);
  launch_control(d_ctl, d_ring_part, K * R, d_m_part, lmax, d_lamcl, d_hist, hist_cap, s);
}

}  // namespace
}  // namespace wfk

using namespace wfk;

#define MU_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

extern "C" {

wf_status wf_multi_create(int nside, int lmax, int ndet, const double *cl, const double *beams,
                          const double *noise_var, const uint8_t *mask, const wf_options *opt, wf_multi_t *out) {
  if (!out || !cl || !noise_var) { set_error("wf_multi_create: NULL argument"); return WF_EINVAL; }
  *out = nullptr;
  if (ndet < 1 || ndet > kMultiMax) { set_error("wf_multi_create: ndet must be in [1, 16]"); return WF_EINVAL; }
  wf_options o;
  if (opt) o = *opt;
  else wf_options_default(&o);
  if (o.precision == WF_PREC_MIXED) {
    set_error("wf_multi_create: several messenger fields run on the FP64 paths (WF_PREC_FP64, WF_PREC_FP64_NATIVE)");
    return WF_EINVAL;
  }
  o.band_limit = 0;  // the band limit stays at lmax
  const long long npix = 12LL * nside * nside;
  if (beams)
    for (long long i = 0; i < (long long)ndet * (lmax + 1); ++i)
      if (!std::isfinite(beams[i])) { set_error("wf_multi_create: beams must be finite"); return WF_EINVAL; }
  Multi *M = new (std::nothrow) Multi();
  if (!M) { set_error("out of host memory"); return WF_ENOMEM; }
  M->K = ndet;
  M->opt = o;
  for (int k = 0; k < ndet; ++k) {
    wf_options ok = o;
    if (k > 0) ok.legendre_table_bytes = 0;  // the first plan's tables serve every map
    wf_plan_t p = nullptr;
    const wf_status st = wf_plan_create(nside, lmax, cl, noise_var + (size_t)k * npix,
                                        mask ? mask + (size_t)k * npix : nullptr, &ok, &p);
    if (st) { delete M; return st; }
    M->P.push_back(static_cast<Plan *>(p));
  }
  Plan *P0 = M->P[0];
  M->nside = nside;
  M->lmax = lmax;
  M->R = P0->R;
  M->npix = npix;
  M->nalm = P0->nalm;
  M->omega = P0->omega;
  M->h_cl.assign(cl, cl + lmax + 1);
  std::vector<double> hb((size_t)ndet * (lmax + 1), 1.0);
  if (beams) hb.assign(beams, beams + hb.size());
  for (Plan *p : M->P) {
    M->taus.push_back(p->tau);
    M->n_obs += p->n_obs;
  }
  // lambda at scale l (controller): C_l sum_k b_k,l^2 / (tau_k Omega) read as lamcl[l] / (1 * Omega)
  M->h_lamcl.assign(lmax + 1, 0.0);
  for (int l = 0; l <= lmax; ++l) {
    double a = 0.0;
    for (int k = 0; k < ndet; ++k) a += hb[(size_t)k * (lmax + 1) + l] * hb[(size_t)k * (lmax + 1) + l] / M->taus[k];
    M->h_lamcl[l] = cl[l] * a;
  }
  wf_status st;
  if ((st = M->dalloc((void **)&M->d_beam, sizeof(double) * hb.size())) ||
      (st = M->dalloc((void **)&M->d_tau, sizeof(double) * ndet)) ||
      (st = M->dalloc((void **)&M->d_cl, sizeof(double) * (lmax + 1))) ||
      (st = M->dalloc((void **)&M->d_lamcl, sizeof(double) * (lmax + 1))) ||
      (st = M->dalloc((void **)&M->d_s, sizeof(double2) * M->nalm)) ||
      (st = M->dalloc((void **)&M->d_balm, sizeof(double2) * M->nalm * ndet)) ||
      (st = M->dalloc((void **)&M->d_ta, sizeof(double2) * M->nalm * ndet)) ||
      (st = M->dalloc((void **)&M->d_ring_part, sizeof(double) * 2 * M->R * ndet)) ||
      (st = M->dalloc((void **)&M->d_m_part, sizeof(double) * 3 * (lmax + 1))) ||
      (st = M->dalloc((void **)&M->d_ctl, sizeof(Ctl))) ||
      (st = M->dalloc((void **)&M->d_hist, sizeof(wf_iter_record) * (size_t)(o.max_iter + 1)))) {
    delete M;
    return st;
  }
  M->hist_cap = o.max_iter + 1;
  cudaError_t e = cudaMemcpy(M->d_beam, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(M->d_tau, M->taus.data(), sizeof(double) * ndet, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(M->d_cl, cl, sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(M->d_lamcl, M->h_lamcl.data(), sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&M->h_ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaEventCreate(&M->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&M->ev1);
  if (e != cudaSuccess) { st = cuda_status(e, "wf_multi_create upload"); delete M; return st; }
  *out = M;
  return WF_OK;
}

wf_status wf_multi_destroy(wf_multi_t multi) {
  if (!multi) return WF_OK;
  Multi *M = static_cast<Multi *>(multi);
  cudaStreamSynchronize(M->stream());
  delete M;
  return WF_OK;
}

wf_status wf_multi_solve(wf_multi_t multi, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                         wf_stats *stats, wf_iter_record *records, int max_records, int *n_records) {
  if (!multi || !d || !alm_out) { set_error("wf_multi_solve: NULL argument"); return WF_EINVAL; }
  Multi *M = static_cast<Multi *>(multi);
  Plan *P0 = M->P[0];
  cudaStream_t s = M->stream();
  const auto kind_in = d_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MU_CUDA(cudaEventRecord(M->ev0, s));
  for (int k = 0; k < M->K; ++k) {
    MU_CUDA(cudaMemcpyAsync(M->P[k]->d_d, d + (size_t)k * M->npix, sizeof(double) * M->npix, kind_in, s));
    M->P[k]->stage_data(s);
  }
  MU_CUDA(cudaMemsetAsync(M->d_s, 0, sizeof(double2) * M->nalm, s));
  double lam0 = 1.0;
  if (M->opt.cooling && M->opt.l_iter0 <= M->lmax) lam0 = std::max(1.0, M->h_lamcl[M->opt.l_iter0] / M->omega);
  Ctl c = P0->make_ctl(1, lam0, M->lmax, 0);
  c.band_limit = 0;
  c.tau = 1.0;  // lambda_for reads lamcl[l] / (tau Omega)
  c.sigma_chi2 = std::sqrt(2.0 * (double)M->n_obs);
  *M->h_ctl = c;
  MU_CUDA(cudaMemcpyAsync(M->d_ctl, M->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  const int gi = M->opt.graph_iters;
  if (!M->graph) {
    cudaGraph_t g;
    MU_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < gi; ++i) M->enqueue_iteration(s);
    MU_CUDA(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&M->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate (several messenger fields)");
  }
  const int max_launch = (M->opt.max_iter + gi - 1) / gi + 1;
  for (int it = 0; it < max_launch; ++it) {
    MU_CUDA(cudaGraphLaunch(M->graph, s));
    MU_CUDA(cudaMemcpyAsync(M->h_ctl, M->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    MU_CUDA(cudaStreamSynchronize(s));
    if (M->h_ctl->done) break;
  }
  MU_CUDA(cudaMemcpyAsync(alm_out, M->d_s, sizeof(double2) * M->nalm,
                          alm_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  MU_CUDA(cudaEventRecord(M->ev1, s));
  const Ctl fin = *M->h_ctl;
  wf_iter_record last{};
  if (fin.iter > 0)
    MU_CUDA(cudaMemcpyAsync(&last, M->d_hist + (fin.iter - 1), sizeof(last), cudaMemcpyDeviceToHost, s));
  int nrec = 0;
  if (records && max_records > 0) {
    nrec = fin.iter < max_records ? fin.iter : max_records;
    if (nrec > 0)
      MU_CUDA(cudaMemcpyAsync(records, M->d_hist, sizeof(wf_iter_record) * nrec, cudaMemcpyDeviceToHost, s));
  }
  MU_CUDA(cudaStreamSynchronize(s));
  if (n_records) *n_records = nrec;
  for (Plan *p : M->P) p->fs_valid = false;
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, M->ev0, M->ev1);
    *stats = wf_stats{};
    stats->iters = fin.iter;
    stats->converged = fin.converged;
    stats->levels = fin.level + 1;
    stats->lmax_sht_final = fin.lsht;
    stats->lambda_final = fin.lambda;
    stats->chi2_prior = last.chi2_prior;
    stats->chi2_noise = last.chi2_noise;
    stats->chi2 = last.chi2_prior + last.chi2_noise;
    stats->chi2_per_dof = stats->chi2 / (double)M->n_obs;
    stats->rel_increment = fin.last_rel;
    stats->ms_device = ms;
    stats->rel_posterior_grad = -1.0;
  }
  if (fin.numeric) { set_error("wf_multi_solve: chi^2 is not finite"); return WF_ENUMERIC; }
  if (!fin.converged) { set_error("wf_multi_solve: max_iter reached before the stop rule"); return WF_ENOTCONVERGED; }
  return WF_OK;
}

}  // extern "C"
