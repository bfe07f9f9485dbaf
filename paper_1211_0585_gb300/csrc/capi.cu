// C ABI of the messenger-field Wiener filter (plan, transforms, solves).
// The host side builds the HEALPix ring geometry and the per-length FFT
// tables, checks inputs, owns device memory and drives the kernels; every
// arithmetic step of the method runs in the kernels of ring.cu,
// legendre.cu and control.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "batch_engine.h"
#include "wf_internal.h"
#include "wf_plan.h"

namespace wfk {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

wf_status cuda_status(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return WF_OK;
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? WF_ENOMEM : WF_ECUDA;
}

#define WF_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

static int ilog2(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

static size_t alm_count(int lmax) { return (size_t)(lmax + 1) * (lmax + 2) / 2; }

wf_status Plan::dalloc(void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
  allocs.push_back(*p);
  device_bytes += bytes;
  return WF_OK;
}

Plan::~Plan() {
  delete engine;
  destroy_f64_batch(f64batch);
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  for (void *p : allocs) cudaFree(p);
  if (h_ctl) cudaFreeHost(h_ctl);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

cudaStream_t Plan::run_stream() const {
  return opt.stream ? static_cast<cudaStream_t>(opt.stream) : stream;
}

void raise_smem_cap(const void *func) {
  static std::mutex mu;
  static std::set<const void *> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(func)) return;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, func) != cudaSuccess)
    return;   // the launch itself then reports the error
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) ==
      cudaSuccess)
    done.insert(func);
}

// Rings sorted by FFT class, largest first: the three largest FFT sizes are a
// class each, every smaller size joins one last class. Within a class the two
// rings of a pair are adjacent.
void ring_classes(const RingDev *rings, int R, std::vector<int> &order, std::vector<RingClass> &cls) {
  int logMmax = 0;
  for (int r = 0; r < R; ++r) logMmax = std::max(logMmax, rings[r].logM);
  const int floor_log = std::max(0, logMmax - 3);
  auto key = [&](int r) { return std::max(rings[r].logM, floor_log); };
  order.resize(R);
  for (int r = 0; r < R; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (key(a) != key(b)) return key(a) > key(b);
    if (rings[a].pair != rings[b].pair) return rings[a].pair < rings[b].pair;
    return rings[a].side < rings[b].side;
  });
  cls.clear();
  for (int i = 0; i < R; ++i) {
    const int k = key(order[i]);
    if (cls.empty() || cls.back().logM != k) cls.push_back(RingClass{k, i, 0, 0});
    ++cls.back().count;
  }
}

static wf_status build_geometry(Plan *P) {
  const int ns = P->nside, R = P->R;
  std::vector<RingDev> rings(R);
  // per-length tables: polar lengths 4i (i = 1 .. nside - 1), then the belt length 4 nside
  std::vector<long long> hs_off(ns + 1), ch_off(ns + 1), B_off(ns + 1, -1);
  std::vector<int> logM(ns + 1), blue(ns + 1);
  long long hs_tot = 0, ch_tot = 0, B_tot = 0;
  int maxM = 1;
  for (int i = 1; i <= ns; ++i) {
    const long long n = 4LL * i;
    hs_off[i] = hs_tot;
    hs_tot += n;
    const bool pow2 = (n & (n - 1)) == 0;
    blue[i] = pow2 ? 0 : 1;
    logM[i] = pow2 ? ilog2(n) : ilog2(2 * n - 1);
    if (!pow2) {
      ch_off[i] = ch_tot;
      ch_tot += n;
      B_off[i] = B_tot;
      B_tot += 1LL << logM[i];
    } else {
      ch_off[i] = 0;
      B_off[i] = 0;
    }
    if ((1 << logM[i]) > maxM) maxM = 1 << logM[i];
  }
  const long long npix = P->npix;
  for (int r = 0; r < R; ++r) {
    const int i = r + 1;
    const int ip = i < 4 * ns - i ? i : 4 * ns - i;  // mirrored ring number
    RingDev g{};
    const bool polar = ip < ns;
    const int cls = polar ? ip : ns;                 // length class
    g.n = 4 * cls;
    if (i < ns) g.off = 2LL * i * (i - 1);
    else if (i <= 3 * ns) g.off = 2LL * ns * (ns - 1) + (long long)(i - ns) * 4 * ns;
    else g.off = npix - 2LL * ip * (ip + 1);
    g.shifted = polar ? 1 : (((i - ns) % 2) == 0 ? 1 : 0);
    g.pair = r < R - 1 - r ? r : R - 1 - r;
    g.side = r > R - 1 - r ? 1 : 0;
    g.logM = logM[cls];
    g.blue = blue[cls];
    g.hs_off = hs_off[cls];
    g.ch_off = ch_off[cls];
    g.B_off = B_off[cls];
    rings[r] = g;
  }
  P->maxM = maxM;
  P->logMmax = ilog2(maxM);
  // tables
  // the chirp table is padded to the longest ring so that an index q < n is
  // always inside it, even on rings that never use it
  std::vector<double2> hs(hs_tot), ch(std::max<long long>(ch_tot, 4LL * ns), make_double2(0.0, 0.0));
  std::vector<double2> tw(maxM);  // e^{-2 pi i k / Mmax}, k < Mmax (radix-4 stages reach 3 Mmax / 4)
  for (int i = 1; i <= ns; ++i) {
    const long long n = 4LL * i;
    for (long long q = 0; q < n; ++q) {
      const double a = M_PI * (double)q / (double)n;
      hs[hs_off[i] + q] = make_double2(cos(a), sin(a));
    }
    if (blue[i]) {
      for (long long j = 0; j < n; ++j) {
        const long long jj = (j * j) % (2 * n);
        const double a = M_PI * (double)jj / (double)n;
        ch[ch_off[i] + j] = make_double2(cos(a), -sin(a));
      }
    }
  }
  for (int k = 0; k < maxM; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)maxM;
    tw[k] = make_double2(cos(a), -sin(a));
  }
  std::vector<double> xk(P->RP);
  for (int k = 0; k < P->RP; ++k) {
    const int i = k + 1;
    xk[k] = (i < ns) ? 1.0 - (double)i * i / (3.0 * (double)ns * ns) : 4.0 / 3.0 - 2.0 * i / (3.0 * ns);
  }
  wf_status st;
  std::vector<int> order;
  ring_classes(rings.data(), R, order, P->rclass);
  // single-solve launches: a class whose FFT buffer (16-byte elements) and real
  // ring values (8 bytes) exceed the shared-memory limit runs on a global
  // scratch array, one launch per such class; all other rings form one launch
  size_t scratch_elems = 0;
  int next = 0;
  P->rsingle.clear();
  for (const RingClass &c : P->rclass) {
    if (((size_t)1 << c.logM) * 24 <= kRingSmemLimit) break;
    RingClass g = c;
    g.global = 1;
    P->rsingle.push_back(g);
    scratch_elems = std::max(scratch_elems, (size_t)c.count << c.logM);
    next = c.first + c.count;
  }
  if (next < R) {
    int lg = 0;
    for (int i = next; i < R; ++i) lg = std::max(lg, rings[order[i]].logM);
    P->rsingle.push_back(RingClass{lg, next, R - next, 0});
  }
  // the same launches in ring pairs (the two rings of a pair are adjacent in a class)
  std::vector<int2> porder;
  P->psingle.clear();
  for (const RingClass &c : P->rsingle) {
    RingClass g = c;
    g.first = (int)porder.size();
    for (int i = c.first; i < c.first + c.count;) {
      const bool both = i + 1 < c.first + c.count && rings[order[i + 1]].pair == rings[order[i]].pair;
      porder.push_back(make_int2(order[i], both ? order[i + 1] : -1));
      i += both ? 2 : 1;
    }
    g.count = (int)porder.size() - g.first;
    P->psingle.push_back(g);
  }
  if ((st = P->dalloc((void **)&P->d_rings, sizeof(RingDev) * R))) return st;
  if ((st = P->dalloc((void **)&P->d_order, sizeof(int) * R))) return st;
  if ((st = P->dalloc((void **)&P->d_porder, sizeof(int2) * porder.size()))) return st;
  if (scratch_elems > 0 && (st = P->dalloc(&P->d_ring_scratch, 16 * scratch_elems))) return st;
  if ((st = P->dalloc((void **)&P->d_hs, sizeof(double2) * hs.size()))) return st;
  if ((st = P->dalloc((void **)&P->d_chirp, sizeof(double2) * ch.size()))) return st;
  if ((st = P->dalloc((void **)&P->d_B, sizeof(double2) * (B_tot > 0 ? B_tot : 1)))) return st;
  if ((st = P->dalloc((void **)&P->d_tw, sizeof(double2) * tw.size()))) return st;
  if ((st = P->dalloc((void **)&P->d_x, sizeof(double) * P->RP))) return st;
  cudaStream_t s = P->stream;
  WF_CUDA(cudaMemcpyAsync(P->d_rings, rings.data(), sizeof(RingDev) * R, cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_order, order.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_porder, porder.data(), sizeof(int2) * porder.size(), cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_hs, hs.data(), sizeof(double2) * hs.size(), cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_chirp, ch.data(), sizeof(double2) * ch.size(), cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_x, xk.data(), sizeof(double) * P->RP, cudaMemcpyHostToDevice, s));
  if (B_tot > 0)
    launch_bluestein_setup(P->d_rings, P->d_order, P->rsingle.data(), (int)P->rsingle.size(), P->d_ring_scratch,
                           P->d_tw, P->logMmax, P->d_chirp, P->d_B, s);
  // double-float copies for the ring_df kernels
  P->n_tw = (long long)tw.size();
  P->n_hs = (long long)hs.size();
  P->n_ch = (long long)ch.size();
  P->n_B = B_tot > 0 ? B_tot : 1;
  if ((st = P->dalloc((void **)&P->d_twf, sizeof(float4) * P->n_tw))) return st;
  if ((st = P->dalloc((void **)&P->d_hsf, sizeof(float4) * P->n_hs))) return st;
  if ((st = P->dalloc((void **)&P->d_chf, sizeof(float4) * P->n_ch))) return st;
  if ((st = P->dalloc((void **)&P->d_Bf, sizeof(float4) * P->n_B))) return st;
  launch_to_df(P->d_tw, P->d_twf, P->n_tw, s);
  launch_to_df(P->d_hs, P->d_hsf, P->n_hs, s);
  launch_to_df(P->d_chirp, P->d_chf, P->n_ch, s);
  launch_to_df(P->d_B, P->d_Bf, P->n_B, s);
  WF_CUDA(cudaStreamSynchronize(s));
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// dynamic shared memory the table form of the Legendre kernel may use (with its
// static arrays within the 227 KB a CTA can have)
constexpr size_t kTabSmemLimit = 220 * 1024;

static wf_status build_legendre(Plan *P) {
  const int lmax = P->lmax;
  std::vector<double2> rec(alm_count(lmax));
  for (int m = 0; m <= lmax; ++m) {
    const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
    for (int l = m; l <= lmax; ++l) {
      double a = 0.0, b = 0.0;
      const double dl = l, dm = m;
      if (l == m + 1) {
        a = sqrt(2.0 * m + 3.0);
      } else if (l >= m + 2) {
        a = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
        b = a * sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
      }
      rec[base + l] = make_double2(a, b);
    }
  }
  wf_status st;
  const size_t nmk = (size_t)(lmax + 1) * P->RP;
  if ((st = P->dalloc((void **)&P->d_rec, sizeof(double2) * rec.size()))) return st;
  if ((st = P->dalloc((void **)&P->d_ls, sizeof(int) * nmk))) return st;
  if ((st = P->dalloc((void **)&P->d_sv, sizeof(double2) * nmk))) return st;
  if ((st = P->dalloc((void **)&P->d_dfA, sizeof(float2) * rec.size()))) return st;
  if ((st = P->dalloc((void **)&P->d_dfg, sizeof(double) * rec.size()))) return st;
  if ((st = P->dalloc((void **)&P->d_dfls, sizeof(int) * nmk))) return st;
  if ((st = P->dalloc((void **)&P->d_dfsv, sizeof(float4) * nmk))) return st;
  WF_CUDA(cudaMemcpyAsync(P->d_rec, rec.data(), sizeof(double2) * rec.size(), cudaMemcpyHostToDevice, P->stream));
  launch_start_values(P->d_x, P->d_rec, lmax, P->RP, P->d_ls, P->d_sv, P->stream);
  launch_df_tables(P->d_x, P->d_rec, lmax, P->RP, P->d_dfg, P->d_dfA, P->d_dfls, P->d_dfsv, P->stream);
  const size_t rows = lam_table_rows(lmax);
  const size_t tab_bytes = rows * (size_t)((P->RP + 31) / 32 * 32) * sizeof(float4);  // tiles of 32 ring pairs
  if (P->opt.precision == WF_PREC_FP64 && tab_bytes <= P->opt.legendre_table_bytes &&
      leg_tab_smem(lmax, P->RP) <= kTabSmemLimit) {
    std::vector<long long> poff(lmax + 1);
    long long r = 0;
    for (int m = 0; m <= lmax; ++m) { poff[m] = r; r += (lmax - m + 2) / 2; }
    if ((st = P->dalloc((void **)&P->d_poff, sizeof(long long) * poff.size()))) return st;
    if ((st = P->dalloc((void **)&P->d_tab, tab_bytes))) return st;
    WF_CUDA(cudaMemcpyAsync(P->d_poff, poff.data(), sizeof(long long) * poff.size(), cudaMemcpyHostToDevice,
                            P->stream));
    if (P->RP % 32) WF_CUDA(cudaMemsetAsync(P->d_tab, 0, tab_bytes, P->stream));  // columns past RP
    launch_lam_table(P->d_x, P->d_rec, P->d_ls, P->d_sv, P->d_dfls, P->d_poff, lmax, P->RP, P->d_tab, P->stream);
    P->tab_bytes = tab_bytes;
  }
  WF_CUDA(cudaStreamSynchronize(P->stream));
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status Plan::alloc_work() {
  wf_status st;
  const size_t nF = (size_t)(lmax + 1) * RP;
  if ((st = dalloc((void **)&d_FS, sizeof(double4_32a) * nF))) return st;
  if ((st = dalloc((void **)&d_FT, sizeof(double4_32a) * nF))) return st;
  if ((st = dalloc((void **)&d_ring_part, sizeof(double) * 2 * R))) return st;
  if ((st = dalloc((void **)&d_m_part, sizeof(double) * 3 * (lmax + 1)))) return st;
  if ((st = dalloc((void **)&d_ctl, sizeof(Ctl)))) return st;
  if ((st = dalloc((void **)&d_d, sizeof(double) * npix))) return st;
  if ((st = dalloc((void **)&d_s, sizeof(double2) * nalm))) return st;
  if ((st = dalloc((void **)&d_gain, sizeof(double) * npix))) return st;
  if ((st = dalloc((void **)&d_gainlam, sizeof(double) * R))) return st;
  if ((st = dalloc((void **)&d_ddf, sizeof(float2) * npix))) return st;
  if ((st = dalloc((void **)&d_wdf, sizeof(float2) * npix))) return st;
  if ((st = dalloc((void **)&d_gdf, sizeof(float2) * npix))) return st;
  if ((st = dalloc((void **)&d_gainlam_df, sizeof(double) * R))) return st;
  {
    std::vector<double> neg(R, -1.0);
    WF_CUDA(cudaMemcpy(d_gainlam, neg.data(), sizeof(double) * R, cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(d_gainlam_df, neg.data(), sizeof(double) * R, cudaMemcpyHostToDevice));
  }
  WF_CUDA(cudaMemsetAsync(d_ddf, 0, sizeof(float2) * npix, stream));
  WF_CUDA(cudaMemsetAsync(d_FS, 0, sizeof(double4_32a) * nF, stream));
  WF_CUDA(cudaMemsetAsync(d_FT, 0, sizeof(double4_32a) * nF, stream));
  WF_CUDA(cudaMallocHost((void **)&h_ctl, sizeof(Ctl)));
  WF_CUDA(cudaEventCreate(&ev0));
  WF_CUDA(cudaEventCreate(&ev1));
  return WF_OK;
}

wf_status Plan::ensure_hist(int cap) {
  if (cap <= hist_cap) return WF_OK;
  if (d_hist) {
    cudaFree(d_hist);
    for (auto &p : allocs)
      if (p == d_hist) p = nullptr;
  }
  d_hist = nullptr;
  hist_cap = 0;
  wf_status st = dalloc((void **)&d_hist, sizeof(wf_iter_record) * (size_t)cap);
  if (st) return st;
  hist_cap = cap;
  if (graph_exec) {  // the captured graph holds the old pointer
    cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
  }
  return WF_OK;
}

wf_status plan_rebind(Plan *P, const double *cl, const double *w, double tau, long long n_obs) {
  cudaStream_t s = P->stream;
  P->h_cl.assign(cl, cl + P->lmax + 1);
  P->tau = tau;
  P->n_obs = n_obs;
  std::vector<double> neg(P->R, -1.0);
  WF_CUDA(cudaMemcpyAsync(P->d_cl, cl, sizeof(double) * (P->lmax + 1), cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_w, w, sizeof(double) * P->npix, cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_gainlam, neg.data(), sizeof(double) * P->R, cudaMemcpyHostToDevice, s));
  WF_CUDA(cudaMemcpyAsync(P->d_gainlam_df, neg.data(), sizeof(double) * P->R, cudaMemcpyHostToDevice, s));
  launch_to_df2(P->d_w, P->d_wdf, P->npix, s);
  WF_CUDA(cudaStreamSynchronize(s));
  if (P->graph_exec) {  // the captured launches hold the old tau
    cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
  }
  P->fs_valid = false;
  return WF_OK;
}

RingArgs Plan::ring_args() const {
  RingArgs a{};
  a.rings = d_rings; a.order = d_order; a.porder = d_porder; a.first = 0; a.scratch = d_ring_scratch; a.tw = d_tw; a.logMmax = logMmax; a.hs = d_hs; a.chirp = d_chirp; a.B = d_B;
  a.FS = d_FS; a.FT = d_FT; a.RP = RP; a.d = d_d; a.w = d_w; a.ring_part = d_ring_part; a.ctl = d_ctl;
  a.lsht = lmax; a.omega = omega; a.tau = tau; a.gain = d_gain; a.gainlam = d_gainlam;
  return a;
}

LegArgs Plan::leg_args() const {
  LegArgs a{};
  a.x = d_x; a.rec = d_rec; a.ls = d_ls; a.sv = d_sv; a.cl = d_cl; a.FT = d_FT; a.FS = d_FS; a.alm = d_s;
  a.m_part = d_m_part; a.ctl = d_ctl; a.lsht = lmax; a.lmax = lmax; a.RP = RP; a.omega = omega; a.tau = tau;
  return a;
}

void Plan::enqueue_iteration(cudaStream_t s) {
  launch_rng(ring_args(), s, RING_ITER);
  launch_leg(leg_args(), s, LEG_ITER);
  launch_control(d_ctl, d_ring_part, R, d_m_part, lmax, d_cl, d_hist, hist_cap, s);
}

Ctl Plan::make_ctl(int mode, double lambda, int lsht, int n_fixed) const {
  Ctl c{};
  c.mode = mode;
  c.n_fixed = n_fixed;
  c.max_iter = opt.max_iter;
  c.cooling = opt.cooling;
  c.l_iter0 = opt.l_iter0;
  c.margin = opt.lmax_margin;
  c.band_limit = opt.band_limit;
  c.min_level_iters = opt.min_level_iters;
  c.max_level_iters = opt.max_level_iters;
  c.lmax = lmax;
  c.tol = opt.tol;
  c.plateau_eps = opt.plateau_eps;
  c.final_dchi2 = opt.final_dchi2;
  c.sigma_chi2 = sqrt(2.0 * (double)n_obs);
  c.tau = tau;
  c.omega = omega;
  c.lambda = lambda;
  c.lsht = lsht;
  c.l_iter = opt.l_iter0;
  return c;
}

double Plan::lambda_of(int l_iter) const {
  if (l_iter > lmax) return 1.0;
  const double r = h_cl[l_iter] / (tau * omega);
  return r > 1.0 ? r : 1.0;
}

}  // namespace wfk

using namespace wfk;

// ============================================================== C ABI

extern "C" {

const char *wf_last_error(void) { return g_err.c_str(); }

wf_status wf_options_default(wf_options *o) {
  if (!o) { set_error("wf_options_default: NULL"); return WF_EINVAL; }
  o->precision = WF_PREC_FP64;
  o->tol = 1e-6;
  o->max_iter = 10000;
  o->cooling = 1;
  o->l_iter0 = 20;
  o->lmax_margin = 100;
  o->band_limit = 1;
  o->plateau_eps = 1e-2;
  o->final_dchi2 = 0.0;
  o->min_level_iters = 3;
  o->max_level_iters = 1000;
  o->graph_iters = 16;
  o->batch_slots = kBatchMax;
  o->legendre_table_bytes = (size_t)8 << 30;
  o->posterior_grad = 1;
  o->synthesis_table = -1;
  o->refine_iters = 0;
  o->refine_tol = 0.0;
  o->stream = nullptr;
  return WF_OK;
}

static wf_status check_options(const wf_options *o) {
  if (o->precision != WF_PREC_FP64 && o->precision != WF_PREC_FP64_NATIVE && o->precision != WF_PREC_MIXED) {
    set_error("wf_options: unknown precision");
    return WF_EINVAL;
  }
  if (!(o->tol >= 0.0) || o->max_iter < 1 || o->l_iter0 < 1 || o->lmax_margin < 0 || o->min_level_iters < 1 ||
      o->max_level_iters < 1 || o->graph_iters < 1 || o->graph_iters > 1024 || o->batch_slots < 1 ||
      o->batch_slots > kBatchMax || !(o->plateau_eps >= 0.0) ||
      !(o->final_dchi2 >= 0.0) || o->refine_iters < 0 || !(o->refine_tol >= 0.0) || o->synthesis_table < -1 ||
      o->synthesis_table > 2 || (o->posterior_grad != 0 && o->posterior_grad != 1)) {
    set_error("wf_options: value out of range");
    return WF_EINVAL;
  }
  return WF_OK;
}

wf_status wf_plan_create(int nside, int lmax, const double *cl, const double *noise_var, const uint8_t *mask,
                         const wf_options *opt, wf_plan_t *out) {
  if (!out || !cl || !noise_var) { set_error("wf_plan_create: NULL argument"); return WF_EINVAL; }
  *out = nullptr;
  if (nside < 1 || nside > 2048 || (nside & (nside - 1)) != 0) {
    set_error("wf_plan_create: nside must be a power of two in [1, 2048]");
    return WF_EINVAL;
  }
  if (lmax < 0 || lmax > 4 * nside || lmax > 4096) {
    set_error("wf_plan_create: lmax must be in [0, min(4 nside, 4096)]");
    return WF_EINVAL;
  }
  wf_options o;
  wf_options_default(&o);
  if (opt) o = *opt;
  if (check_options(&o)) return WF_EINVAL;
  for (int l = 0; l <= lmax; ++l)
    if (!std::isfinite(cl[l]) || cl[l] < 0.0) { set_error("wf_plan_create: C_l must be finite and >= 0"); return WF_EINVAL; }
  const long long npix = 12LL * nside * nside;
  double tau = INFINITY;
  long long nobs = 0;
  std::vector<double> w(npix);
  for (long long p = 0; p < npix; ++p) {
    const bool obs = !mask || mask[p] != 0;
    if (!obs) { w[p] = 0.0; continue; }
    const double v = noise_var[p];
    if (!std::isfinite(v) || !(v > 0.0)) {
      set_error("wf_plan_create: noise variance must be finite and > 0 on observed pixels");
      return WF_EINVAL;
    }
    w[p] = 1.0 / v;
    if (v < tau) tau = v;
    ++nobs;
  }
  if (nobs == 0) { set_error("wf_plan_create: no observed pixel"); return WF_EINVAL; }

  Plan *P = new (std::nothrow) Plan();
  if (!P) { set_error("out of host memory"); return WF_ENOMEM; }
  P->nside = nside; P->lmax = lmax; P->npix = npix; P->nalm = (long long)alm_count(lmax);
  P->R = 4 * nside - 1; P->RP = 2 * nside;
  P->tau = tau; P->omega = 4.0 * M_PI / (double)npix; P->n_obs = nobs;
  P->opt = o;
  P->h_cl.assign(cl, cl + lmax + 1);
  wf_status st = WF_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { st = cuda_status(e, "cudaStreamCreate"); delete P; return st; }
  P->own_stream = true;
  if ((st = build_geometry(P)) || (st = build_legendre(P)) || (st = P->alloc_work()) ||
      (st = P->dalloc((void **)&P->d_w, sizeof(double) * npix)) ||
      (st = P->dalloc((void **)&P->d_cl, sizeof(double) * (lmax + 1)))) {
    delete P;
    return st;
  }
  e = cudaMemcpyAsync(P->d_w, w.data(), sizeof(double) * npix, cudaMemcpyHostToDevice, P->stream);
  if (e == cudaSuccess) {
    launch_to_df2(P->d_w, P->d_wdf, npix, P->stream);  // the double-float ring stage's copy
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->d_cl, cl, sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) { st = cuda_status(e, "plan upload"); delete P; return st; }
  if ((st = P->ensure_hist(o.max_iter + 1))) { delete P; return st; }
  *out = P;
  return WF_OK;
}

wf_status wf_plan_destroy(wf_plan_t plan) {
  if (!plan) return WF_OK;
  cudaStreamSynchronize(static_cast<Plan *>(plan)->stream);
  delete static_cast<Plan *>(plan);
  return WF_OK;
}

wf_status wf_plan_info(wf_plan_t plan, int64_t *npix, int64_t *nalm, double *tau, int64_t *n_obs,
                       size_t *device_bytes) {
  if (!plan) { set_error("wf_plan_info: NULL plan"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (npix) *npix = P->npix;
  if (nalm) *nalm = P->nalm;
  if (tau) *tau = P->tau;
  if (n_obs) *n_obs = P->n_obs;
  if (device_bytes) *device_bytes = P->device_bytes;
  return WF_OK;
}

wf_status wf_plan_kernels_per_iteration(wf_plan_t plan, int *n) {
  if (!plan || !n) { set_error("wf_plan_kernels_per_iteration: NULL argument"); return WF_EINVAL; }
  // the ring stage (one launch per single-solve ring class), Legendre stage, controller
  *n = (int)static_cast<const Plan *>(plan)->rsingle.size() + 2;
  return WF_OK;
}

wf_status wf_plan_legendre_terms(wf_plan_t plan, int lsht, int64_t *evaluated, int64_t *full) {
  if (!plan) { set_error("wf_plan_legendre_terms: NULL plan"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (lsht < 0 || lsht > P->lmax) { set_error("wf_plan_legendre_terms: lsht out of range"); return WF_EINVAL; }
  const size_t nmk = (size_t)(P->lmax + 1) * P->RP;
  std::vector<int> ls(nmk);
  WF_CUDA(cudaMemcpy(ls.data(), P->d_dfls, sizeof(int) * nmk, cudaMemcpyDeviceToHost));
  int64_t ev = 0;
  for (int m = 0; m <= lsht; ++m)
    for (int k = 0; k < P->RP; ++k) {
      const int l0 = ls[(size_t)m * P->RP + k];
      if (l0 <= lsht) ev += lsht - l0 + 1;
    }
  if (evaluated) *evaluated = ev;
  if (full) *full = (int64_t)(lsht + 1) * (lsht + 2) / 2 * P->RP;
  return WF_OK;
}

wf_status wf_plan_legendre_table(wf_plan_t plan, int lsht, int64_t *held, int64_t *per_pass) {
  if (!plan) { set_error("wf_plan_legendre_table: NULL plan"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (lsht < 0 || lsht > P->lmax) { set_error("wf_plan_legendre_table: lsht out of range"); return WF_EINVAL; }
  if (held) *held = (int64_t)P->tab_bytes;
  if (per_pass) {
    const size_t nmk = (size_t)(P->lmax + 1) * P->RP;
    std::vector<int> ls(nmk);
    WF_CUDA(cudaMemcpy(ls.data(), P->d_dfls, sizeof(int) * nmk, cudaMemcpyDeviceToHost));
    int64_t rows = 0;
    for (int m = 0; m <= lsht; ++m)
      for (int k = 0; k < P->RP; ++k) {
        const int l0 = ls[(size_t)m * P->RP + k];
        if (l0 <= lsht) rows += (lsht - m) / 2 - (l0 - m) / 2 + 1;
      }
    *per_pass = rows * (int64_t)sizeof(float4);
  }
  return WF_OK;
}

wf_status wf_plan_set_options(wf_plan_t plan, const wf_options *opt) {
  if (!plan || !opt) { set_error("wf_plan_set_options: NULL"); return WF_EINVAL; }
  if (check_options(opt)) return WF_EINVAL;
  Plan *P = static_cast<Plan *>(plan);
  // the captured iteration holds the kernels of the precision and the launch shape
  const bool regraph = opt->graph_iters != P->opt.graph_iters || opt->stream != P->opt.stream ||
                       opt->precision != P->opt.precision;
  P->opt = *opt;
  wf_status st = P->ensure_hist(opt->max_iter + 1);
  if (st) return st;
  if (regraph && P->graph_exec) {
    cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
  }
  return WF_OK;
}

wf_status wf_alm2map(wf_plan_t plan, int lsht, const double *alm_dev, double *map_dev) {
  if (!plan || !alm_dev || !map_dev) { set_error("wf_alm2map: NULL argument"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (lsht < 0 || lsht > P->lmax) { set_error("wf_alm2map: lsht out of range"); return WF_EINVAL; }
  cudaStream_t s = P->run_stream();
  LegArgs la = P->leg_args();
  la.lsht = lsht;
  la.alm_in = reinterpret_cast<const double2 *>(alm_dev);
  P->launch_leg(la, s,LEG_SYNTH);
  RingArgs ra = P->ring_args();
  ra.lsht = lsht;
  ra.map_out = map_dev;
  P->launch_rng(ra, s, RING_SYNTH);
  P->fs_valid = false;
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status wf_map2alm(wf_plan_t plan, int lsht, const double *map_dev, double *alm_dev) {
  if (!plan || !alm_dev || !map_dev) { set_error("wf_map2alm: NULL argument"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (lsht < 0 || lsht > P->lmax) { set_error("wf_map2alm: lsht out of range"); return WF_EINVAL; }
  cudaStream_t s = P->run_stream();
  RingArgs ra = P->ring_args();
  ra.lsht = lsht;
  ra.map_in = map_dev;
  P->launch_rng(ra, s, RING_ANALYSIS);
  LegArgs la = P->leg_args();
  la.lsht = lsht;
  la.alm = reinterpret_cast<double2 *>(alm_dev);
  P->launch_leg(la, s,LEG_ANALYSIS);
  P->fs_valid = false;
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status wf_iterate(wf_plan_t plan, const double *d_dev, double *s_dev, double lambda, int lsht, int niter,
                     int reset_state, wf_iter_record *records) {
  if (!plan || !d_dev || !s_dev) { set_error("wf_iterate: NULL argument"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (lsht < 0 || lsht > P->lmax || niter < 0 || !(lambda >= 1.0) || !std::isfinite(lambda)) {
    set_error("wf_iterate: lambda must be >= 1, 0 <= lsht <= lmax, niter >= 0");
    return WF_EINVAL;
  }
  if (niter == 0) return WF_OK;
  wf_status st = P->ensure_hist(niter + 1);
  if (st) return st;
  cudaStream_t s = P->run_stream();
  WF_CUDA(cudaMemcpyAsync(P->d_d, d_dev, sizeof(double) * P->npix, cudaMemcpyDeviceToDevice, s));
  P->stage_data(s);
  WF_CUDA(cudaMemcpyAsync(P->d_s, s_dev, sizeof(double2) * P->nalm, cudaMemcpyDeviceToDevice, s));
  if (reset_state || !P->fs_valid || P->fs_lsht != lsht) {
    LegArgs la = P->leg_args();
    la.lsht = lsht;
    la.alm_in = P->d_s;
    P->launch_leg(la, s,LEG_SYNTH);
  }
  Ctl c = P->make_ctl(0, lambda, lsht, niter);
  *P->h_ctl = c;
  WF_CUDA(cudaMemcpyAsync(P->d_ctl, P->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  for (int i = 0; i < niter; ++i) P->enqueue_iteration(s);
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaMemcpyAsync(s_dev, P->d_s, sizeof(double2) * P->nalm, cudaMemcpyDeviceToDevice, s));
  if (records)
    WF_CUDA(cudaMemcpyAsync(records, P->d_hist, sizeof(wf_iter_record) * niter, cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaMemcpyAsync(P->h_ctl, P->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  P->fs_valid = true;
  P->fs_lsht = lsht;
  if (P->h_ctl->numeric) { set_error("wf_iterate: chi^2 is not finite"); return WF_ENUMERIC; }
  return WF_OK;
}

wf_status wf_profile_iterations(wf_plan_t plan, const double *d_dev, double *s_dev, double lambda, int lsht,
                                int niter, float ms[3]) {
  if (!plan || !d_dev || !s_dev || !ms) { set_error("wf_profile_iterations: NULL argument"); return WF_EINVAL; }
  Plan *P = static_cast<Plan *>(plan);
  if (lsht < 0 || lsht > P->lmax || niter < 1 || !(lambda >= 1.0)) {
    set_error("wf_profile_iterations: bad lambda / lsht / niter");
    return WF_EINVAL;
  }
  wf_status st = P->ensure_hist(niter + 1);
  if (st) return st;
  cudaStream_t s = P->run_stream();
  WF_CUDA(cudaMemcpyAsync(P->d_d, d_dev, sizeof(double) * P->npix, cudaMemcpyDeviceToDevice, s));
  P->stage_data(s);
  WF_CUDA(cudaMemcpyAsync(P->d_s, s_dev, sizeof(double2) * P->nalm, cudaMemcpyDeviceToDevice, s));
  LegArgs la = P->leg_args();
  la.lsht = lsht;
  la.alm_in = P->d_s;
  P->launch_leg(la, s,LEG_SYNTH);
  Ctl c = P->make_ctl(0, lambda, lsht, niter);
  *P->h_ctl = c;
  WF_CUDA(cudaMemcpyAsync(P->d_ctl, P->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  std::vector<cudaEvent_t> ev(4 * niter);
  for (auto &e : ev) WF_CUDA(cudaEventCreate(&e));
  for (int i = 0; i < niter; ++i) {
    cudaEventRecord(ev[4 * i], s);
    P->launch_rng(P->ring_args(), s, RING_ITER);
    cudaEventRecord(ev[4 * i + 1], s);
    P->launch_leg(P->leg_args(), s, LEG_ITER);
    cudaEventRecord(ev[4 * i + 2], s);
    launch_control(P->d_ctl, P->d_ring_part, P->R, P->d_m_part, P->lmax, P->d_cl, P->d_hist, P->hist_cap, s);
    cudaEventRecord(ev[4 * i + 3], s);
  }
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaMemcpyAsync(s_dev, P->d_s, sizeof(double2) * P->nalm, cudaMemcpyDeviceToDevice, s));
  WF_CUDA(cudaStreamSynchronize(s));
  double acc[3] = {0, 0, 0};
  for (int i = 0; i < niter; ++i)
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[4 * i + k], ev[4 * i + k + 1]);
      acc[k] += t;
    }
  for (auto &e : ev) cudaEventDestroy(e);
  for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / niter);
  P->fs_valid = false;
  return WF_OK;
}

// rel_posterior_grad of the plan's state d_s against its data d_d (posterior.cu):
// synthesis, W (d - Y a) and W d, two analyses, per-m norms summed in order.
static wf_status posterior_grad(Plan *P, cudaStream_t s, double *rel) {
  const long long npix = P->npix, nalm = P->nalm;
  if (!P->d_pmap) {  // on first use: plans that never report it (mixed) do not hold the buffers
    wf_status st;
    if ((st = P->dalloc((void **)&P->d_pmap, sizeof(double) * 2 * npix))) return st;
    if ((st = P->dalloc((void **)&P->d_palm, sizeof(double2) * 2 * nalm))) return st;
    if ((st = P->dalloc((void **)&P->d_ppart, sizeof(double) * 2 * (P->lmax + 1)))) return st;
  }
  double *ya = P->d_pmap, *wd = P->d_pmap + npix;
  double2 *ta = P->d_palm, *tb = P->d_palm + nalm;
  LegArgs la = P->leg_args();
  la.lsht = P->lmax;
  la.alm_in = P->d_s;
  P->launch_leg(la, s, LEG_SYNTH);
  RingArgs ra = P->ring_args();
  ra.lsht = P->lmax;
  ra.map_out = ya;
  P->launch_rng(ra, s, RING_SYNTH);
  launch_posterior_maps(P->d_d, P->d_w, ya, wd, npix, s);
  for (int i = 0; i < 2; ++i) {
    ra.map_in = i ? wd : ya;
    P->launch_rng(ra, s, RING_ANALYSIS);
    la.alm = i ? tb : ta;
    P->launch_leg(la, s, LEG_ANALYSIS);
  }
  launch_posterior_norms(P->d_s, ta, tb, P->d_cl, P->lmax, 1.0 / P->omega, P->d_ppart, s);
  std::vector<double> part(2 * (P->lmax + 1));
  WF_CUDA(cudaMemcpyAsync(part.data(), P->d_ppart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  P->fs_valid = false;
  double rr = 0.0, bb = 0.0;
  for (int m = 0; m <= P->lmax; ++m) { rr += part[2 * m]; bb += part[2 * m + 1]; }
  *rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  return WF_OK;
}

static wf_status solve_impl(Plan *P, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                            const double *alm_init, wf_stats *stats, wf_iter_record *records, int max_records,
                            int *n_records);

}  // extern "C"

namespace wfk {

wf_status posterior_grad_plan(Plan *P, cudaStream_t s, double *rel) { return posterior_grad(P, s, rel); }

wf_status refine_fp64(Plan *P, const double *d, int d_on_device, const double *alm_dev, double *alm_out,
                      int alm_on_device, wf_stats *stats) {
  const wf_options saved = P->opt;
  if (P->graph_exec && P->graph_prec != WF_PREC_FP64) {  // a graph of other kernels
    cudaGraphExecDestroy(P->graph_exec);
    P->graph_exec = nullptr;
  }
  wf_status hs = P->ensure_hist(saved.refine_iters + 1);  // the last record is read back
  if (hs) return hs;
  P->opt.precision = WF_PREC_FP64;
  P->opt.cooling = 0;
  P->opt.max_iter = saved.refine_iters;
  P->opt.tol = saved.refine_tol;
  wf_stats rs{};
  wf_status st = solve_impl(P, d, d_on_device, alm_out, alm_on_device, alm_dev, &rs, nullptr, 0, nullptr);
  P->opt = saved;
  if (st == WF_ENOTCONVERGED) st = WF_OK;  // at most refine_iters iterations by design
  if (st == WF_OK && stats) {
    stats->iters += rs.iters;
    stats->converged = stats->converged || rs.converged;
    stats->lambda_final = 1.0;
    stats->lmax_sht_final = P->lmax;
    stats->chi2 = rs.chi2;
    stats->chi2_prior = rs.chi2_prior;
    stats->chi2_noise = rs.chi2_noise;
    stats->chi2_per_dof = rs.chi2_per_dof;
    stats->rel_increment = rs.rel_increment;
    stats->ms_device += rs.ms_device;
    stats->rel_posterior_grad = rs.rel_posterior_grad;
  }
  return st;
}

}  // namespace wfk

extern "C" {

static wf_status solve_impl(Plan *P, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                            const double *alm_init, wf_stats *stats, wf_iter_record *records, int max_records,
                            int *n_records) {
  if (P->opt.precision == WF_PREC_MIXED) {
    if (n_records) *n_records = 0;
    if (alm_init) { set_error("wf_solve: warm start is available on the FP64 paths only"); return WF_EINVAL; }
    return solve_mixed(P, 1, d, d_on_device, alm_out, alm_on_device, stats);
  }
  cudaStream_t s = P->run_stream();
  const auto kind_in = d_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  WF_CUDA(cudaEventRecord(P->ev0, s));
  WF_CUDA(cudaMemcpyAsync(P->d_d, d, sizeof(double) * P->npix, kind_in, s));
  P->stage_data(s);
  const double lam0 = P->opt.cooling ? P->lambda_of(P->opt.l_iter0) : 1.0;
  const int lb = P->opt.l_iter0 + P->opt.lmax_margin;
  const int lsht0 = (lam0 <= 1.0 || !P->opt.band_limit) ? P->lmax : (lb < P->lmax ? lb : P->lmax);
  if (alm_init) {  // host or device (the refinement of a mixed solve starts from device state)
    WF_CUDA(cudaMemcpyAsync(P->d_s, alm_init, sizeof(double2) * P->nalm, cudaMemcpyDefault, s));
    LegArgs la = P->leg_args();
    la.lsht = lsht0;
    la.alm_in = P->d_s;
    P->launch_leg(la, s,LEG_SYNTH);
  } else {
    WF_CUDA(cudaMemsetAsync(P->d_s, 0, sizeof(double2) * P->nalm, s));
    WF_CUDA(cudaMemsetAsync(P->d_FS, 0, sizeof(double4_32a) * (size_t)(P->lmax + 1) * P->RP, s));
  }
  Ctl c = P->make_ctl(1, lam0, lsht0, 0);
  *P->h_ctl = c;
  WF_CUDA(cudaMemcpyAsync(P->d_ctl, P->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  // one CUDA graph holds graph_iters iterations; the controller stops the rest early
  if (!P->graph_exec) {
    cudaGraph_t g;
    WF_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < P->opt.graph_iters; ++i) P->enqueue_iteration(s);
    WF_CUDA(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&P->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
    P->graph_prec = P->opt.precision;
  }
  const int max_launch = (P->opt.max_iter + P->opt.graph_iters - 1) / P->opt.graph_iters + 1;
  bool cancelled = false;
  for (int it = 0; it < max_launch; ++it) {
    WF_CUDA(cudaGraphLaunch(P->graph_exec, s));
    WF_CUDA(cudaMemcpyAsync(P->h_ctl, P->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    WF_CUDA(cudaStreamSynchronize(s));
    if (P->h_ctl->done) break;
    if (P->cancel && P->cancel->load()) { cancelled = true; break; }
  }
  if (cancelled) {
    P->fs_valid = false;
    set_error("wf_solve: cancelled");
    return WF_ECANCELLED;
  }
  const auto kind_out = alm_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  WF_CUDA(cudaMemcpyAsync(alm_out, P->d_s, sizeof(double2) * P->nalm, kind_out, s));
  WF_CUDA(cudaEventRecord(P->ev1, s));
  const Ctl fin = *P->h_ctl;
  wf_iter_record last{};
  if (fin.iter > 0)
    WF_CUDA(cudaMemcpyAsync(&last, P->d_hist + (fin.iter - 1), sizeof(last), cudaMemcpyDeviceToHost, s));
  int nrec = 0;
  if (records && max_records > 0) {
    nrec = fin.iter < max_records ? fin.iter : max_records;
    if (nrec > 0)
      WF_CUDA(cudaMemcpyAsync(records, P->d_hist, sizeof(wf_iter_record) * nrec, cudaMemcpyDeviceToHost, s));
  }
  WF_CUDA(cudaStreamSynchronize(s));
  if (n_records) *n_records = nrec;
  P->fs_valid = false;
  double rel_pg = -1.0;
  if (stats && P->opt.posterior_grad) {
    wf_status st = posterior_grad(P, s, &rel_pg);
    if (st) return st;
  }
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P->ev0, P->ev1);
    stats->iters = fin.iter;
    stats->converged = fin.converged;
    stats->levels = fin.level + 1;
    stats->lmax_sht_final = fin.lsht;
    stats->lambda_final = fin.lambda;
    stats->chi2_prior = last.chi2_prior;
    stats->chi2_noise = last.chi2_noise;
    stats->chi2 = last.chi2_prior + last.chi2_noise;
    stats->chi2_per_dof = stats->chi2 / (double)P->n_obs;
    stats->rel_increment = fin.last_rel;
    stats->ms_device = ms;
    stats->rel_posterior_grad = rel_pg;
  }
  if (fin.numeric) { set_error("wf_solve: chi^2 is not finite"); return WF_ENUMERIC; }
  if (!fin.converged) { set_error("wf_solve: max_iter reached before the stop rule"); return WF_ENOTCONVERGED; }
  return WF_OK;
}

wf_status wf_solve(wf_plan_t plan, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                   const double *alm_init, wf_stats *stats) {
  if (!plan || !d || !alm_out) { set_error("wf_solve: NULL argument"); return WF_EINVAL; }
  return solve_impl(static_cast<Plan *>(plan), d, d_on_device, alm_out, alm_on_device, alm_init, stats, nullptr, 0,
                    nullptr);
}

wf_status wf_solve_history(wf_plan_t plan, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                           wf_stats *stats, wf_iter_record *records, int max_records, int *n_records) {
  if (!plan || !d || !alm_out) { set_error("wf_solve_history: NULL argument"); return WF_EINVAL; }
  return solve_impl(static_cast<Plan *>(plan), d, d_on_device, alm_out, alm_on_device, nullptr, stats, records,
                    max_records, n_records);
}

}  // extern "C"
