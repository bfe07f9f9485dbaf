// Batched engine (host side) and the multi-right-hand-side entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "batch_engine.h"
#include "wf_internal.h"
#include "wf_plan.h"

namespace wfk {

#define ENG_CUDA(call)                                     \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);  \
  } while (0)

static size_t nalm_of(int lmax) { return (size_t)(lmax + 1) * (lmax + 2) / 2; }

static int n_par(int m, int p, int L) { return L >= m + p ? (L - m - p) / 2 + 1 : 0; }

// Work lists and offsets of the tensor-core Legendre stage: analysis tiles
// (m, parity, first i, first lamA row of (m, parity)), synthesis tiles (m,
// first ring pair), and the first 32-wide chunk of i of every (m, parity).
static void make_tc_lists(int lmax, int RPp, std::vector<int4> &ana, std::vector<int2> &syn, std::vector<int> &offTc,
                          int &nchunks) {
  ana.clear();
  syn.clear();
  offTc.assign(2 * (size_t)(lmax + 1), 0);
  nchunks = 0;
  size_t row = 0;
  for (int m = 0; m <= lmax; ++m) {
    for (int p = 0; p < 2; ++p) {
      const int np = n_par(m, p, lmax);
      offTc[2 * m + p] = nchunks;
      nchunks += (np + 31) / 32;
      for (int i0 = 0; i0 < np; i0 += 128) ana.push_back(make_int4(m, p, i0, (int)row));
      row += np;
    }
    for (int k0 = 0; k0 < RPp; k0 += 128) syn.push_back(make_int2(m, k0));
  }
}

static int round_up(int v, int q) { return (v + q - 1) / q * q; }

size_t Engine::bytes_needed(int nside, int lmax, int nslots, int mode) {
  const size_t RP = 2 * (size_t)nside, R = 4 * (size_t)nside - 1, npix = 12 * (size_t)nside * nside;
  const size_t RPp = (size_t)round_up((int)RP, 32);
  const size_t nalm = nalm_of(lmax), nF = (size_t)(lmax + 1) * RP;
  size_t ntiles = 0, nchunks = 0;
  for (int m = 0; m <= lmax; ++m)
    for (int p = 0; p < 2; ++p) {
      ntiles += (size_t)(n_par(m, p, lmax) + 127) / 128;
      nchunks += (size_t)(n_par(m, p, lmax) + 31) / 32;
    }
  const size_t B = (size_t)round_up(nslots, 8), L1 = (size_t)lmax + 1, Nc = 2 * B;
  const size_t tables = (nalm + 32 * nchunks) * RPp * sizeof(float) * (mode == 2 ? 2 : 1)     // lamA, lamT
                        + sizeof(float2) * (8 * (size_t)nside + 16 * (size_t)nside * nside);  // FP32 FFT tables
  const size_t operands = 3 * (L1 * 2 * RPp + 32 * nchunks) * Nc * sizeof(float);             // XT, SPT (3 parts)
  const size_t per_slot = 2 * nF * sizeof(float4)                                             // FS, FT
                          + nalm * (sizeof(double2) + sizeof(float4))                          // s, sdf
                          + npix * 2 * sizeof(float)                                           // (d, w) in FP32
                          + L1 * (sizeof(double) + sizeof(float2) + sizeof(float))              // C_l, filter tables
                          + R * 2 * sizeof(double) + ntiles * 3 * sizeof(double)                // partials
                          + sizeof(Ctl) + sizeof(wf_iter_record) + 8;
  return tables + operands + B * per_slot + npix * 2 * sizeof(double)  // d, w staging of one slot
         + (ntiles + L1 * RPp / 128 + 2 * L1) * 16;
}

wf_status Engine::dalloc(void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc (batched engine)");
  allocs.push_back(*p);
  device_bytes += bytes;
  return WF_OK;
}

Engine::~Engine() {
  if (stream) cudaStreamSynchronize(stream);
  if (graph) cudaGraphExecDestroy(graph);
  for (void *p : allocs) cudaFree(p);
  if (h_err) cudaFreeHost(h_err);
  if (h_ctl) cudaFreeHost(h_ctl);
  if (h_active) cudaFreeHost(h_active);
  if (h_last) cudaFreeHost(h_last);
}

BatchArgs Engine::args() const {
  BatchArgs a{};
  a.rings = geo->d_rings;
  a.order = geo->d_order;
  a.first = 0;
  a.twf = geo->d_twf; a.hsf = geo->d_hsf; a.chf = geo->d_chf; a.Bf = geo->d_Bf;
  a.tw2 = tw2; a.Bf2 = Bf2;
  a.logMmax = geo->logMmax;
  a.lmax = geo->lmax; a.RP = geo->RP; a.R = geo->R; a.B = B;
  a.npix = geo->npix; a.nalm = geo->nalm; a.omega = geo->omega;
  a.d = d; a.w = w; a.cl = cl; a.dw32 = dw32;
  a.s = s; a.sdf = sdf; a.alm_of_row = alm_of_row; a.fdf = fdf; a.icl = icl; a.FS = FS; a.FT = FT;
  a.ctl = ctl; a.active = active; a.ring_part = ring_part; a.m_part = m_part;
  a.ntiles = natiles; a.bstate = bstate; a.last = last;
  return a;
}

TcArgs Engine::tc_args() const {
  TcArgs t{};
  t.Nc = 2 * B;
  t.RPp = RPp;
  t.nkc = RPp / 32;
  t.atiles = atiles;
  t.natiles = natiles;
  t.stiles = tstiles;
  t.nstiles = ntstiles;
  t.offTc = offTc;
  t.XT = XT;
  t.SPT = SPT;
  t.err = err;
  t.tile0 = 0;
  t.qbase = 0;
  t.chunk_info = chunk_info;
  t.lamA = lamA;
  t.lamTs = lamTs;
  t.pre = pre ? 1 : 0;
  t.loA = pre ? (int)geo->nalm : 0;                    // rows of lamA's map
  t.loT = pre ? nchunks * RPp : 0;                     // rows of lamT's map
  return t;
}


wf_status Engine::create(Plan *shape_plan, int nslots, cudaStream_t s_, int max_mode) {
  geo = shape_plan;
  stream = s_;
  if (nslots < 1 || nslots > kBatchMax) { set_error("batched engine: slots must be in [1, 64]"); return WF_EINVAL; }
  B = round_up(nslots, 8);   // GEMM columns 2 B: a multiple of 16
  const int lmax = geo->lmax, RP = geo->RP, R = geo->R;
  const size_t nalm = geo->nalm, npix = geo->npix, nF = (size_t)(lmax + 1) * RP;
  RPp = round_up(RP, 32);
  const size_t Nc = 2 * (size_t)B;
  std::vector<int4> ana;
  std::vector<int2> syn;
  std::vector<int> off;
  make_tc_lists(lmax, RPp, ana, syn, off, nchunks);
  natiles = (int)ana.size();
  ntstiles = (int)syn.size();
  // operands in three tf32 parts (part-major within each 32-wide chunk)
  const size_t nXT = 3 * (size_t)(lmax + 1) * 2 * RPp * Nc, nSPT = 3 * (size_t)nchunks * 32 * Nc;
  wf_status st;
  // the synthesis-ordered table: resident, or rebuilt band by band of m from the
  // analysis table each iteration (half the table memory; Nside 2048 needs it);
  // mode 2 holds both tables split into their tf32 parts (twice the memory, no
  // split in the GEMMs). Auto: the largest mode up to max_mode that fits.
  int mode = geo->opt.synthesis_table;
  if (mode < 0) {
    size_t fr = 0, tot = 0;
    ENG_CUDA(cudaMemGetInfo(&fr, &tot));
    mode = 0;
    for (int md = std::min(max_mode, 2); md >= 1 && mode == 0; --md)
      if (bytes_needed(geo->nside, lmax, nslots, md) + ((size_t)1 << 30) <= fr) mode = md;
  }
  pre = mode == 2;
  const size_t tsplit = pre ? 2 : 1;
  std::vector<int4> cinfo;
  size_t band_chunks = 0;
  bands.clear();
  if (mode == 0) {
    size_t row = 0;
    std::vector<int> per_m(lmax + 1, 0);
    for (int m = 0; m <= lmax; ++m)
      for (int p = 0; p < 2; ++p) {
        const int np = n_par(m, p, lmax);
        for (int i0 = 0; i0 < np; i0 += 32) cinfo.push_back(make_int4((int)(row + i0), std::min(32, np - i0), m, 0));
        per_m[m] += (np + 31) / 32;
        row += np;
      }
    const int ntk = (RPp + 127) / 128;  // synthesis tiles per m
    size_t cap = std::max<size_t>(((size_t)nchunks + 7) / 8, (size_t)*std::max_element(per_m.begin(), per_m.end()));
    for (int m = 0; m <= lmax;) {
      SynBand bd{off[2 * m], 0, m * ntk, 0};
      size_t c = 0;
      int m1 = m;
      while (m1 <= lmax && (m1 == m || c + per_m[m1] <= cap)) c += per_m[m1++];
      bd.q1 = bd.q0 + (int)c;
      bd.tile1 = m1 * ntk;
      bands.push_back(bd);
      band_chunks = std::max(band_chunks, c);
      m = m1;
    }
  }
  if ((st = dalloc((void **)&lamA, sizeof(float) * tsplit * nalm * RPp)) ||
      (mode >= 1 && (st = dalloc((void **)&lamT, sizeof(float) * tsplit * (size_t)nchunks * 32 * RPp))) ||
      (mode == 0 && (st = dalloc((void **)&lamTs, sizeof(float) * band_chunks * 32 * RPp))) ||
      (mode == 0 && (st = dalloc((void **)&chunk_info, sizeof(int4) * cinfo.size()))) ||
      (st = dalloc((void **)&XT, sizeof(float) * nXT)) || (st = dalloc((void **)&SPT, sizeof(float) * nSPT)) ||
      (st = dalloc((void **)&atiles, sizeof(int4) * ana.size())) ||
      (st = dalloc((void **)&tstiles, sizeof(int2) * syn.size())) ||
      (st = dalloc((void **)&offTc, sizeof(int) * off.size())) || (st = dalloc((void **)&err, sizeof(int))) ||
      (st = dalloc((void **)&alm_of_row, sizeof(int) * nalm)) ||
      (st = dalloc((void **)&tw2, sizeof(float2) * std::max<long long>(geo->n_tw, 1))) ||
      (st = dalloc((void **)&Bf2, sizeof(float2) * std::max<long long>(geo->n_B, 1))) ||
      (st = dalloc((void **)&FS, sizeof(float4) * nF * B)) || (st = dalloc((void **)&FT, sizeof(float4) * nF * B)) ||
      (st = dalloc((void **)&d, sizeof(double) * npix)) || (st = dalloc((void **)&w, sizeof(double) * npix)) ||
      (st = dalloc((void **)&dw32, sizeof(float2) * npix * B)) ||
      (st = dalloc((void **)&cl, sizeof(double) * (lmax + 1) * B)) ||
      (st = dalloc((void **)&s, sizeof(double2) * nalm * B)) || (st = dalloc((void **)&sdf, sizeof(float4) * nalm * B)) ||
      (st = dalloc((void **)&fdf, sizeof(float2) * (lmax + 1) * B)) ||
      (st = dalloc((void **)&icl, sizeof(float) * (lmax + 1) * B)) || (st = dalloc((void **)&ctl, sizeof(Ctl) * B)) ||
      (st = dalloc((void **)&active, sizeof(int) * B)) ||
      (st = dalloc((void **)&ring_part, sizeof(double) * 2 * R * B)) ||
      (st = dalloc((void **)&m_part, sizeof(double) * 3 * (size_t)natiles * B)) ||
      (st = dalloc((void **)&bstate, sizeof(int) * 2)) || (st = dalloc((void **)&last, sizeof(wf_iter_record) * B)))
    return st;
  if (!make_tc_map(&maps.A, lamA, RPp, tsplit * nalm, 128) || !make_tc_map(&maps.X, XT, 32, nXT / 32, (unsigned)Nc) ||
      !make_tc_map(&maps.T, mode >= 1 ? lamT : lamTs, 32,
                   (mode >= 1 ? tsplit * (size_t)nchunks : band_chunks) * RPp, 128) ||
      !make_tc_map(&maps.S, SPT, 32, nSPT / 32, (unsigned)Nc)) {
    set_error("batched engine: cuTensorMapEncodeTiled failed");
    return WF_ECUDA;
  }
  ENG_CUDA(cudaMallocHost((void **)&h_ctl, sizeof(Ctl) * B));
  ENG_CUDA(cudaMallocHost((void **)&h_active, sizeof(int) * B));
  ENG_CUDA(cudaMallocHost((void **)&h_last, sizeof(wf_iter_record) * B));
  ENG_CUDA(cudaMallocHost((void **)&h_err, sizeof(int)));
  std::fill(h_active, h_active + B, 0);
  *h_err = 0;
  ENG_CUDA(cudaMemcpyAsync(atiles, ana.data(), sizeof(int4) * ana.size(), cudaMemcpyHostToDevice, stream));
  ENG_CUDA(cudaMemcpyAsync(tstiles, syn.data(), sizeof(int2) * syn.size(), cudaMemcpyHostToDevice, stream));
  ENG_CUDA(cudaMemcpyAsync(offTc, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, stream));
  if (mode == 0)
    ENG_CUDA(cudaMemcpyAsync(chunk_info, cinfo.data(), sizeof(int4) * cinfo.size(), cudaMemcpyHostToDevice, stream));
  {
    // state rows in the analysis table's order: (m, parity of l - m, (l - m) / 2)
    std::vector<int> a_of_r(nalm);
    size_t r = 0;
    for (int m = 0; m <= lmax; ++m)
      for (int p = 0; p < 2; ++p)
        for (int l = m + p; l <= lmax; l += 2) a_of_r[r++] = (int)((size_t)m * (2 * lmax + 1 - m) / 2 + l);
    ENG_CUDA(cudaMemcpyAsync(alm_of_row, a_of_r.data(), sizeof(int) * nalm, cudaMemcpyHostToDevice, stream));
    ENG_CUDA(cudaStreamSynchronize(stream));   // a_of_r and cinfo are released by then
  }
  launch_hi_table(geo->d_twf, tw2, geo->n_tw, stream);
  launch_hi_table(geo->d_Bf, Bf2, geo->n_B, stream);
  ENG_CUDA(cudaMemsetAsync(SPT, 0, sizeof(float) * nSPT, stream));
  ENG_CUDA(cudaMemsetAsync(dw32, 0, sizeof(float2) * npix * B, stream));
  ENG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), stream));
  ENG_CUDA(cudaMemsetAsync(FS, 0, sizeof(float4) * nF * B, stream));
  ENG_CUDA(cudaMemsetAsync(FT, 0, sizeof(float4) * nF * B, stream));
  ENG_CUDA(cudaMemsetAsync(s, 0, sizeof(double2) * nalm * B, stream));
  ENG_CUDA(cudaMemsetAsync(sdf, 0, sizeof(float4) * nalm * B, stream));
  ENG_CUDA(cudaMemsetAsync(fdf, 0, sizeof(float2) * (lmax + 1) * B, stream));
  ENG_CUDA(cudaMemsetAsync(icl, 0, sizeof(float) * (lmax + 1) * B, stream));
  ENG_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl) * B, stream));
  ENG_CUDA(cudaMemsetAsync(active, 0, sizeof(int) * B, stream));
  ENG_CUDA(cudaMemsetAsync(last, 0, sizeof(wf_iter_record) * B, stream));
  launch_lam_tc_tables(geo->d_x, geo->legdf_args(), lmax, RP, RPp, offTc, lamA, mode >= 1 ? lamT : nullptr, pre,
                       nalm * RPp, (size_t)nchunks * 32 * RPp, stream);
  launch_batch_state(args(), bstate, stream);
  ENG_CUDA(cudaGetLastError());
  ENG_CUDA(cudaStreamSynchronize(stream));
  return autotune();
}

wf_status Engine::autotune() {
  const int ncls = (int)geo->rclass.size();
  ring_groups.assign(ncls, 0);
  // every slot active on a full-band step (the data are zero)
  const Ctl c = geo->make_ctl(1, 1.0, geo->lmax, 0);
  for (int b = 0; b < B; ++b) { h_ctl[b] = c; h_active[b] = 1; }
  ENG_CUDA(cudaMemcpyAsync(ctl, h_ctl, sizeof(Ctl) * B, cudaMemcpyHostToDevice, stream));
  ENG_CUDA(cudaMemcpyAsync(active, h_active, sizeof(int) * B, cudaMemcpyHostToDevice, stream));
  launch_batch_state(args(), bstate, stream);
  cudaEvent_t e0, e1;
  ENG_CUDA(cudaEventCreate(&e0));
  ENG_CUDA(cudaEventCreate(&e1));
  const BatchArgs a = args();
  for (int k = 0; k < ncls; ++k) {
    const RingClass &rc = geo->rclass[k];
    float best = 0.f;
    for (int G = 2; G <= 8; G *= 2) {
      if (!batch_ring_group_ok(rc.logM, G)) continue;
      launch_batch_ring_class(a, rc, G, stream);   // warm-up
      cudaEventRecord(e0, stream);
      for (int r = 0; r < 3; ++r) launch_batch_ring_class(a, rc, G, stream);
      cudaEventRecord(e1, stream);
      ENG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ring_groups[k] == 0 || ms < best) { best = ms; ring_groups[k] = G; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // back to empty slots
  for (int b = 0; b < B; ++b) h_active[b] = 0;
  ENG_CUDA(cudaMemcpyAsync(active, h_active, sizeof(int) * B, cudaMemcpyHostToDevice, stream));
  ENG_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl) * B, stream));
  ENG_CUDA(cudaMemsetAsync(FT, 0, sizeof(float4) * (size_t)(geo->lmax + 1) * geo->RP * B, stream));
  launch_batch_state(args(), bstate, stream);
  ENG_CUDA(cudaGetLastError());
  ENG_CUDA(cudaStreamSynchronize(stream));
  return WF_OK;
}

wf_status Engine::load_slot(int b, const double *dsrc, int d_on_device, const double *wsrc_dev, const double *cl_host,
                            const Ctl &c) {
  const int lmax = geo->lmax;
  const size_t npix = geo->npix;
  launch_batch_zero_slot(args(), tc_args(), nchunks, b, stream);
  // d, w: one staging slot, converted into the slot's FP32 (d, w) in stream order
  ENG_CUDA(cudaMemcpyAsync(d, dsrc, sizeof(double) * npix,
                           d_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
  ENG_CUDA(cudaMemcpyAsync(w, wsrc_dev, sizeof(double) * npix, cudaMemcpyDeviceToDevice, stream));
  launch_batch_convert_slot(args(), b, stream);
  ENG_CUDA(cudaMemcpyAsync(cl + (size_t)b * (lmax + 1), cl_host, sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice,
                           stream));
  h_ctl[b] = c;
  ENG_CUDA(cudaMemcpyAsync(ctl + b, h_ctl + b, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
  h_active[b] = 1;
  ENG_CUDA(cudaMemcpyAsync(active + b, h_active + b, sizeof(int), cudaMemcpyHostToDevice, stream));
  return WF_OK;
}

wf_status Engine::load_slot_host(int b, const double *d_host, const double *w_host, const double *cl_host,
                                 const Ctl &c) {
  const int lmax = geo->lmax;
  const size_t npix = geo->npix;
  launch_batch_zero_slot(args(), tc_args(), nchunks, b, stream);
  ENG_CUDA(cudaMemcpyAsync(d, d_host, sizeof(double) * npix, cudaMemcpyHostToDevice, stream));
  ENG_CUDA(cudaMemcpyAsync(w, w_host, sizeof(double) * npix, cudaMemcpyHostToDevice, stream));
  launch_batch_convert_slot(args(), b, stream);
  ENG_CUDA(cudaMemcpyAsync(cl + (size_t)b * (lmax + 1), cl_host, sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice,
                           stream));
  h_ctl[b] = c;
  ENG_CUDA(cudaMemcpyAsync(ctl + b, h_ctl + b, sizeof(Ctl), cudaMemcpyHostToDevice, stream));
  h_active[b] = 1;
  ENG_CUDA(cudaMemcpyAsync(active + b, h_active + b, sizeof(int), cudaMemcpyHostToDevice, stream));
  return WF_OK;
}

wf_status Engine::release_slot(int b) {
  h_active[b] = 0;
  ENG_CUDA(cudaMemcpyAsync(active + b, h_active + b, sizeof(int), cudaMemcpyHostToDevice, stream));
  return WF_OK;
}

wf_status Engine::export_slot(int b) {
  launch_batch_export_slot(args(), b, stream);
  ENG_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status Engine::refresh_state() {
  launch_batch_state(args(), bstate, stream);
  ENG_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status Engine::step() {
  if (!graph) {
    cudaGraph_t g;
    ENG_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < graph_iters; ++i)
      launch_batch_iteration(args(), tc_args(), maps, geo->rclass.data(), (int)geo->rclass.size(),
                             ring_groups.empty() ? nullptr : ring_groups.data(), bstate, stream, bands.data(),
                             (int)bands.size());
    ENG_CUDA(cudaStreamEndCapture(stream, &g));
    cudaError_t e = cudaGraphInstantiate(&graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate (batched engine)");
  }
  ENG_CUDA(cudaGraphLaunch(graph, stream));
  ENG_CUDA(cudaMemcpyAsync(h_ctl, ctl, sizeof(Ctl) * B, cudaMemcpyDeviceToHost, stream));
  ENG_CUDA(cudaMemcpyAsync(h_last, last, sizeof(wf_iter_record) * B, cudaMemcpyDeviceToHost, stream));
  ENG_CUDA(cudaMemcpyAsync(h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  return WF_OK;
}

wf_status Engine::sync_host() {
  ENG_CUDA(cudaStreamSynchronize(stream));
  if (*h_err) {
    set_error("batched engine: a tensor-core pipeline wait timed out");
    return WF_ECUDA;
  }
  return WF_OK;
}

static void fill_stats(wf_stats *st, const Ctl &c, const wf_iter_record &r, long long n_obs, double ms) {
  if (!st) return;
  st->iters = c.iter;
  st->converged = c.converged;
  st->levels = c.level + 1;
  st->lmax_sht_final = c.lsht;
  st->lambda_final = c.lambda;
  st->chi2_prior = r.chi2_prior;
  st->chi2_noise = r.chi2_noise;
  st->chi2 = r.chi2_prior + r.chi2_noise;
  st->chi2_per_dof = st->chi2 / (double)n_obs;
  st->rel_increment = c.last_rel;
  st->ms_device = ms;
  st->rel_posterior_grad = -1.0;  // not computed on the mixed path
}

// Mixed-precision solves of nrhs data maps sharing the plan's C_l, noise and
// mask, streamed through the plan's batched engine: every slot that finishes
// is refilled with the next right-hand side before the next step.
wf_status solve_mixed(Plan *P, int nrhs, const double *dsrc, int d_on_device, double *alm_out, int alm_on_device,
                      wf_stats *stats) {
  const int want = std::min(nrhs, P->opt.batch_slots);
  // an engine serves every batch up to its slot count (rounded to 8): rebuilt only to grow
  if (!P->engine || P->engine->B < round_up(want, 8)) {
    delete P->engine;
    P->engine = new (std::nothrow) Engine();
    if (!P->engine) { set_error("out of host memory"); return WF_ENOMEM; }
    wf_status st = P->engine->create(P, want, P->run_stream());
    if (st) { delete P->engine; P->engine = nullptr; return st; }
  }
  Engine *E = P->engine;
  E->stream = P->run_stream();
  const double lam0 = P->opt.cooling ? P->lambda_of(P->opt.l_iter0) : 1.0;
  const int lb = P->opt.l_iter0 + P->opt.lmax_margin;
  const int lsht0 = (lam0 <= 1.0 || !P->opt.band_limit) ? P->lmax : std::min(lb, P->lmax);
  const Ctl c0 = P->make_ctl(1, lam0, lsht0, 0);
  std::vector<int> slot_of(E->B, -1);
  std::vector<std::chrono::steady_clock::time_point> t_in(E->B);
  int next = 0, finished = 0;
  bool any_not_conv = false, any_numeric = false;
  wf_status st;
  auto admit = [&](int b) -> wf_status {
    if (next >= nrhs) { slot_of[b] = -1; return WF_OK; }
    wf_status s2 = E->load_slot(b, dsrc + (size_t)next * P->npix, d_on_device, P->d_w, P->h_cl.data(), c0);
    if (s2) return s2;
    slot_of[b] = next++;
    t_in[b] = std::chrono::steady_clock::now();
    return WF_OK;
  };
  for (int b = 0; b < E->B; ++b)
    if ((st = admit(b))) return st;
  if ((st = E->refresh_state())) return st;
  const long long max_steps = (long long)nrhs * ((P->opt.max_iter + E->graph_iters - 1) / E->graph_iters + 2);
  for (long long it = 0; finished < nrhs && it < max_steps; ++it) {
    if ((st = E->step()) || (st = E->sync_host())) return st;
    bool changed = false;
    for (int b = 0; b < E->B; ++b) {
      if (slot_of[b] < 0 || !E->h_ctl[b].done) continue;
      const int i = slot_of[b];
      const double ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_in[b]).count();
      if ((st = E->export_slot(b))) return st;
      ENG_CUDA(cudaMemcpyAsync(alm_out + (size_t)i * 2 * P->nalm, E->s + (size_t)b * P->nalm,
                               sizeof(double2) * P->nalm,
                               alm_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, E->stream));
      wf_stats tmp{};
      wf_stats *sr = stats ? stats + i : &tmp;
      fill_stats(sr, E->h_ctl[b], E->h_last[b], P->n_obs, ms);
      any_numeric |= E->h_ctl[b].numeric != 0;
      if (P->opt.refine_iters > 0 && !E->h_ctl[b].numeric) {  // FP64 iterations from the mixed result
        const double *from = reinterpret_cast<const double *>(E->s + (size_t)b * P->nalm);
        if ((st = refine_fp64(P, dsrc + (size_t)i * P->npix, d_on_device, from, alm_out + (size_t)i * 2 * P->nalm,
                              alm_on_device, sr)))
          return st;
      }
      any_not_conv |= !sr->converged;
      if ((st = E->release_slot(b))) return st;
      ++finished;
      if ((st = admit(b))) return st;
      changed = true;
    }
    if (changed && (st = E->refresh_state())) return st;
  }
  if ((st = E->sync_host())) return st;
  if (finished < nrhs) { set_error("batched solve: step limit reached"); return WF_ENOTCONVERGED; }
  if (any_numeric) { set_error("batched solve: chi^2 is not finite"); return WF_ENUMERIC; }
  if (any_not_conv) { set_error("batched solve: max_iter reached before the stop rule"); return WF_ENOTCONVERGED; }
  return WF_OK;
}

}  // namespace wfk

using namespace wfk;

extern "C" wf_status wf_solve_batch(wf_plan_t plan, int nrhs, const double *d, int d_on_device, double *alm_out,
                                    int alm_on_device, wf_stats *stats) {
  if (!plan || !d || !alm_out || nrhs < 0) { set_error("wf_solve_batch: bad argument"); return WF_EINVAL; }
  if (nrhs == 0) return WF_OK;
  Plan *P = static_cast<Plan *>(plan);
  if (P->opt.precision == WF_PREC_MIXED)
    return solve_mixed(P, nrhs, d, d_on_device, alm_out, alm_on_device, stats);
  return solve_fp64_batch(P, nrhs, d, d_on_device, alm_out, alm_on_device, stats);
}
