// Serving loop: continuous batching of Wiener-filter requests.
//
// Requests of any (nside, lmax, C_l, noise, mask) arrive through wf_submit
// and never block on the GPU. A worker thread admits them:
//   - tol > 1e-7 (mixed precision): into a free slot of the batched engine of
//     their shape (one engine, stream and FP32 Lambda table per shape, created
//     on first use when its device-memory footprint fits the budget, evicted
//     when idle and the budget is needed). Every step advances all live slots
//     of an engine by a block of iterations; finished slots are harvested and
//     refilled before the next step, so a request that arrives while others
//     iterate joins at the next step with its own lambda schedule.
//   - tol <= 1e-7 (FP64 path): on kFp64Workers worker threads (shortest job
//     first, by Nside, unless a request has waited kFp64MaxWait), each solve on
//     a plan of its shape taken from a pool (created on first use within the
//     budget, re-pointed at the request's C_l, noise and mask by plan_rebind,
//     returned afterwards), so that geometry, Legendre and lambda tables stay
//     resident; the workers' streams overlap with each other and with the
//     engines' work on the device.
//   - a mixed request whose shape's engine has no live slot runs on the FP64
//     pool instead while two of its workers are free (one stays for the
//     requests that need FP64): the engine's tensor-core GEMMs stream
//     its whole FP32 table per iteration however few slots are live, which for
//     one request costs more than the FP64 single solve (Nside 512: about
//     3 ms against 1.7 ms per iteration), and the FP64 result meets any
//     tolerance. Under load the engines fill and batch as above.
// Latency is measured from wf_submit to the moment the result is on the host
// (wf_stats.ms_latency). wf_cancel drops a queued request, takes a running
// one out of its slot after the current step, or stops its FP64 solve after
// the current block of iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch_engine.h"
#include "wf_internal.h"
#include "wf_plan.h"

using namespace wfk;
using Clock = std::chrono::steady_clock;

namespace {

constexpr double kFp64Tol = 1e-7;
constexpr int kFp64Workers = 3;
constexpr auto kFp64MaxWait = std::chrono::seconds(20);

struct Request {
  uint64_t ticket = 0;
  int nside = 0, lmax = 0;
  double tol = 1e-6;
  std::vector<double> cl, noise, w, d;
  std::vector<uint8_t> mask;
  double tau = 0.0;
  long long n_obs = 0;
  Clock::time_point t_submit, t_slot;
  std::atomic<int> cancel{0};
  // result
  bool done = false;
  wf_status status = WF_OK;
  std::vector<double> alm;
  wf_stats stats{};
};

struct WarmTask {
  int nside = 0, lmax = 0;
  bool done = false;
  wf_status status = WF_OK;
};

struct IdlePlan {
  Plan *plan = nullptr;
  size_t bytes = 0;
  Clock::time_point last_used;
};

struct ShapeRunner {
  int nside = 0, lmax = 0;
  Plan *shape = nullptr;              // tables of the shape (unit noise)
  std::unique_ptr<Engine> engine;
  std::vector<std::shared_ptr<Request>> slot;  // request in each slot (or null)
  size_t bytes = 0;
  bool in_flight = false;             // a step launched and not yet harvested
  bool dirty = false;                 // slots changed since the live band limit was computed
  Clock::time_point last_used;
  ~ShapeRunner() {
    engine.reset();
    if (shape) wf_plan_destroy(shape);
  }
  int live() const {
    int n = 0;
    for (auto &r : slot) n += r != nullptr;
    return n;
  }
};

}  // namespace

struct wf_server_s {
  size_t budget = 0;
  int max_batch = 16;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<std::shared_ptr<Request>> pending;      // mixed requests not yet in a slot
  std::deque<std::shared_ptr<Request>> fp64_queue;   // FP64 requests
  std::deque<std::shared_ptr<WarmTask>> warm_queue;  // shapes whose engine the worker builds next
  std::map<uint64_t, std::shared_ptr<Request>> all;  // every uncollected request
  int in_flight = 0;                                 // submitted and not finished
  std::vector<double> latencies_ms;
  int64_t completed = 0;
  std::map<std::pair<int, int>, std::unique_ptr<ShapeRunner>> runners;  // worker thread only
  size_t fp64_bytes_in_use = 0;                      // every FP64 plan, busy or idle
  int fp64_busy = 0;                                 // FP64 workers solving
  std::map<std::pair<int, int>, std::vector<IdlePlan>> fp64_idle;  // FP64 plans not solving, per shape
  std::thread worker;
  std::vector<std::thread> fp64_workers;
  std::string worker_error;

  // caller holds mu
  void finish_locked(const std::shared_ptr<Request> &r) {
    r->done = true;
    r->stats.ms_latency = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    if (r->status == WF_ECANCELLED) {
      r->alm.clear();
    } else {
      latencies_ms.push_back(r->stats.ms_latency);
      ++completed;
    }
    --in_flight;
    cv_done.notify_all();
  }
  void finish(const std::shared_ptr<Request> &r) {
    std::lock_guard<std::mutex> lk(mu);
    finish_locked(r);
  }
};

namespace {

size_t engine_bytes(int nside, int lmax, int slots) {
  // engine buffers plus the shape plan's tables (about 70 bytes per (m, ring pair) entry)
  return Engine::bytes_needed(nside, lmax, slots) + (size_t)(lmax + 1) * 2 * nside * 72 + 64 * nside * (size_t)nside;
}

Ctl request_ctl(const Plan *shape, const Request &r) {
  wf_options o;
  wf_options_default(&o);
  Ctl c{};
  c.mode = 1;
  c.max_iter = o.max_iter;
  c.cooling = o.cooling;
  c.l_iter0 = o.l_iter0;
  c.margin = o.lmax_margin;
  c.band_limit = o.band_limit;
  c.min_level_iters = o.min_level_iters;
  c.max_level_iters = o.max_level_iters;
  c.lmax = r.lmax;
  c.tol = r.tol;
  c.plateau_eps = o.plateau_eps;
  c.final_dchi2 = o.final_dchi2;
  c.sigma_chi2 = std::sqrt(2.0 * (double)r.n_obs);
  c.tau = r.tau;
  c.omega = shape->omega;
  double lam = 1.0;
  if (o.cooling && o.l_iter0 <= r.lmax) lam = std::max(1.0, r.cl[o.l_iter0] / (r.tau * shape->omega));
  c.lambda = lam;
  const int lb = o.l_iter0 + o.lmax_margin;
  c.lsht = (lam <= 1.0 || !o.band_limit) ? r.lmax : std::min(lb, r.lmax);
  c.l_iter = o.l_iter0;
  return c;
}

// Options of the pool's FP64 plans: the defaults, with the precomputed lambda
// table allowed up to a fifth of the budget (at most 48 GiB, at least the
// default 8 GiB), so that on a large GPU the Nside 1024 plans (34 GB table)
// read the table instead of running the recurrence.
wf_options fp64_plan_options(size_t budget) {
  wf_options o;
  wf_options_default(&o);
  const size_t cap = size_t(48) << 30, fifth = budget / 5;
  o.legendre_table_bytes = std::max(o.legendre_table_bytes, std::min(cap, fifth));
  return o;
}

// an FP64 plan: its Fourier arrays (two 32-byte double-float complexes per (m,
// ring pair)), recurrence tables (40 bytes per (m, ring pair), 48 per a_lm), the
// per-pixel buffers and ring FFT tables (about 176 bytes per pixel in all), the
// posterior-gradient buffers, plus the precomputed lambda table when it is
// within the pool's limit
size_t fp64_bytes(size_t budget, int nside, int lmax) {
  const wf_options o = fp64_plan_options(budget);
  const size_t tab = lam_table_rows(lmax) * (size_t)((2 * nside + 31) / 32 * 32) * 16;
  const size_t npix = 12 * (size_t)nside * nside, nalm = (size_t)(lmax + 1) * (lmax + 2) / 2;
  const size_t nmk = (size_t)(lmax + 1) * 2 * nside;
  const size_t posterior = 2 * npix * sizeof(double) + 2 * nalm * 16;  // rel_posterior_grad buffers
  return nmk * (64 + 40) + nalm * 48 + npix * 176 + posterior + (tab <= o.legendre_table_bytes ? tab : 0);
}

size_t bytes_in_use(wf_server_s *S) {
  size_t b;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    b = S->fp64_bytes_in_use;
  }
  for (auto &kv : S->runners) b += kv.second->bytes;
  return b;
}

// Take the least recently used idle FP64 plan out of the pool (caller holds mu
// and destroys the plan without it); nullptr when none is idle.
Plan *evict_idle_fp64(wf_server_s *S) {
  auto best = S->fp64_idle.end();
  size_t bi = 0;
  for (auto it = S->fp64_idle.begin(); it != S->fp64_idle.end(); ++it)
    for (size_t i = 0; i < it->second.size(); ++i)
      if (best == S->fp64_idle.end() || it->second[i].last_used < best->second[bi].last_used) {
        best = it;
        bi = i;
      }
  if (best == S->fp64_idle.end()) return nullptr;
  Plan *p = best->second[bi].plan;
  S->fp64_bytes_in_use -= best->second[bi].bytes;
  best->second.erase(best->second.begin() + bi);
  return p;
}

// Find or create the runner of a shape within the budget (evicting idle ones).
ShapeRunner *runner_for(wf_server_s *S, int nside, int lmax) {
  auto key = std::make_pair(nside, lmax);
  auto it = S->runners.find(key);
  if (it != S->runners.end()) return it->second.get();
  const size_t need = engine_bytes(nside, lmax, S->max_batch);
  while (bytes_in_use(S) + need > S->budget) {
    // evict the least recently used idle runner
    auto victim = S->runners.end();
    for (auto jt = S->runners.begin(); jt != S->runners.end(); ++jt)
      if (jt->second->live() == 0 && !jt->second->in_flight &&
          (victim == S->runners.end() || jt->second->last_used < victim->second->last_used))
        victim = jt;
    if (victim == S->runners.end()) {
      Plan *p = nullptr;  // no idle runner: an idle FP64 plan gives its memory back
      {
        std::lock_guard<std::mutex> lk(S->mu);
        p = evict_idle_fp64(S);
      }
      if (!p) return nullptr;  // no room yet: wait for slots to free
      wf_plan_destroy(p);
      continue;
    }
    S->runners.erase(victim);
  }
  auto R = std::make_unique<ShapeRunner>();
  R->nside = nside;
  R->lmax = lmax;
  std::vector<double> unit(12LL * nside * nside, 1.0), cl(lmax + 1, 1.0);
  wf_plan_t p = nullptr;
  if (wf_plan_create(nside, lmax, cl.data(), unit.data(), nullptr, nullptr, &p) != WF_OK) return nullptr;
  R->shape = static_cast<Plan *>(p);
  R->engine = std::make_unique<Engine>();
  // tables kept unsplit (synthesis_table 1, or 0 when free memory is short): the budget counts them so
  if (R->engine->create(R->shape, S->max_batch, R->shape->stream, 1) != WF_OK) return nullptr;
  // iterations per engine step by shape, so that a step of any shape takes a few ms and a large shape's
  // step does not hold back the harvest of a small one (one iteration at Nside 1024 is ~30 ms)
  R->engine->graph_iters = nside <= 128 ? 32 : nside <= 256 ? 16 : nside <= 512 ? 4 : 1;
  R->slot.assign(S->max_batch, nullptr);
  R->bytes = need;
  R->last_used = Clock::now();
  ShapeRunner *raw = R.get();
  S->runners[key] = std::move(R);
  return raw;
}

void worker_loop(wf_server_s *S) {
  for (;;) {
    // admission
    std::vector<std::shared_ptr<Request>> take;
    std::vector<std::shared_ptr<WarmTask>> warm;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      bool busy = false;
      for (auto &kv : S->runners) busy |= kv.second->live() > 0 || kv.second->in_flight;
      if (!busy)
        S->cv.wait_for(lk, std::chrono::milliseconds(20),
                       [&] { return S->stop || !S->pending.empty() || !S->warm_queue.empty(); });
      if (S->stop) return;
      take.assign(S->pending.begin(), S->pending.end());
      S->pending.clear();
      warm.assign(S->warm_queue.begin(), S->warm_queue.end());
      S->warm_queue.clear();
    }
    for (auto &w : warm) {
      const wf_status st = runner_for(S, w->nside, w->lmax) ? WF_OK : WF_ENOMEM;
      std::lock_guard<std::mutex> lk(S->mu);
      w->status = st;
      w->done = true;
      S->cv_done.notify_all();
    }
    std::vector<std::shared_ptr<Request>> keep;
    for (auto &r : take) {
      if (r->cancel.load()) {
        r->status = WF_ECANCELLED;
        S->finish(r);
        continue;
      }
      {
        auto it = S->runners.find(std::make_pair(r->nside, r->lmax));
        const bool idle_engine = it == S->runners.end() || it->second->live() == 0;
        std::lock_guard<std::mutex> lk(S->mu);
        // one worker stays free for the requests that need FP64
        if (idle_engine && S->fp64_queue.empty() && S->fp64_busy < kFp64Workers - 1) {
          S->fp64_queue.push_back(r);  // a lone request: the FP64 single solve is faster
          S->cv.notify_all();
          continue;
        }
      }
      ShapeRunner *R = runner_for(S, r->nside, r->lmax);
      // a stepping engine is not loaded: its pending copy of the controllers to the host would
      // overwrite the new slot's host controller before that is copied to the device
      if (R && R->in_flight) { keep.push_back(r); continue; }
      int b = -1;
      if (R)
        for (int i = 0; i < (int)R->slot.size(); ++i)
          if (!R->slot[i]) { b = i; break; }
      if (!R || b < 0) { keep.push_back(r); continue; }
      const Ctl c = request_ctl(R->shape, *r);
      if (R->engine->load_slot_host(b, r->d.data(), r->w.data(), r->cl.data(), c) != WF_OK) {
        r->status = WF_ECUDA;
        S->finish(r);
        continue;
      }
      R->slot[b] = r;
      r->t_slot = Clock::now();
      R->dirty = true;
    }
    if (!keep.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->pending.insert(S->pending.begin(), keep.begin(), keep.end());
    }
    // launch a step of every engine with live slots that is not already stepping (their streams
    // overlap on the device), then harvest the engines whose step has finished; an engine still
    // stepping is left running, so small shapes are served while a large one works
    for (auto &kv : S->runners) {
      ShapeRunner *R = kv.second.get();
      if (R->live() == 0 || R->in_flight) continue;
      if (R->dirty) { R->engine->refresh_state(); R->dirty = false; }
      if (R->engine->step() == WF_OK) R->in_flight = true;
    }
    std::vector<ShapeRunner *> stepped;
    for (auto &kv : S->runners) {
      ShapeRunner *R = kv.second.get();
      if (R->in_flight && cudaStreamQuery(R->engine->stream) != cudaErrorNotReady) stepped.push_back(R);
    }
    if (stepped.empty()) {
      bool any = false;
      for (auto &kv : S->runners) any |= kv.second->in_flight;
      if (any) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    for (ShapeRunner *R : stepped) {
      R->in_flight = false;
      R->engine->sync_host();
      R->last_used = Clock::now();
      bool any = false;
      for (int b = 0; b < (int)R->slot.size(); ++b) {
        auto &r = R->slot[b];
        if (r && r->cancel.load()) {  // cancelled while in its slot: leave without a result
          r->status = WF_ECANCELLED;
          R->engine->release_slot(b);
          S->finish(r);
          r.reset();
          any = true;
          continue;
        }
        if (!r || !R->engine->h_ctl[b].done) continue;
        const Ctl &c = R->engine->h_ctl[b];
        const wf_iter_record &last = R->engine->h_last[b];
        r->alm.resize(2 * (size_t)R->shape->nalm);
        R->engine->export_slot(b);
        cudaMemcpyAsync(r->alm.data(), R->engine->s + (size_t)b * R->shape->nalm,
                        sizeof(double2) * R->shape->nalm, cudaMemcpyDeviceToHost, R->engine->stream);
        cudaStreamSynchronize(R->engine->stream);
        r->stats.iters = c.iter;
        r->stats.converged = c.converged;
        r->stats.levels = c.level + 1;
        r->stats.lmax_sht_final = c.lsht;
        r->stats.lambda_final = c.lambda;
        r->stats.chi2_prior = last.chi2_prior;
        r->stats.chi2_noise = last.chi2_noise;
        r->stats.chi2 = last.chi2_prior + last.chi2_noise;
        r->stats.chi2_per_dof = r->stats.chi2 / (double)r->n_obs;
        r->stats.rel_increment = c.last_rel;
        r->stats.ms_device = std::chrono::duration<double, std::milli>(Clock::now() - r->t_slot).count();
        r->stats.rel_posterior_grad = -1.0;  // not computed on the mixed path
        r->status = c.numeric ? WF_ENUMERIC : (c.converged ? WF_OK : WF_ENOTCONVERGED);
        R->engine->release_slot(b);
        S->finish(r);
        r.reset();
        any = true;
      }
      if (any) R->dirty = true;
    }
  }
}

void fp64_loop(wf_server_s *S) {
  for (;;) {
    std::shared_ptr<Request> r;
    Plan *plan = nullptr;
    size_t bytes = 0;
    std::vector<Plan *> victims;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return S->stop || !S->fp64_queue.empty(); });
      if (S->stop) return;
      if (S->fp64_queue.empty()) continue;
      // shortest job first (smallest Nside, then arrival), except that a request queued for more than
      // kFp64MaxWait goes first: small requests are not held behind minutes of large solves, and a
      // large one is not starved
      auto pick = S->fp64_queue.begin();
      const auto now = Clock::now();
      for (auto it = S->fp64_queue.begin(); it != S->fp64_queue.end(); ++it) {
        if (now - (*it)->t_submit > kFp64MaxWait) { pick = it; break; }
        if ((*it)->nside < (*pick)->nside) pick = it;
      }
      r = *pick;
      auto &idle = S->fp64_idle[std::make_pair(r->nside, r->lmax)];
      if (!idle.empty()) {  // a resident plan of the shape
        plan = idle.back().plan;
        bytes = idle.back().bytes;
        idle.pop_back();
      } else {
        bytes = fp64_bytes(S->budget, r->nside, r->lmax);
        while (S->fp64_bytes_in_use + bytes > S->budget)
          if (Plan *v = evict_idle_fp64(S)) victims.push_back(v);
          else break;
        if (S->fp64_bytes_in_use + bytes > S->budget) {  // wait for a plan to come back
          lk.unlock();
          for (Plan *v : victims) wf_plan_destroy(v);
          std::unique_lock<std::mutex> lk2(S->mu);
          S->cv.wait_for(lk2, std::chrono::milliseconds(20));
          continue;
        }
        S->fp64_bytes_in_use += bytes;
      }
      S->fp64_queue.erase(std::find(S->fp64_queue.begin(), S->fp64_queue.end(), r));
      ++S->fp64_busy;
    }
    for (Plan *v : victims) wf_plan_destroy(v);
    wf_options o = fp64_plan_options(S->budget);
    o.tol = r->tol;
    wf_status st = WF_OK;
    if (plan) {
      st = plan_rebind(plan, r->cl.data(), r->w.data(), r->tau, r->n_obs);
      if (st == WF_OK) st = wf_plan_set_options(plan, &o);
    } else {
      wf_plan_t p = nullptr;
      st = wf_plan_create(r->nside, r->lmax, r->cl.data(), r->noise.data(),
                          r->mask.empty() ? nullptr : r->mask.data(), &o, &p);
      plan = static_cast<Plan *>(p);
    }
    if (st == WF_OK) {
      r->alm.resize(2 * (size_t)(r->lmax + 1) * (r->lmax + 2) / 2);
      plan->cancel = &r->cancel;  // the solve stops after its current block of iterations once set
      st = wf_solve(plan, r->d.data(), 0, r->alm.data(), 0, nullptr, &r->stats);
      plan->cancel = nullptr;
    }
    r->status = st;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      --S->fp64_busy;
      if (plan && (st == WF_OK || st == WF_ENOTCONVERGED || st == WF_ENUMERIC || st == WF_ECANCELLED)) {
        S->fp64_idle[std::make_pair(r->nside, r->lmax)].push_back(IdlePlan{plan, bytes, Clock::now()});
        plan = nullptr;
      } else {
        S->fp64_bytes_in_use -= bytes;
      }
    }
    if (plan) wf_plan_destroy(plan);
    S->cv.notify_all();
    S->finish(r);
  }
}

}  // namespace

extern "C" {

wf_status wf_server_create(size_t hbm_budget_bytes, int max_batch, wf_server_t *out) {
  if (!out) { set_error("wf_server_create: NULL out"); return WF_EINVAL; }
  *out = nullptr;
  if (max_batch < 1 || max_batch > kBatchMax) { set_error("wf_server_create: max_batch must be in [1, 64]"); return WF_EINVAL; }
  size_t budget = hbm_budget_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return cuda_status(e, "cudaMemGetInfo");
    budget = (size_t)(0.9 * (double)fr);
  }
  wf_server_s *S = new (std::nothrow) wf_server_s();
  if (!S) { set_error("out of host memory"); return WF_ENOMEM; }
  S->budget = budget;
  S->max_batch = max_batch;
  S->worker = std::thread(worker_loop, S);
  for (int i = 0; i < kFp64Workers; ++i) S->fp64_workers.emplace_back(fp64_loop, S);
  *out = S;
  return WF_OK;
}

wf_status wf_submit(wf_server_t S, int nside, int lmax, const double *cl, const double *noise_var,
                    const uint8_t *mask, const double *d, double tol, uint64_t *ticket) {
  if (!S || !cl || !noise_var || !d || !ticket) { set_error("wf_submit: NULL argument"); return WF_EINVAL; }
  if (nside < 1 || nside > 1024 || (nside & (nside - 1)) != 0 || lmax < 0 || lmax > 4 * nside) {
    set_error("wf_submit: nside must be a power of two in [1, 1024] and 0 <= lmax <= 4 nside");
    return WF_EINVAL;
  }
  if (!(tol > 0.0) || !std::isfinite(tol)) { set_error("wf_submit: tol must be > 0"); return WF_EINVAL; }
  auto r = std::make_shared<Request>();
  const long long npix = 12LL * nside * nside;
  r->nside = nside;
  r->lmax = lmax;
  r->tol = tol;
  r->cl.assign(cl, cl + lmax + 1);
  for (double c : r->cl)
    if (!std::isfinite(c) || c < 0.0) { set_error("wf_submit: C_l must be finite and >= 0"); return WF_EINVAL; }
  r->noise.assign(noise_var, noise_var + npix);
  r->d.assign(d, d + npix);
  if (mask) r->mask.assign(mask, mask + npix);
  r->w.assign(npix, 0.0);
  double tau = INFINITY;
  for (long long p = 0; p < npix; ++p) {
    if (mask && !mask[p]) continue;
    const double v = noise_var[p];
    if (!std::isfinite(v) || !(v > 0.0)) {
      set_error("wf_submit: noise variance must be finite and > 0 on observed pixels");
      return WF_EINVAL;
    }
    r->w[p] = 1.0 / v;
    tau = std::min(tau, v);
    ++r->n_obs;
  }
  if (r->n_obs == 0) { set_error("wf_submit: no observed pixel"); return WF_EINVAL; }
  r->tau = tau;
  // a request no path of which fits the whole budget could never be admitted
  const bool fp64_fits = fp64_bytes(S->budget, nside, lmax) <= S->budget;
  const bool engine_fits = engine_bytes(nside, lmax, S->max_batch) <= S->budget;
  const bool to_fp64 = tol <= kFp64Tol || !engine_fits;
  if (to_fp64 && !fp64_fits) {
    set_error("wf_submit: the request's " + std::string(tol <= kFp64Tol ? "FP64 plan" : "engine and FP64 plan") +
              " exceed the server's HBM budget");
    return WF_ENOMEM;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    ++S->in_flight;
    if (to_fp64) S->fp64_queue.push_back(r);
    else S->pending.push_back(r);
  }
  S->cv.notify_all();
  *ticket = r->ticket;
  return WF_OK;
}

wf_status wf_poll(wf_server_t S, uint64_t ticket, int *done, double *alm_out, wf_stats *stats) {
  if (!S || !done) { set_error("wf_poll: NULL argument"); return WF_EINVAL; }
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { *done = 0; set_error("wf_poll: unknown ticket"); return WF_ENOTFOUND; }
    if (!it->second->done) { *done = 0; return WF_EBUSY; }
    r = it->second;
    S->all.erase(it);
  }
  *done = 1;
  if (alm_out && !r->alm.empty()) std::copy(r->alm.begin(), r->alm.end(), alm_out);
  if (stats) *stats = r->stats;
  if (r->status != WF_OK) set_error("wf_poll: request finished with an error status");
  return r->status;
}

wf_status wf_cancel(wf_server_t S, uint64_t ticket) {
  if (!S) { set_error("wf_cancel: NULL server"); return WF_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) { set_error("wf_cancel: unknown ticket"); return WF_ENOTFOUND; }
  std::shared_ptr<Request> r = it->second;
  if (r->done) { set_error("wf_cancel: the request had already finished"); return WF_EINVAL; }
  r->cancel.store(1);
  // still queued: drop it now; otherwise its worker ends it
  for (auto *q : {&S->pending, &S->fp64_queue}) {
    auto jt = std::find(q->begin(), q->end(), r);
    if (jt != q->end()) {
      q->erase(jt);
      r->status = WF_ECANCELLED;
      S->finish_locked(r);
      break;
    }
  }
  return WF_OK;
}

wf_status wf_server_warm(wf_server_t S, int nside, int lmax, int precision) {
  if (!S) { set_error("wf_server_warm: NULL server"); return WF_EINVAL; }
  if (nside < 1 || nside > 1024 || (nside & (nside - 1)) != 0 || lmax < 0 || lmax > 4 * nside) {
    set_error("wf_server_warm: nside must be a power of two in [1, 1024] and 0 <= lmax <= 4 nside");
    return WF_EINVAL;
  }
  if (precision == WF_PREC_MIXED) {
    auto w = std::make_shared<WarmTask>();
    w->nside = nside;
    w->lmax = lmax;
    std::unique_lock<std::mutex> lk(S->mu);
    S->warm_queue.push_back(w);
    S->cv.notify_all();
    S->cv_done.wait(lk, [&] { return w->done || S->stop; });
    if (!w->done) { set_error("wf_server_warm: the server is shutting down"); return WF_ECANCELLED; }
    if (w->status != WF_OK) set_error("wf_server_warm: the shape's engine does not fit the budget now");
    return w->status;
  }
  if (precision != WF_PREC_FP64) { set_error("wf_server_warm: precision must be WF_PREC_MIXED or WF_PREC_FP64"); return WF_EINVAL; }
  const size_t bytes = fp64_bytes(S->budget, nside, lmax);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fp64_bytes_in_use + bytes > S->budget) {
      set_error("wf_server_warm: an FP64 plan of the shape does not fit the budget now");
      return WF_ENOMEM;
    }
    S->fp64_bytes_in_use += bytes;
  }
  std::vector<double> unit(12LL * nside * nside, 1.0), cl(lmax + 1, 1.0);
  wf_plan_t p = nullptr;
  const wf_options o = fp64_plan_options(S->budget);
  const wf_status st = wf_plan_create(nside, lmax, cl.data(), unit.data(), nullptr, &o, &p);
  std::lock_guard<std::mutex> lk(S->mu);
  if (st != WF_OK) {
    S->fp64_bytes_in_use -= bytes;
    return st;
  }
  S->fp64_idle[std::make_pair(nside, lmax)].push_back(IdlePlan{static_cast<Plan *>(p), bytes, Clock::now()});
  return WF_OK;
}

wf_status wf_server_drain(wf_server_t S, int timeout_ms) {
  if (!S) { set_error("wf_server_drain: NULL server"); return WF_EINVAL; }
  std::unique_lock<std::mutex> lk(S->mu);
  const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                      [&] { return S->in_flight == 0; });
  if (!ok) { set_error("wf_server_drain: timed out"); return WF_ETIMEOUT; }
  return WF_OK;
}

wf_status wf_server_stats(wf_server_t S, double *p50_ms, double *p99_ms, int64_t *completed) {
  if (!S) { set_error("wf_server_stats: NULL server"); return WF_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->latencies_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)std::ceil(q * (double)v.size()) - (q > 0 ? 1 : 0));
    return v[i];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (completed) *completed = S->completed;
  return WF_OK;
}

wf_status wf_server_destroy(wf_server_t S) {
  if (!S) return WF_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  S->cv_done.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &t : S->fp64_workers)
    if (t.joinable()) t.join();
  S->runners.clear();
  for (auto &kv : S->fp64_idle)
    for (auto &ip : kv.second) wf_plan_destroy(ip.plan);
  delete S;
  return WF_OK;
}

}  // extern "C"
