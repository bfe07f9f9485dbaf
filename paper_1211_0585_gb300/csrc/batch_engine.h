// Host side of the batched engine: B slots of one (nside, lmax) shape that
// advance one messenger iteration per step, each with its own data, noise,
// mask, C_l and schedule. Slots are filled and emptied between graph launches,
// so a finished solve frees its slot for the next one while the others keep
// iterating (continuous batching).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "wf_internal.h"
#include "wf_plan.h"

namespace wfk {

// TMA descriptors of the tensor-core Legendre stage (batch_tc.cu)
struct TcMaps {
  CUtensorMap A, X, T, S;    // lamA, XT, lamT, SPT
};

bool make_tc_map(CUtensorMap *map, const float *base, unsigned long long inner, unsigned long long rows,
                 unsigned box_rows);
// which = 0: FT -> XT and the analysis GEMM with Eq. 4; 1: the synthesis GEMM (with a
// streamed synthesis table, band by band)
void launch_batch_gemms_tc(const BatchArgs &a, const TcArgs &t, const TcMaps &maps, cudaStream_t s, int which,
                           const SynBand *bands, int nbands);

struct Engine {
  Plan *geo = nullptr;  // tables of the shape (not owned)
  int B = 0;
  int graph_iters = 4;
  cudaStream_t stream = nullptr;
  size_t device_bytes = 0;
  std::vector<void *> allocs;

  float2 *tw2 = nullptr, *Bf2 = nullptr;   // FP32 twiddle / Bluestein tables
  // tensor-core Legendre stage
  float *lamA = nullptr, *lamT = nullptr, *XT = nullptr, *SPT = nullptr;
  // streamed synthesis table (when both tables do not fit): scratch for one band of m at a time
  float *lamTs = nullptr;
  int4 *chunk_info = nullptr;
  std::vector<SynBand> bands;
  int4 *atiles = nullptr;
  int2 *tstiles = nullptr;
  int *offTc = nullptr;
  int *alm_of_row = nullptr;
  int *err = nullptr, *h_err = nullptr;
  int natiles = 0, ntstiles = 0, nchunks = 0, RPp = 0;
  bool pre = false;   // tables held split into their tf32 parts (synthesis_table mode 2)
  TcMaps maps{};
  std::vector<int> ring_groups;   // slots per ring-stage CTA of each ring class (autotuned)
  float4 *FS = nullptr, *FT = nullptr;
  double *d = nullptr, *w = nullptr, *cl = nullptr;
  float2 *dw32 = nullptr;   // [B][npix] (d, w) in FP32 for the ring stage
  double2 *s = nullptr;      // exported a_lm of finished slots
  float4 *sdf = nullptr;     // double-float state
  float2 *fdf = nullptr;
  float *icl = nullptr;
  Ctl *ctl = nullptr;
  int *active = nullptr;
  double *ring_part = nullptr, *m_part = nullptr;
  int *bstate = nullptr;
  wf_iter_record *last = nullptr;
  // pinned host mirrors
  Ctl *h_ctl = nullptr;
  int *h_active = nullptr;
  wf_iter_record *h_last = nullptr;
  cudaGraphExec_t graph = nullptr;

  ~Engine();
  // max_mode: the largest synthesis_table mode an automatic choice may take (2: split tables)
  wf_status create(Plan *shape_plan, int nslots, cudaStream_t s, int max_mode = 2);
  BatchArgs args() const;
  TcArgs tc_args() const;
  wf_status dalloc(void **p, size_t bytes);
  // Load one problem into slot b (device state zeroed, controller initialised).
  //   dsrc: [npix] data (host or device), wsrc: [npix] inverse noise (device),
  //   clsrc: [lmax+1] (host), c: controller configuration for this request.
  wf_status load_slot(int b, const double *dsrc, int d_on_device, const double *wsrc_dev, const double *cl_host,
                      const Ctl &c);
  // As load_slot, with the inverse noise given on the host (serving).
  wf_status load_slot_host(int b, const double *d_host, const double *w_host, const double *cl_host, const Ctl &c);
  wf_status refresh_state();           // recompute the live band limit after slots changed
  // Time every admissible slot group of each ring class on a full-band step of
  // all slots (zero data) and keep the fastest; the slots are reset after.
  wf_status autotune();
  wf_status step();                    // one graph launch (graph_iters iterations), then mirror ctl to host
  wf_status sync_host();               // wait for the last step's mirrors
  wf_status release_slot(int b);
  // Write slot b's double-float state as double a_lm into s + b nalm (stream-ordered).
  wf_status export_slot(int b);
  // device bytes of an engine whose synthesis table is in `mode` (0 and 1 are sized as 1)
  static size_t bytes_needed(int nside, int lmax, int nslots, int mode = 1);
};

}  // namespace wfk
