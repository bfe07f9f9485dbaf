// Internal declarations of the GB300 messenger-field Wiener filter library.
// Device data layout (one plan = one HEALPix nside and one lmax):
//   rings      R  = 4 nside - 1, north to south; ring pairs RP = 2 nside
//              (pair k = north ring k and south ring R-1-k; the equator ring
//              2 nside - 1 is a pair of its own, its south slot unused).
//   Fourier    F[m * RP + k] = double4_32a (north re, north im, south re, south im),
//              m = 0 .. lmax, the azimuthal coefficients of ring pair k.
//              FS: synthesis side (from a_lm), FT: analysis side (to a_lm).
//   a_lm       m-major complex doubles, index(l, m) = m (2 lmax + 1 - m) / 2 + l.
//   maps       RING order doubles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/wf.h"

namespace wfk {

constexpr int kThreads = 256;       // block size of the per-m Legendre kernels
constexpr int kRingThreads = 512;   // block size of the ring (FFT) kernels: one CTA per ring fills
                                    // an SM's shared memory, so its own warps must hide the latency
constexpr int kLB = 16;             // l values per block of the analysis reduction
constexpr int kStartExp = -100;     // Legendre terms below 2^-100 are not evaluated

// Per-ring description (host-built, read by the ring kernel).
struct RingDev {
  long long off;      // first pixel (RING index)
  int n;              // pixels in the ring (nphi)
  int pair;           // ring pair index k
  int side;           // 0 = north slot, 1 = south slot of the pair
  int shifted;        // first pixel at phi = pi / n (else at phi = 0)
  int logM;           // log2 of the FFT size (n itself, or the Bluestein size)
  int blue;           // 1: n is not a power of two, Bluestein convolution of size M
  long long hs_off;   // offset of this ring length's half-shift table e^{i pi q / n}
  long long ch_off;   // offset of this ring length's chirp e^{-i pi j^2 / n} (Bluestein only)
  long long B_off;    // offset of this ring length's Bluestein filter (bit-reversed, / M)
};

// Rings grouped by FFT size for the ring-stage launches: each class is one
// launch whose shared memory is sized for its own largest FFT (instead of the
// plan's largest), so the many rings with small or power-of-two FFTs run more
// CTAs per SM. order[first .. first + count) lists the class's rings, the two
// rings of a pair next to each other so that the halves of each Fourier
// coefficient record are read and written close together in time.
struct RingClass {
  int logM;    // the largest log2 FFT size in the class
  int first;   // offset into the ring order
  int count;   // rings in the class
  int global;  // 1: the class's FFT buffers do not fit shared memory and live in a global
               //    scratch array, 2^logM 16-byte elements per CTA (CTA i of the class at i 2^logM)
};

// Largest dynamic shared memory a ring-stage CTA asks for (of the 227 KB a CTA
// may use on this GPU; the rest is left for static arrays).
constexpr size_t kRingSmemLimit = 200 * 1024;

// Iteration controller state, resident on the device (Sect. 3 schedule).
struct Ctl {
  // configuration
  int mode;             // 0: fixed lambda and lsht for n_fixed iterations; 1: cooling schedule
  int n_fixed;
  int max_iter;
  int cooling, l_iter0, margin, band_limit, min_level_iters, max_level_iters;
  int lmax;
  double tol, plateau_eps, final_dchi2, sigma_chi2, tau, omega;
  // live state
  double lambda;
  int lsht, l_iter, level, level_iters, iter, done, converged, numeric;
  int have_prev;
  double prev_chi2;
  double last_rel;
};

// Record layout of one iteration (mirrors wf_iter_record).
static_assert(sizeof(wf_iter_record) == 6 * 8 + 2 * 4, "record layout");

struct Plan;

// ---------------------------------------------------------------- launches
// ring kernel modes
enum { RING_SYNTH = 0, RING_ANALYSIS = 1, RING_ITER = 2 };
// Legendre kernel modes
enum { LEG_SYNTH = 0, LEG_ANALYSIS = 1, LEG_ITER = 2 };

struct RingArgs {
  const RingDev *rings;
  const int *order;       // ring of CTA i is order[first + i] (nullptr: first + i)
  const int2 *porder;     // double-float ring stage: (north ring, south ring or -1) of CTA i at porder[first + i]
  int first;
  void *scratch;          // global FFT buffers of a class that does not fit shared memory (else nullptr)
  const double2 *tw;      // e^{-2 pi i k / Mmax}, k < Mmax / 2
  int logMmax;
  const double2 *hs, *chirp, *B;
  const double4_32a *FS;      // synthesis input (RING_SYNTH / RING_ITER)
  double4_32a *FT;            // analysis output (RING_ANALYSIS / RING_ITER)
  int RP;
  const double *map_in;   // RING_ANALYSIS input
  double *map_out;        // RING_SYNTH output
  const double *d, *w;    // RING_ITER: data, inverse noise (0 = masked)
  double *ring_part;      // RING_ITER: [R][2] chi2_N, chi2_lambda_N partials
  const Ctl *ctl;         // RING_ITER: lambda, lsht, done
  int lsht;               // standalone modes
  double omega, tau;
  double *gain;           // [npix] cached w / (1 + (lambda - 1) tau w) (double-float ring kernel)
  double *gainlam;        // [R] lambda the cached gains of each ring belong to (-1: none)
  const Ctl *gate;        // RING_SYNTH / RING_ANALYSIS inside a controlled iteration: skip once gate->done
};

struct LegArgs {
  const double *x;        // [RP] cos(theta) of the north ring of each pair
  const double2 *rec;     // [nalm] recurrence coefficients (a_l, b_l)
  const int *ls;          // [(lmax+1) RP] first evaluated l
  const double2 *sv;      // [(lmax+1) RP] (lambda_{ls}, lambda_{ls+1})
  const double *cl;       // [lmax+1]
  const double4_32a *FT;      // analysis input
  double4_32a *FS;            // synthesis output
  double2 *alm;           // state / output a_lm
  const double2 *alm_in;  // LEG_SYNTH input
  double *m_part;         // LEG_ITER: [lmax+1][3] chi2_S, incr2, norm2
  const Ctl *ctl;
  const Ctl *gate;        // LEG_SYNTH / LEG_ANALYSIS inside a controlled iteration: skip once gate->done
                          // (nullptr for the standalone transforms)
  int lsht, lmax, RP;
  double omega, tau;
};

// Tables of the double-float Legendre kernel (legendre_df.cu).
struct LegDfArgs {
  const float2 *A;        // [nalm] rescaled recurrence coefficient A_l (hi, lo)
  const double *g;        // [nalm] rescaling factor g_l (lambda = g mu)
  const int *ls;          // [(lmax+1) RP] first evaluated l (|lambda| >= 2^-60)
  const float4 *sv;       // [(lmax+1) RP] mu_{ls} (hi, lo), mu_{ls+1} (hi, lo)
  const float4 *tab;      // precomputed lambda (hi, lo) in rows of two l, or nullptr (recurrence)
  const long long *poff;  // [lmax+1] first table row of each m
};

// Per-map buffers of the batched FP64 Legendre stage (legendre_batch.cu): up to
// kLegBatchMax maps of one shape, each with its own Fourier arrays, state, C_l,
// tau, partial sums and controller.
constexpr int kLegBatchMax = 2;
constexpr int kSynRowsB = 4;      // batched synthesis: table rows per load batch
struct LegBatchMaps {
  int n;                          // maps in use (the rest are skipped)
  const double4_32a *FT[kLegBatchMax];
  double4_32a *FS[kLegBatchMax];
  double2 *alm[kLegBatchMax];
  double *m_part[kLegBatchMax];
  const Ctl *ctl[kLegBatchMax];
  const double *cl[kLegBatchMax];
  double tau[kLegBatchMax];
};
size_t leg_batch_smem(int nb, int lmax, int RP);
// mode: LEG_ITER (NB independent iterations), LEG_SYNTH or LEG_ANALYSIS (NB maps' transforms, a_lm in / t_l out
// through Bm.alm); the table form only
void launch_legendre_batch(const LegArgs &a, const LegDfArgs &d, const LegBatchMaps &bm, int nb, cudaStream_t s,
                           int mode = LEG_ITER);

// Double-float copies of the ring-stage tables (ring_df.cu): float4 =
// (re hi, re lo, im hi, im lo).
struct RingDfArgs {
  const float4 *tw, *hs, *chirp, *B;
  const float2 *d, *w;    // [npix] data and inverse noise as double-float (RING_ITER)
  float2 *gain;           // [npix] cached Eq. 3 gains as double-float
  double *gainlam;        // [R] lambda the cached gains of each ring belong to (-1: none)
};
void launch_to_df2(const double *src, float2 *dst, long long n, cudaStream_t s);

// Batched engine (batch_kernels.cu): B slots of one shape in lockstep.
constexpr int kBatchMax = 64;

struct BatchArgs {
  const RingDev *rings;
  const int *order;          // ring of ring-stage CTA i is order[first + i]
  int first;
  const float4 *twf, *hsf, *chf, *Bf;
  const float2 *tw2, *Bf2;   // FP32 twiddle and Bluestein filter tables (hi parts of twf, Bf)
  int logMmax;
  int lmax, RP, R, B;
  long long npix, nalm;
  double omega;
  const double *d, *w, *cl;  // [B][npix], [B][npix], [B][lmax+1]
  float2 *dw32;              // [B][npix] (d, w) in FP32, read by the mixed-precision ring stage
  double2 *s;                // [B][nalm] exported a_lm of finished slots
  float4 *sdf;               // [B][nalm] state, double-float (re hi, re lo, im hi, im lo), in the
                             // order of the analysis table rows: (m, parity of l - m, (l - m) / 2)
  const int *alm_of_row;     // [nalm] a_lm index m (2 lmax + 1 - m) / 2 + l of each state row
  float2 *fdf;               // [lmax+1][B] Eq. 4 filter f_l(lambda_b) of this iteration, double-float
  float *icl;                // [lmax+1][B] 1 / C_l (0 where C_l = 0)
  float4 *FS, *FT;           // [(m RP + k) B + b] (north re, north im, south re, south im)
  Ctl *ctl;                  // [B]
  const int *active;         // [B]
  double *ring_part;         // [B][R][2]
  double *m_part;            // [B][ntiles][3]
  int ntiles;                // analysis tiles (partials per slot)
  const int *bstate;         // [0] largest live band limit, [1] live slots
  wf_iter_record *last;      // [B]
};

// Tensor-core Legendre stage of the batched engine (batch_tc.cu): work lists,
// per-iteration operands and the error flag of the bounded pipeline waits.
struct TcArgs {
  int Nc;                    // GEMM columns: 2 B (re, im of every slot), a multiple of 16
  int RPp, nkc;              // ring pairs padded to a multiple of 32, and RPp / 32
  const int4 *atiles;        // analysis tiles (m, parity, first i, first lamA row of (m, parity))
  int natiles;
  const int2 *stiles;        // synthesis tiles (m, first ring pair)
  int nstiles;
  const int *offTc;          // [2 (lmax+1)] first 32-wide i chunk of (m, parity)
  float *XT, *SPT;           // analysis / synthesis B operands
  int *err;                  // set when a pipeline wait gave up
  // streamed synthesis table: a launch covers synthesis tiles from tile0 and reads the
  // synthesis-ordered rows of chunks from qbase, rebuilt from lamA into a scratch array
  int tile0, qbase;
  const int4 *chunk_info;    // [nchunks] (first lamA row of the chunk, rows in it, m, 0)
  const float *lamA;
  float *lamTs;              // scratch of the streamed synthesis table (nullptr: resident lamT)
  // split tables: lamA and lamT hold th in their first rows and tl from row loA / loT
  int pre;
  int loA, loT;
};

// A band of m whose synthesis table is rebuilt and used in one step: chunks
// [q0, q1) and synthesis tiles [tile0, tile1).
struct SynBand {
  int q0, q1, tile0, tile1;
};

void launch_lam_tc_tables(const double *x, const LegDfArgs &D, int lmax, int RP, int RPp, const int *offTc,
                          float *lamA, float *lamT, bool split, size_t loA, size_t loT, cudaStream_t s);
struct TcMaps;
// groups: slots per ring-stage CTA for each class (0 or nullptr: the default rule)
void launch_batch_iteration(const BatchArgs &a, const TcArgs &t, const TcMaps &maps, const RingClass *cls, int ncls,
                            const int *groups, int *bstate, cudaStream_t s, const SynBand *bands, int nbands);
void launch_batch_ring_class(const BatchArgs &a, const RingClass &c, int G, cudaStream_t s);
bool batch_ring_group_ok(int logM, int G);
void launch_batch_state(const BatchArgs &a, int *bstate, cudaStream_t s);
void launch_batch_zero_slot(const BatchArgs &a, const TcArgs &t, long long nchunks, int b, cudaStream_t s);
void launch_batch_convert_slot(const BatchArgs &a, int b, cudaStream_t s);
void launch_batch_export_slot(const BatchArgs &a, int b, cudaStream_t s);
void launch_hi_table(const float4 *src, float2 *dst, long long n, cudaStream_t s);

void launch_ring(const RingArgs &a, const RingClass *cls, int ncls, cudaStream_t s, int mode);
void launch_ring_df(const RingArgs &a, const RingDfArgs &t, const RingClass *cls, int ncls, cudaStream_t s,
                    int mode);
// ring order and classes of a ring table (host; rings as built for the plan)
void ring_classes(const RingDev *rings, int R, std::vector<int> &order, std::vector<RingClass> &cls);
void launch_to_df(const double2 *src, float4 *dst, long long n, cudaStream_t s);
void launch_legendre(const LegArgs &a, cudaStream_t s, int mode);
void launch_legendre_df(const LegArgs &a, const LegDfArgs &d, cudaStream_t s, int mode);
void launch_posterior_maps(const double *d, const double *w, double *ya, double *wd, long long npix, cudaStream_t s);
void launch_posterior_norms(const double2 *a, const double2 *ta, const double2 *tb, const double *cl, int lmax,
                            double inv_omega, double *part, cudaStream_t s);
// rows of the precomputed double-float lambda table (sum over m of ceil((lmax - m + 1) / 2)),
// each RP float4
size_t lam_table_rows(int lmax);
// dynamic shared memory of the table form of the Legendre kernel
size_t leg_tab_smem(int lmax, int RP);
void launch_lam_table(const double *x, const double2 *rec, const int *ls64, const double2 *sv64, const int *ls_df,
                      const long long *poff, int lmax, int RP, float4 *tab, cudaStream_t s);
void launch_df_tables(const double *x, const double2 *rec, int lmax, int RP, double *g, float2 *A, int *ls,
                      float4 *sv, cudaStream_t s);
void launch_start_values(const double *x, const double2 *rec, int lmax, int RP, int *ls,
                         double2 *sv, cudaStream_t s);
void launch_bluestein_setup(const RingDev *rings, const int *order, const RingClass *cls, int ncls, void *scratch,
                            const double2 *tw, int logMmax, const double2 *chirp, double2 *B, cudaStream_t s);
void launch_control(Ctl *ctl, const double *ring_part, int R, const double *m_part, int lmax,
                    const double *cl, wf_iter_record *hist, int hist_cap, cudaStream_t s);

// Raise a kernel's dynamic shared-memory cap to the device's opt-in maximum
// (once per function). The cap is an attribute of the function, read when a
// launch or a captured graph node runs, so launches of one kernel with
// different shared-memory sizes (ring classes, plans of different shapes)
// must never lower it under one another.
void raise_smem_cap(const void *func);

// error plumbing
void set_error(const std::string &msg);
wf_status cuda_status(cudaError_t e, const char *where);

}  // namespace wfk
