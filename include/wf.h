/*
 * wf.h -- C ABI of the GB300 messenger-field Wiener filter library.
 *
 * Method: Elsner & Wandelt, "Fast Wiener filtering of CMB maps",
 * arXiv:1211.0585. The library solves Eq. 2,
 *     (S^-1 + N^-1) s_WF = N^-1 d,
 * for a HEALPix map d (RING order), noise covariance N diagonal in pixel space
 * (masked pixels carry N^-1 = 0) and signal covariance S = diag(C_l) in
 * spherical-harmonic space, by the messenger-field iteration of Sect. 2
 * (Eqs. 3 and 4, messenger covariance T = tau * 1, tau = min diag(N),
 * Nbar = N - T) with the cooling of lambda and the band limit
 * lmax_SHT = l_iter + margin of Sect. 3.
 *
 * One iteration, all on the GPU:
 *   s_p  = (Y s)_p                         synthesis (Legendre stage, ring FFT)
 *   u_p  = a_p(lambda) (d_p - s_p)          Eq. 3 solved per pixel: t = s + u,
 *                                           a_p = lambda tau w_p / (1 + (lambda-1) tau w_p),
 *                                           w_p = 1/sigma_p^2 (0 where masked)
 *   t_lm = s_lm + (Y^dagger u)_lm           basis change of the increment t - s
 *                                           (ring FFT, Legendre stage); Y^dagger =
 *                                           (4 pi / Npix) Y^T, uniform weights
 *   s_lm = f_l(lambda) t_lm                 Eq. 4 solved per mode,
 *                                           f_l = C_l / (C_l + lambda tau 4 pi / Npix)
 * plus the chi^2 = s^+ S^-1 s + (d - s)^+ N^-1 (d - s) monitor of Sect. 3.
 *
 * Conventions shared by every entry point
 *   - a_lm: m >= 0 only (real field), m-major, index(l, m) = m (2 lmax + 1 - m) / 2 + l,
 *     nalm = (lmax + 1)(lmax + 2) / 2 complex numbers stored as interleaved
 *     doubles (re, im): 2 * nalm doubles. Orthonormal spherical harmonics with
 *     the Condon-Shortley phase.
 *   - maps: Npix = 12 nside^2 doubles in HEALPix RING order.
 *   - Pointers named *_dev are CUDA device pointers; an `on_device` flag says
 *     whether a pointer that may be either is device (1) or host (0) memory.
 *     The caller owns every buffer it passes; the library copies what it keeps.
 *   - Every function returns a wf_status and never aborts; after an error,
 *     wf_last_error() gives a message (thread-local).
 *   - A plan is not thread-safe: one thread at a time per plan. The server is
 *     thread-safe.
 *   - Units are free but consistent: d and sigma in one unit, C_l in that unit
 *     squared times steradian.
 */
#ifndef WF_H
#define WF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WF_OK = 0,
  WF_EINVAL = 1,          /* bad argument (sizes, NaN or <= 0 variance on an observed pixel, ...) */
  WF_ENOMEM = 2,          /* device or host allocation failed, or over the server's HBM budget */
  WF_ECUDA = 3,           /* a CUDA call failed (message in wf_last_error) */
  WF_ENOTCONVERGED = 4,   /* max_iter reached before the stop rule held (result still written) */
  WF_ENUMERIC = 5,        /* chi^2 became NaN or infinite */
  WF_ETIMEOUT = 6,        /* a bounded wait gave up */
  WF_EBUSY = 7,           /* result not ready (wf_poll) */
  WF_ECANCELLED = 8,      /* request cancelled */
  WF_ENOTFOUND = 9        /* unknown ticket */
} wf_status;

/* WF_PREC_FP64        FP64-accurate: the Legendre stage, the ring FFTs and the Eq. 3 update in
 *                     double-float arithmetic (pairs of floats with error-free transformations,
 *                     48-bit significands) because GB300 runs FP64 at 1/63 of its FP32 rate;
 *                     lambda_lm read from a precomputed table where it fits
 *                     (legendre_table_bytes); reductions, Eq. 4 and the controller in double.
 * WF_PREC_MIXED       the batched engine: FP32 ring FFTs, Legendre contractions on tensor cores
 *                     (tf32 with exact splits), double-float state and Eq. 4, double reductions;
 *                     optional FP64 refinement of each result (refine_iters).
 * WF_PREC_FP64_NATIVE every step in native double arithmetic (the plain reference kernels). */
typedef enum { WF_PREC_FP64 = 0, WF_PREC_MIXED = 1, WF_PREC_FP64_NATIVE = 2 } wf_precision;

typedef struct wf_plan_s *wf_plan_t;
typedef struct wf_server_s *wf_server_t;

/* Solver options (Sect. 3). Fill with wf_options_default, then override. */
typedef struct {
  int precision;         /* wf_precision */
  double tol;            /* stop when ||s_k - s_{k-1}|| / ||s_k|| <= tol at lambda = 1 (1e-6) */
  int max_iter;          /* iteration cap (10000) */
  int cooling;           /* 1: cool lambda as in Sect. 3; 0: lambda = 1 throughout (1) */
  int l_iter0;           /* first l_iter (20) */
  int lmax_margin;       /* lmax_SHT = min(lmax, l_iter + margin) while lambda > 1 (100) */
  int band_limit;        /* 1: use lmax_SHT while lambda > 1; 0: always lmax (1) */
  double plateau_eps;    /* plateau: |chi2_k - chi2_{k-1}| < eps * sqrt(2 n_obs) (1e-2) */
  double final_dchi2;    /* > 0: also stop at lambda = 1 when |d chi2| < final_dchi2 * sqrt(2 n_obs);
                            the paper uses 1e-4 (0 = off) */
  int min_level_iters;   /* iterations at a lambda level before a plateau can end it (3) */
  int max_level_iters;   /* a level ends after this many iterations regardless (1000) */
  int graph_iters;       /* iterations captured per CUDA graph launch (16) */
  int batch_slots;       /* slots of the batched mixed-precision engine, 1 .. 64 (64) */
  size_t legendre_table_bytes; /* WF_PREC_FP64 plans: hold lambda_lm(x_k) precomputed (double-float,
                            8 bytes per (l, m, ring pair), ring pairs padded to a multiple of 32) when
                            the table takes at most this many device
                            bytes; the Legendre stage then reads it instead of running the recurrence.
                            Decided at wf_plan_create; 0 = always the recurrence (8 GiB: Nside <= 512
                            at lmax = 2 Nside) */
  int posterior_grad;    /* 1: wf_solve on the FP64 paths also reports rel_posterior_grad (one synthesis
                            and two analyses after the solve) (1) */
  int refine_iters;      /* WF_PREC_MIXED: after the batched solve of each right-hand side, up to this many
                            FP64 iterations (double-float kernels) at lambda = 1 from its result, stopping
                            early once the relative increment is <= refine_tol; the result, chi^2 and
                            rel_posterior_grad are then the refined ones (0 = none) (0) */
  double refine_tol;     /* stop rule of the refinement (0 = run all refine_iters) (0) */
  int synthesis_table;   /* batched engine: 1 keeps the synthesis-ordered FP32 Legendre table resident;
                            0 rebuilds it band by band of m from the analysis table every iteration (half
                            the table memory, one transpose pass more); 2 keeps both tables resident and
                            split into their two tf32 parts (twice the table memory; the GEMMs then make
                            no split of their own, same results bit for bit); -1 chooses the largest of
                            2, 1, 0 with which the engine fits the free device memory (-1; the server's
                            engines choose between 1 and 0) */
  void *stream;          /* cudaStream_t to run on; NULL = the plan's own stream */
} wf_options;

/* Result summary of a solve. */
typedef struct {
  int iters;             /* iterations run */
  int converged;         /* 1 if the stop rule held */
  int levels;            /* lambda levels visited */
  int lmax_sht_final;
  double lambda_final;
  double chi2;           /* chi^2 of the input state of the last iteration (Sect. 3 definition) */
  double chi2_prior;     /* s^+ S^-1 s part */
  double chi2_noise;     /* (d - s)^+ N^-1 (d - s) part */
  double chi2_per_dof;   /* chi2 / n_obs */
  double rel_increment;  /* ||s_k - s_{k-1}|| / ||s_k|| of the last iteration */
  double ms_device;      /* time of the solve on the device: CUDA events around wf_solve's work; for a
                            mixed solve in the batched engine (wf_solve_batch, served requests), the
                            time its slot was occupied, from admission to harvest (host clock) */
  double rel_posterior_grad; /* ||Y^T W (d - Y a) - C^-1 a|| / ||Y^T W d|| of the result (modes with C_l > 0,
                            m > 0 counted twice; Y^T = map2alm / Omega): how far it is from the posterior
                            mean on the grid (Eq. 2), bounded below by the quadrature error of the HEALPix
                            analysis. FP64 paths with opt.posterior_grad = 1; -1 when not computed */
  double ms_latency;     /* served requests (wf_poll): from wf_submit to the result on the host; 0 for
                            direct solves */
} wf_stats;

/* Per-iteration record written by wf_iterate / wf_solve_history. */
typedef struct {
  double chi2_prior, chi2_noise, chi2_lambda;  /* of the iteration's input state */
  double incr2, norm2;                         /* ||s_k - s_{k-1}||^2, ||s_k||^2 (m > 0 weighted x2) */
  double lambda;
  int lmax_sht;
  int level;
} wf_iter_record;

/* Defaults listed beside each field above. */
wf_status wf_options_default(wf_options *opt);

/* Create a plan for one (nside, lmax, C_l, noise, mask) problem: builds the
 * ring geometry, FFT tables, Legendre recurrence tables, tau = min over
 * observed pixels of noise_var (Sect. 2), and allocates all device buffers.
 *   nside      : power of two, 1 .. 2048 (rings whose FFT buffers do not fit shared memory
 *                use a global scratch array)
 *   lmax       : 0 .. min(4 nside, 4096) (the range over which the rescaled recurrence is pinned)
 *   cl         : host [lmax+1], beam folded in, >= 0 and finite (C_l = 0: mode not solved for)
 *   noise_var  : host [Npix] sigma_p^2, finite and > 0 on observed pixels
 *   mask       : host [Npix] 1 = observed, 0 = masked (N^-1 = 0); NULL = all observed
 *   opt        : NULL = defaults; copied into the plan
 * Errors: WF_EINVAL on bad sizes/values or no observed pixel; WF_ENOMEM; WF_ECUDA. */
wf_status wf_plan_create(int nside, int lmax, const double *cl, const double *noise_var,
                         const uint8_t *mask, const wf_options *opt, wf_plan_t *out);

wf_status wf_plan_destroy(wf_plan_t plan);

/* Sizes and constants of a plan. Any out pointer may be NULL. */
wf_status wf_plan_info(wf_plan_t plan, int64_t *npix, int64_t *nalm, double *tau,
                       int64_t *n_obs, size_t *device_bytes);

/* Work of the Legendre stage at band limit lsht: the number of (l, m, ring
 * pair) terms with l, m <= lsht that the double-float kernels evaluate (terms
 * with |lambda_lm| below 2^-60 are skipped), and the full count
 * (lsht+1)(lsht+2)/2 * 2 nside for comparison. Either out pointer may be NULL. */
wf_status wf_plan_legendre_terms(wf_plan_t plan, int lsht, int64_t *evaluated, int64_t *full);

/* The precomputed lambda table of a WF_PREC_FP64 plan (Sect. 2 Legendre stage):
 * *held = its device bytes (0 when the plan runs the recurrence), *per_pass =
 * the bytes of it that one Legendre pass (analysis or synthesis) at band limit
 * lsht needs: for every m <= lsht and ring pair, the 16-byte rows of two l
 * from the row holding the first term at or above the 2^-60 cut through the
 * row holding lsht. Either out pointer may be NULL. */
wf_status wf_plan_legendre_table(wf_plan_t plan, int lsht, int64_t *held, int64_t *per_pass);

/* Kernel launches in one messenger iteration of the plan's single-solve path
 * (WF_PREC_FP64 or WF_PREC_FP64_NATIVE): the ring stage (one launch, or at
 * Nside 2048 two: the rings whose FFT buffers exceed shared memory run apart),
 * the Legendre stage and the controller. Used to count device launches; *n
 * must not be NULL. */
wf_status wf_plan_kernels_per_iteration(wf_plan_t plan, int *n);

/* Replace the plan's options (precision, tolerances, schedule knobs, stream). */
wf_status wf_plan_set_options(wf_plan_t plan, const wf_options *opt);

/* Synthesis map = Y alm with band limit lsht (<= lmax; modes with l > lsht are
 * ignored): the "transform back" of Sect. 2. Device pointers, alm in the plan's
 * lmax layout. Runs on the plan's stream; returns after enqueueing (no sync). */
wf_status wf_alm2map(wf_plan_t plan, int lsht, const double *alm_dev, double *map_dev);

/* Adjoint alm = Y^dagger map = (4 pi / Npix) Y^T map with band limit lsht
 * (entries with l > lsht are set to 0): the basis change of Sect. 2. */
wf_status wf_map2alm(wf_plan_t plan, int lsht, const double *map_dev, double *alm_dev);

/* Allocation-free map2alm: alm = Y^dagger map as wf_map2alm with lsht = lmax,
 * but with no plan and no device allocation on the call path. It runs the
 * native FP64 kernels: it agrees with wf_map2alm of a WF_PREC_FP64_NATIVE plan
 * to rounding (1e-14) and with that of a default (double-float) plan to about
 * 1e-12. The
 * paper has no counterpart; this entry point exists for callers that cannot
 * call cudaMalloc -- code running under a device-memory budget owned by another
 * allocator (a framework's caching allocator or a fixed pool) and
 * latency-critical loops that cannot take cudaMalloc's implicit device
 * synchronisation.
 *   nside, lmax : as wf_plan_create, nside <= 1024; the tables and Fourier
 *                 scratch for this size must fit the library's static 16 MiB
 *                 device array: every lmax <= 4 nside fits for nside <= 128,
 *                 lmax <= 243 for nside 256, nothing for nside >= 512. Larger
 *                 sizes return WF_EINVAL with the bytes they would need.
 *   map_dev     : device [Npix] input; alm_dev : device [2*nalm] output.
 *   stream      : cudaStream_t, NULL = the default stream. Enqueues and returns.
 * The scratch array is one per GPU, held from library load to process exit and
 * shared by every call on that GPU: calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * The first call on each device (with that device current) looks up the
 * array's device address; make that first call before any stream capture. */
wf_status wf_map2alm_noalloc(int nside, int lmax, const double *map_dev, double *alm_dev, void *stream);

/* Run `niter` messenger iterations (Eqs. 3-4) at fixed lambda (>= 1) and band
 * limit lsht, in place on the device state s_dev [2*nalm], with data d_dev
 * [Npix]. If `reset_state` is 1, s_dev is taken as a fresh start (its synthesis
 * is recomputed first); the plan otherwise reuses the synthesis left by the
 * previous call. `records` (host, may be NULL) receives niter entries.
 * Synchronises the plan's stream before returning. */
wf_status wf_iterate(wf_plan_t plan, const double *d_dev, double *s_dev, double lambda, int lsht,
                     int niter, int reset_state, wf_iter_record *records);

/* Timing aid: like wf_iterate (no records, state in s_dev), but with CUDA
 * events around each kernel of the iteration on the plan's stream. Writes the
 * average device time in ms per launch of: ms[0] the ring kernel (FFTs and the
 * Eq. 3 update), ms[1] the Legendre kernel (analysis, Eq. 4, synthesis),
 * ms[2] the controller. Synchronises before returning. */
wf_status wf_profile_iterations(wf_plan_t plan, const double *d_dev, double *s_dev, double lambda, int lsht,
                                int niter, float ms[3]);

/* Full solve with the cooling schedule and stop rule of Sect. 3.
 *   d        : [Npix] data, host or device (d_on_device)
 *   alm_out  : [2*nalm] result, host or device (alm_on_device)
 *   alm_init : NULL (start at s = 0, Sect. 2) or a warm start, same memory kind as alm_out
 *   stats    : may be NULL
 * Returns WF_OK, or WF_ENOTCONVERGED (result written) / WF_ENUMERIC. */
wf_status wf_solve(wf_plan_t plan, const double *d, int d_on_device, double *alm_out,
                   int alm_on_device, const double *alm_init, wf_stats *stats);

/* As wf_solve, also copying up to max_records per-iteration records to host. */
wf_status wf_solve_history(wf_plan_t plan, const double *d, int d_on_device, double *alm_out,
                           int alm_on_device, wf_stats *stats, wf_iter_record *records,
                           int max_records, int *n_records);

/* Solve nrhs right-hand sides that share the plan's C_l, noise and mask.
 *   d       : [nrhs][Npix], alm_out : [nrhs][2*nalm], stats : [nrhs] or NULL.
 * All right-hand sides advance together through one batched iteration per
 * step; each stops on its own rule. */
wf_status wf_solve_batch(wf_plan_t plan, int nrhs, const double *d, int d_on_device,
                         double *alm_out, int alm_on_device, wf_stats *stats);

/* Constrained realisations (Sect. 3, WMAP analysis: the Wiener filter map plus
 * a fluctuation map is a constrained realisation with the correct signal
 * variance; the power-spectra figure):
 *     s_CR,i = s_WF(d) + xi_i - s_WF(Y xi_i + n_i),   i = 0 .. nreal-1,
 * a draw from the posterior of s given d, with xi_i ~ N(0, S) (a_l0 = sqrt(C_l) z,
 * a_lm = sqrt(C_l / 2)(z + i z') for m > 0) and n_i ~ N(0, N) (sigma_p z on
 * observed pixels, 0 where masked) drawn on the device. The normals are a
 * function of (seed, realisation, entry) alone: Philox4x64-10 (Salmon et al.,
 * SC 2011) with key (seed, 0) and counter (block, kind, i, 0), kind 0 for the
 * signal (normals 2q, 2q + 1 for a_lm entry q) and 1 for the noise (normal p
 * for pixel p), four normals per block by Box-Muller on the uniforms
 * ((x >> 11) + 1/2) 2^-53 of words (0, 1) and (2, 3). The nreal + 1 Wiener
 * filters (d first) run as one wf_solve_batch in the plan's precision and
 * options.
 *   d       : [Npix] data, host or device (d_on_device)
 *   cr_out  : [nreal][2*nalm] realisations, host or device (out_on_device)
 *   wf_out  : [2*nalm] s_WF(d), same memory kind as cr_out, or NULL
 *   stats   : [nreal + 1] or NULL: the solve of d, then of each fluctuation map
 * Allocates its working buffers ((nreal + 1) maps and 3 nreal + 1 a_lm vectors)
 * for the call. Returns WF_OK, or WF_ENOTCONVERGED (results written) and the
 * errors of wf_solve_batch. */
wf_status wf_constrained_realisations(wf_plan_t plan, int nreal, uint64_t seed, const double *d, int d_on_device,
                                      double *cr_out, int out_on_device, double *wf_out, wf_stats *stats);

/* Several messenger fields (Sect. 4, Conclusion: more than one messenger field
 * to combine several observations, e.g. of different detectors, in one
 * analysis). ndet maps of one sky on one grid, d_k = Y B_k s + n_k, each with
 * a beam B_k = diag(b_k,l), noise N_k (diagonal in pixel space, masked
 * pixels N_k^-1 = 0) and its own messenger t_k with T_k = tau_k 1,
 * tau_k = min diag(N_k). One iteration solves Eq. 3 per map and pixel,
 *     t_k = Y B_k s + a_k (d_k - Y B_k s),
 * and Eq. 4 with every messenger, per mode,
 *     s_lm = sum_k g_k b_k,l t_k,lm / (1 / C_l + sum_k g_k b_k,l^2),  g_k = 1 / (lambda tau_k Omega),
 * the basis change applied to t_k - Y B_k s, so that the result at lambda = 1 is
 * the joint Wiener filter (S^-1 + sum_k B_k Y^T N_k^-1 Y B_k) s = sum_k B_k Y^T N_k^-1 d_k.
 * The chi^2 monitor sums every map's noise term; cooling (Sect. 3) sets lambda
 * at scale l to C_l sum_k b_k,l^2 / (tau_k Omega), clamped to >= 1; the band
 * limit stays at lmax (opt->band_limit is ignored).
 *   ndet      : 1 .. 16 maps
 *   cl        : host [lmax+1] sky spectrum (beams NOT folded in)
 *   beams     : host [ndet][lmax+1] b_k,l, or NULL for b = 1
 *   noise_var : host [ndet][Npix]; mask : host [ndet][Npix] or NULL (all observed)
 *   opt       : as wf_plan_create; precision WF_PREC_FP64 or WF_PREC_FP64_NATIVE
 *               (WF_EINVAL for WF_PREC_MIXED)
 * One plan per map is created inside (its noise, mask and buffers); the first
 * holds the Legendre tables every map's transforms read. */
typedef struct wf_multi_s *wf_multi_t;
wf_status wf_multi_create(int nside, int lmax, int ndet, const double *cl, const double *beams,
                          const double *noise_var, const uint8_t *mask, const wf_options *opt, wf_multi_t *out);

/* Joint solve of the ndet maps d ([ndet][Npix], host or device): alm_out [2*nalm]
 * (host or device), stats and up to max_records per-iteration records (both
 * may be NULL). Returns WF_OK, WF_ENOTCONVERGED (result written) or WF_ENUMERIC. */
wf_status wf_multi_solve(wf_multi_t multi, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                         wf_stats *stats, wf_iter_record *records, int max_records, int *n_records);

wf_status wf_multi_destroy(wf_multi_t multi);

/* Temperature and polarisation (Sect. 4, Conclusion: the filter on T and P maps
 * together; the power-spectra figure's TT, EE and TE). Pixels carry (T, Q, U)
 * with a 3 x 3 noise covariance N_p (T independent of the Q-U block) and
 * separate temperature and polarisation masks (N^-1 = 0 on masked components);
 * the signal covariance per (l, m) is [[C_TT, C_TE, 0], [C_TE, C_EE, 0],
 * [0, 0, C_BB]] on (a^T, a^E, a^B). The messenger covariance is T = tau 1 on all
 * three components, tau = the smallest eigenvalue of N_p over the observed
 * components; Eq. 3 becomes a 3 x 3 solve per pixel,
 *     t_p = s_p + A_p (d_p - s_p),  A_p = lambda tau (N_p + (lambda - 1) tau 1)^-1,
 * Eq. 4 the 2 x 2 (T, E) block and B per mode, s = S_l (S_l + lambda tau Omega)^-1 t,
 * with the basis change applied to t - s. (Q, U) <-> (E, B) by spin-2 harmonics,
 * Q +- iU = - sum_lm (a^E_lm +- i a^B_lm) _{+-2}Y_lm, _{+-2}Y from the spin-raising
 * operator on Y_lm (Condon-Shortley phase). Cooling takes lambda from
 * C_TT / (tau Omega) at l_iter (Sect. 3); the band limit stays at lmax.
 *   cls       : host [4][lmax+1] = C_TT, C_EE, C_BB, C_TE (beams folded in; C_TE^2 <= C_TT C_EE)
 *   noise     : host [Npix][4] = (TT, QQ, QU, UU) noise (co)variances per pixel
 *   mask_t, mask_p : host [Npix] (1 = observed) or NULL (all observed)
 *   opt       : WF_PREC_FP64 or WF_PREC_FP64_NATIVE for the T channel and the ring
 *               FFTs (WF_EINVAL for WF_PREC_MIXED); the spin-2 Legendre stage runs in
 *               FP64 from a table of (F+, F-) per (l, m, ring pair) (16 bytes each,
 *               64 GiB at most: Nside <= 1024 at lmax = 2 Nside)
 * a_lm of the three fields are stored one after the other: [3][2*nalm] (T, E, B);
 * maps likewise [3][Npix] (T, Q, U). */
typedef struct wf_pol_s *wf_pol_t;
wf_status wf_pol_create(int nside, int lmax, const double *cls, const double *noise, const uint8_t *mask_t,
                        const uint8_t *mask_p, const wf_options *opt, wf_pol_t *out);

/* Joint (T, Q, U) solve: d [3][Npix] host or device, alm_out [3][2*nalm] host or
 * device; stats, records as wf_multi_solve. */
wf_status wf_pol_solve(wf_pol_t pol, const double *d, int d_on_device, double *alm_out, int alm_on_device,
                       wf_stats *stats, wf_iter_record *records, int max_records, int *n_records);

/* The transform pair of the polarised fields (device pointers, full band, on the
 * plan's stream, no sync): maps = Y alm and alm = Y^dagger maps = (4 pi / Npix) Y^T maps. */
wf_status wf_pol_alm2map(wf_pol_t pol, const double *alm_dev, double *map_dev);
wf_status wf_pol_map2alm(wf_pol_t pol, const double *map_dev, double *alm_dev);

wf_status wf_pol_destroy(wf_pol_t pol);

/* Serving: continuous batching of solve requests of any (nside, lmax, C_l,
 * noise, mask) under a device-memory budget.
 *   hbm_budget_bytes : admission limit for plans + per-request buffers (0 = 90 % of free memory)
 *   max_batch        : most requests of one shape that advance in one step */
wf_status wf_server_create(size_t hbm_budget_bytes, int max_batch, wf_server_t *out);

/* Submit a request (host arrays, copied). tol <= 1e-7 selects the FP64 path,
 * larger tol the mixed path (a mixed request that finds its shape's engine
 * without live requests may run on the FP64 pool instead, which meets any
 * tolerance; so does one whose shape's engine exceeds the whole budget).
 * Never blocks on the GPU. WF_ENOMEM at once when no path for the request
 * fits the server's whole HBM budget (it could never be admitted). */
wf_status wf_submit(wf_server_t server, int nside, int lmax, const double *cl,
                    const double *noise_var, const uint8_t *mask, const double *d, double tol,
                    uint64_t *ticket);

/* Non-blocking: *done = 1 and alm_out (host, [2*nalm]) / stats filled when the
 * request finished; *done = 0 otherwise. Returns the request's own status once
 * done; WF_ENOTFOUND for an unknown or already collected ticket. */
wf_status wf_poll(wf_server_t server, uint64_t ticket, int *done, double *alm_out, wf_stats *stats);

/* Cancel a request. A request still queued is dropped at once; one in a slot of
 * a batched engine leaves it at the end of the current step; one being solved
 * on the FP64 path stops after the current block of iterations. wf_poll then
 * reports it done with WF_ECANCELLED and no a_lm. Returns WF_OK when the
 * cancellation is recorded, WF_EINVAL (nothing changed) when the request had
 * already finished -- its result stands --, WF_ENOTFOUND for an unknown or
 * collected ticket. The paper has no counterpart (serving control). */
wf_status wf_cancel(wf_server_t server, uint64_t ticket);

/* Make a shape resident before its requests arrive, as a serving system loads
 * its models: precision WF_PREC_MIXED builds the shape's batched engine
 * (tables, FP32 Lambda tables, autotuned ring tiles) on the server's worker,
 * WF_PREC_FP64 adds one idle FP64 plan of the shape (geometry, Legendre and
 * lambda tables) to the pool its FP64 requests run on. Blocks until done.
 * WF_ENOMEM when the shape does not fit the budget now; WF_EINVAL for a bad
 * shape or precision. */
wf_status wf_server_warm(wf_server_t server, int nside, int lmax, int precision);

/* Block until every admitted request has finished or timeout_ms passed
 * (WF_ETIMEOUT). */
wf_status wf_server_drain(wf_server_t server, int timeout_ms);

/* Request latency percentiles (ms) and completed-solve count since creation. */
wf_status wf_server_stats(wf_server_t server, double *p50_ms, double *p99_ms, int64_t *completed);

wf_status wf_server_destroy(wf_server_t server);

/* Message of the last error on this thread ("" if none). */
const char *wf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WF_H */
