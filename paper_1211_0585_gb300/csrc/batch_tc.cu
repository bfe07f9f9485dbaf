// Tensor-core Legendre stage of the batched engine (tcgen05, kind::tf32).
//
// Per m, the two contractions of the messenger iteration are GEMMs over the
// shape's Legendre table Lambda_m[l][k] = lambda_lm(x_k) (Sect. 2: the basis
// change between pixel and harmonic space, its Legendre half):
//   analysis   t_p[i][c] = sum_k  Lambda[l_i][k] X_p[k][c]   (X_0 = N + S, X_1 = N - S)
//   synthesis  D_p[k][c] = sum_i  Lambda[l_i][k] s[l_i][c]   (E = D_0, O = D_1; N = E + O, S = E - O)
// with l_i = m + p + 2 i (parity p of l - m), c = 2 b + (re, im) over the slots.
// The Legendre tables hold lambda rounded to 22 significant bits, so that a
// table value is exactly the sum of two tf32 numbers, th + tl; the data operand
// (X or s, FP32) is split exactly into three, ah + am + al (11 + 11 + 2 bits).
// The tensor cores form th ah + th am + tl ah + tl am + th al (every partial
// product at or above 2^-24 of the whole; the one dropped, tl al, is 2^-33) with
// fp32 accumulation in tensor memory: FP32-level products from tf32 inputs.
//
// Tables (built once per shape from the double-float recurrence):
//   lamA  rows (m, p, i) in that order, ring pairs k contiguous (padded to RPp, a
//         multiple of 32): the analysis A operand, one TMA box = 128 rows x 32 k;
//   lamT  rows (m, p, chunk of 32 i, k), 32 values of i contiguous: the synthesis
//         A operand, one TMA box = 128 ring pairs x 32 i.
// With split tables (T.pre) each table holds th in its first half of rows and
// tl in its second, so the GEMMs load both parts; otherwise the 22-bit values
// are loaded and split in shared memory by four splitting warps.
// Per-iteration operands (written by the engine's own kernels), each value
// already split into its three tf32 parts (part-major within a chunk):
//   XT    rows (m, p, chunk of 32 k, part, c), 32 values of k contiguous (from FT);
//   SPT   rows (m, p, chunk of 32 i, part, c), 32 values of i contiguous (written
//         by the analysis epilogue for the next synthesis).
// A data chunk is split once where it is produced, not once per GEMM tile that
// reads it (an analysis chunk is read by every tile of i of its (m, p), a
// synthesis chunk by every tile of ring pairs of its m).
//
// Each GEMM CTA is warp-specialised: warp 0 issues the table's TMA loads into a
// ring of three stages (two with split tables), warp 2 the data operand's into
// a ring of three stages and brings the chunks kDAhead ahead into L2 (they come
// mostly from L2: every tile of an (m, p) or m reads them), warp 1 owns the
// tensor memory and issues the MMAs, warps 3-6 split the table tiles (when the
// table is not split already) and, in the synthesis GEMM, run the epilogue; in
// the analysis GEMM warps 8-15 fold the chunk sums and all sixteen warps run
// the Eq. 4 epilogue.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "batch_engine.h"
#include "df.cuh"
#include "tc.cuh"
#include "wf_internal.h"

namespace wfk {

namespace {

constexpr int kTileRows = 128;                       // M of every MMA
constexpr int kTileBytes = kTileRows * 128;          // 128 rows x 32 fp32 (a data tile: at most 128 columns)
constexpr int kSmemTiles = 14;                       // 224 KB of operand tiles per CTA
constexpr int kDAhead = 5;                           // data chunks brought into L2 this far ahead of their load
constexpr int kSplitWarps = 4;                       // warps 3-6
constexpr int kSynThreads = 224;                     // synthesis: table TMA, MMA, data TMA, 4 split / epilogue warps
constexpr uint32_t kWaitLimit = 1u << 22;            // polls of one bounded mbarrier wait

__device__ __forceinline__ size_t aidx(int lmax, int l, int m) { return (size_t)m * (2 * lmax + 1 - m) / 2 + l; }

// number of l in [m, L] with l - m = p (mod 2)
__host__ __device__ __forceinline__ int n_par(int m, int p, int L) { return L >= m + p ? (L - m - p) / 2 + 1 : 0; }

// Shared memory rings of one GEMM CTA, every tile 1024-byte aligned:
//   table  TS stages that TMA fills: (th, tl) with split tables, else th alone
//          (the 22-bit values, split in place by the splitting warps);
//   tl     (tables not split) LS slots the splitting warps write tl into;
//   data   DS stages of the operand's (h, m, l) parts.
// Loads wait about three MMA chunks' time to land, so each ring holds three
// stages where shared memory allows.
template <bool PRE>
struct Ring {
  static constexpr int TS = PRE ? 2 : 3;
  static constexpr int LS = PRE ? 0 : 2;
  static constexpr int DS = 3;
  static_assert(TS * (PRE ? 2 : 1) + LS + 3 * DS <= kSmemTiles, "rings exceed the operand tiles");
  __device__ static uint8_t *th(uint8_t *base, int s) { return base + (size_t)s * (PRE ? 2 : 1) * kTileBytes; }
  __device__ static uint8_t *tl(uint8_t *base, int s, int kc) {
    return PRE ? base + ((size_t)2 * s + 1) * kTileBytes : base + ((size_t)TS + kc % (LS ? LS : 1)) * kTileBytes;
  }
  __device__ static uint8_t *dat(uint8_t *base, int s, int part) {
    return base + ((size_t)TS * (PRE ? 2 : 1) + LS + (size_t)s * 3 + part) * kTileBytes;
  }
};
constexpr int kRingMax = 3;   // barrier array sizes

// v rounded to 11 significant bits (a tf32 number; ties away from zero) by
// integer arithmetic on its bits; v - hi is then exact. Rounding to nearest
// keeps the remainders unbiased, so the correction sums partly cancel.
__device__ __forceinline__ float tf32_rn(float v) {
  return __int_as_float((__float_as_int(v) + 0x1000) & (int)0xffffe000);
}

// table tile (22-bit values): th = v rounded to 11 bits in place, tl = v - th
// (exact, and a tf32 number). Each thread loads kSplitU float4 before it
// splits and stores any of them, so that their shared-memory loads overlap.
constexpr int kSplitU = 4;
__device__ __forceinline__ void split_table(uint8_t *hi, uint8_t *lo, int t, int nt) {
  float4 *h4 = reinterpret_cast<float4 *>(hi);
  float4 *l4 = reinterpret_cast<float4 *>(lo);
  constexpr int n = kTileBytes / 16;
  for (int e0 = t; e0 < n; e0 += kSplitU * nt) {
    float4 v[kSplitU];
#pragma unroll
    for (int u = 0; u < kSplitU; ++u)
      if (e0 + u * nt < n) v[u] = h4[e0 + u * nt];
#pragma unroll
    for (int u = 0; u < kSplitU; ++u) {
      if (e0 + u * nt >= n) break;
      float4 h, l;
      h.x = tf32_rn(v[u].x); l.x = v[u].x - h.x;
      h.y = tf32_rn(v[u].y); l.y = v[u].y - h.y;
      h.z = tf32_rn(v[u].z); l.z = v[u].z - h.z;
      h.w = tf32_rn(v[u].w); l.w = v[u].w - h.w;
      h4[e0 + u * nt] = h;
      l4[e0 + u * nt] = l;
    }
  }
}

// v = h + m + l exactly: 11 + 11 + at most 3 significant bits, every part a tf32 number
__device__ __forceinline__ void split3(float v, float &h, float &m, float &l) {
  h = tf32_rn(v);
  const float r = v - h;   // exact
  m = tf32_rn(r);
  l = r - m;               // exact: the last bits
}

// h + l += v with the rounding error of the leading sum kept (two-sum)
__device__ __forceinline__ void two_sum_acc(float &h, float &l, float v) {
  const float s = h + v, bv = s - h;
  l += (h - (s - bv)) + (v - bv);
  h = s;
}

// (h, l) += (h2, l2), renormalised; the result does not depend on the order of
// the two operands, so a butterfly leaves the same sum on every lane
__device__ __forceinline__ void df_pair_add(float &h, float &l, float h2, float l2) {
  const float s = h + h2, bv = s - h;
  const float e = (h - (s - bv)) + (h2 - bv) + (l + l2);
  h = s + e;
  l = e - (h - s);
}

// 4 k-steps of 8 over one 32-wide chunk: table parts th, tl; data parts h, m,
// l. The leading product th h accumulates alone in `dmain`; the correction
// products (2^-11 and less of it) accumulate in `dcorr`, so the rounding of
// the tensor-core accumulation stays relative to each sum's own size. REV runs
// the k-steps from the end of the chunk to its start.
template <bool REV = false>
__device__ __forceinline__ void mma_chunk(uint32_t dmain, uint32_t dcorr, uint8_t *th, uint8_t *tl, uint8_t *dh,
                                          uint8_t *dm, uint8_t *dl, uint32_t idesc, bool acc_main, bool acc_corr) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int ks = REV ? 3 - kk : kk;
    const uint64_t off = (uint64_t)((ks * 32) >> 4);   // 32 bytes along K inside the swizzle atom
    const uint64_t a_h = tc::sw128_desc(th) + off, a_l = tc::sw128_desc(tl) + off;
    const uint64_t b_h = tc::sw128_desc(dh) + off, b_m = tc::sw128_desc(dm) + off, b_l = tc::sw128_desc(dl) + off;
    tc::mma_tf32(dmain, a_h, b_h, idesc, acc_main || kk > 0);
    tc::mma_tf32(dcorr, a_h, b_l, idesc, acc_corr || kk > 0);
    tc::mma_tf32(dcorr, a_l, b_h, idesc, true);
    tc::mma_tf32(dcorr, a_h, b_m, idesc, true);
    tc::mma_tf32(dcorr, a_l, b_m, idesc, true);
  }
}

}  // namespace

// ---------------------------------------------------------------- tables
// One thread per (m, k): the double-float recurrence from the start values
// writes lambda_lm(x_k) (rounded to 22 bits, 0 below l_start) into both table
// layouts (only the analysis layout when lamT is nullptr: the synthesis rows are
// then rebuilt per band, lamt_band_kernel); rows of the transposed layout are
// written 32 values at a time from registers. With `split`, each layout holds
// th = tf32_rn(v) in its first half of rows and tl = v - th in its second (the
// split the GEMMs otherwise make in shared memory, value for value).
__global__ void lam_tc_tables_kernel(const double *xk, const LegDfArgs D, int lmax, int RP, int RPp,
                                     const int *offTc, float *lamA, float *lamT, int split, size_t loA,
                                     size_t loT) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)(lmax + 1) * RPp) return;
  const int m = (int)(id / RPp), k = (int)(id % RPp);
  const size_t base = aidx(lmax, m, m);
  const int n0 = n_par(m, 0, lmax);
  float buf[2][32];
  if (k >= RP) {   // padding ring pairs: zeros
    for (int h = 0; h <= split; ++h) {
      float *tA = lamA + (h ? loA : 0), *tT = lamT ? lamT + (h ? loT : 0) : nullptr;
      for (int p = 0; p < 2; ++p) {
        const int np = n_par(m, p, lmax);
        for (int i = 0; i < np; ++i) tA[(base + (p ? n0 + i : i)) * (size_t)RPp + k] = 0.f;
        for (int ic = 0; tT && ic < (np + 31) / 32; ++ic) {
          float4 *dst = reinterpret_cast<float4 *>(tT + ((size_t)(offTc[2 * m + p] + ic) * RPp + k) * 32);
          for (int j = 0; j < 8; ++j) dst[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
    return;
  }
  const size_t mk = (size_t)m * RP + k;
  const int ls = D.ls[mk];
  const float4 s4 = D.sv[mk];
  const dfl x = df_from(xk[k]);
  dfl p1 = {0.f, 0.f}, p2 = {0.f, 0.f};
  for (int l = m; l <= lmax; ++l) {
    float v = 0.f;
    if (l >= ls) {
      dfl mu;
      if (l == ls) mu = dfl{s4.x, s4.y};
      else if (l == ls + 1) mu = dfl{s4.z, s4.w};
      else {
        const float2 a2 = D.A[base + (l - m)];
        mu = df_step(dfl{a2.x, a2.y}, x, p1, p2);
      }
      p2 = p1;
      p1 = mu;
      // lambda rounded to 22 significant bits: the sum of two tf32 numbers
      const double lam = D.g[base + (l - m)] * df_to(mu);
      const float h = tc::to_tf32((float)lam);
      v = h + tc::to_tf32((float)(lam - (double)h));
    }
    const int p = (l - m) & 1, i = (l - m) >> 1;
    const size_t ra = (base + (p ? n0 + i : i)) * (size_t)RPp + k;
    if (split) {
      const float th = tf32_rn(v);
      lamA[ra] = th;
      lamA[loA + ra] = v - th;
    } else {
      lamA[ra] = v;
    }
    buf[p][i & 31] = v;
    const int np = n_par(m, p, lmax);
    if (lamT && ((i & 31) == 31 || i == np - 1)) {   // a chunk of 32 values of i is complete: write its row
      for (int j = (i & 31) + 1; j < 32; ++j) buf[p][j] = 0.f;
      const size_t rt = ((size_t)(offTc[2 * m + p] + (i >> 5)) * RPp + k) * 32;
      float4 *dst = reinterpret_cast<float4 *>(lamT + rt);
      if (split) {
        float4 *dlo = reinterpret_cast<float4 *>(lamT + loT + rt);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 v4 = make_float4(buf[p][4 * j], buf[p][4 * j + 1], buf[p][4 * j + 2], buf[p][4 * j + 3]);
          const float4 h4 = make_float4(tf32_rn(v4.x), tf32_rn(v4.y), tf32_rn(v4.z), tf32_rn(v4.w));
          dst[j] = h4;
          dlo[j] = make_float4(v4.x - h4.x, v4.y - h4.y, v4.z - h4.z, v4.w - h4.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          dst[j] = make_float4(buf[p][4 * j], buf[p][4 * j + 1], buf[p][4 * j + 2], buf[p][4 * j + 3]);
      }
    }
  }
}

// Streamed synthesis table: the rows of the chunks [q0, q0 + gridDim.x) in the
// synthesis order (32 values of i contiguous per ring pair) from the analysis
// table (ring pairs contiguous per i), into the scratch from chunk q0. One CTA
// per (chunk, 32 ring pairs): a 32 x 32 transpose through shared memory; the
// values are lamA's, so the GEMM sees the same operand as with the resident
// table. Chunks of m above the live band limit are skipped (the GEMM skips them).
__global__ void __launch_bounds__(256) lamt_band_kernel(const TcArgs T, int q0, const int *bstate) {
  __shared__ float tile[32][33];
  const int q = q0 + blockIdx.x, kb = blockIdx.y;
  const int4 ci = T.chunk_info[q];
  if (ci.z > bstate[0]) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int j = ty; j < 32; j += 8)
    tile[j][tx] = j < ci.y ? T.lamA[((size_t)ci.x + j) * T.RPp + 32 * kb + tx] : 0.f;
  __syncthreads();
  for (int r = ty; r < 32; r += 8)
    T.lamTs[((size_t)(q - T.qbase) * T.RPp + 32 * kb + r) * 32 + tx] = tile[tx][r];
}

// ---------------------------------------------------------------- FT -> XT
// One CTA per (m, chunk of 32 ring pairs): the Fourier coefficients of every
// slot, (N re, N im, S re, S im), become the analysis B operand of both
// parities, X_0 = N + S and X_1 = N - S, with ring pairs contiguous, each
// value written as its three tf32 parts.
__global__ void __launch_bounds__(256) xt_kernel(const BatchArgs A, const TcArgs T) {
  __shared__ float4 sF[32][kBatchMax + 1];
  const int m = blockIdx.y, kc = blockIdx.x;
  if (m > A.bstate[0]) return;
  const int B = A.B, RP = A.RP;
  for (int e = threadIdx.x; e < 32 * B; e += blockDim.x) {
    const int kk = e / B, b = e % B, k = 32 * kc + kk;
    sF[kk][b] = k < RP ? A.FT[((size_t)m * RP + k) * B + b] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t part = (size_t)T.Nc * 32;
  for (int row = warp; row < 2 * T.Nc; row += blockDim.x / 32) {
    const int p = row / T.Nc, c = row % T.Nc, b = c >> 1;
    float v = 0.f;
    if (b < B) {
      const float4 f = sF[lane][b];
      const float n = (c & 1) ? f.y : f.x, s = (c & 1) ? f.w : f.z;
      v = p ? n - s : n + s;
    }
    float h, mid, l;
    split3(v, h, mid, l);
    float *dst = T.XT + ((((size_t)m * 2 + p) * T.nkc + kc) * 3 * T.Nc + c) * 32 + lane;
    dst[0] = h;
    dst[part] = mid;
    dst[2 * part] = l;
  }
}

// ---------------------------------------------------------------- analysis GEMM + Eq. 4
// One CTA per (m, parity p, 128 values of i): t_p = Lambda X_p over every ring
// pair, then Eq. 4 on the double-float state, the prior chi^2 / increment /
// norm partials, and the next synthesis operand SPT.
//
// The leading products of every 32-wide chunk of ring pairs accumulate in one
// of two tensor-memory blocks (ping-pong), and eight folding warps add each
// finished chunk into a double-float accumulator: hi in tensor memory, lo in
// the folding threads' registers, as the FP32 path folded its chunk sums. The
// correction products accumulate over all chunks in a third block. Warps: 0
// table TMA, 1 MMA (and tensor memory), 2 data TMA, 3-6 table split (when the
// table is not split already), 7-14 folding and the epilogue (warp w: TMEM
// lanes 32 (w % 4) .., columns 64 ((w - 7) / 4) ..). Tiles wholly above the
// live band limit hold zero state (band limits only grow within a solve and
// new slots start from zero): they only report zero partials.
constexpr int kAnaThreads = 512;
constexpr int kFoldWarp0 = 8;
constexpr int kFoldThreads = 256;
constexpr int kFoldChunks = 1;   // chunks of 32 ring pairs per folded segment
constexpr uint32_t kColSeg0 = 0, kColSeg1 = 128, kColCorr = 256, kColHi = 384;

template <bool PRE>
__global__ void __launch_bounds__(kAnaThreads, 1)
    bana_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapX,
                   const BatchArgs A, const TcArgs T) {
  extern __shared__ __align__(1024) uint8_t tsm_raw[];
  uint8_t *tsm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~(uintptr_t)1023);
  using R = Ring<PRE>;
  __shared__ uint64_t tfull[kRingMax], tready[kRingMax], tempty[kRingMax], dfull[kRingMax], dempty[kRingMax];
  __shared__ uint64_t lfree[2], segf[2], segfree[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ unsigned long long live_slots;   // bit b: slot b iterates
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 tile = T.atiles[blockIdx.x];
  const int m = tile.x, p = tile.y, i0 = tile.z, rowA = tile.w;
  const int lmax = A.lmax, B = A.B, Nc = T.Nc;
  const int Lact = A.bstate[0];
  const bool live = m <= Lact && m + p + 2 * i0 <= Lact;
  if (!live) {
    for (int qb = threadIdx.x; qb < 3 * B; qb += blockDim.x)
      A.m_part[((size_t)(qb % B) * A.ntiles + blockIdx.x) * 3 + qb / B] = 0.0;
    return;
  }
  const int nkc = T.nkc;
  if (threadIdx.x == 0) {
    for (int s = 0; s < R::TS; ++s) {
      tc::mbar_init(&tfull[s], 1);
      tc::mbar_init(&tready[s], kSplitWarps);   // one arrival per splitting warp
      tc::mbar_init(&tempty[s], 1);
    }
    for (int s = 0; s < R::DS; ++s) {
      tc::mbar_init(&dfull[s], 1);
      tc::mbar_init(&dempty[s], 1);
    }
    for (int s = 0; s < 2; ++s) tc::mbar_init(&lfree[s], 1);
    for (int j = 0; j < 2; ++j) {
      tc::mbar_init(&segf[j], 1);
      tc::mbar_init(&segfree[j], kFoldThreads / 32);   // one arrival per folding warp
    }
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  if (warp < 2) {   // live slots: one slot per thread of warps 0-1, gathered by ballots
    const int b = threadIdx.x;
    const unsigned bits = __ballot_sync(0xffffffffu, b < B && A.active[b] && !A.ctl[b].done);
    if (lane == 0) reinterpret_cast<unsigned *>(&live_slots)[warp] = bits;
  }
  if (warp == 1) tc::tmem_alloc(&tmem_slot, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc::tf32_idesc(kTileRows, Nc);
  const uint32_t bbytes = (uint32_t)Nc * 128;
  int issued = 0;   // TMA stages issued by this thread's ring (for the drain on abort)

  // Each role branch is taken by a whole warp (lane 0 does the work) and ends in
  // __syncwarp, so that every warp reaches the block barriers below converged.
  if (warp == 0) {   // table ring
    if (lane == 0) {
      tc::prefetch_tensormap(&mapA);
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % R::TS;
        if (kc >= R::TS && !tc::mbar_wait(&tempty[s], ((kc / R::TS) - 1) & 1, kWaitLimit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag) break;
        tc::mbar_arrive_expect_tx(&tfull[s], PRE ? 2 * kTileBytes : kTileBytes);
        tc::tma_load_2d(R::th(tsm, s), &mapA, 32 * kc, rowA + i0, &tfull[s]);
        if (PRE) tc::tma_load_2d(R::tl(tsm, s, kc), &mapA, 32 * kc, T.loA + rowA + i0, &tfull[s]);
        issued = kc + 1;
      }
    }
    __syncwarp();
  } else if (warp == 2) {   // data ring: the three parts of X_p's chunk, brought into L2 kDAhead chunks early
    if (lane == 0) {
      tc::prefetch_tensormap(&mapX);
      const int y0 = (int)(((size_t)m * 2 + p) * T.nkc * 3 * Nc);
      for (int kc = R::DS; kc < kDAhead && kc < nkc; ++kc)
        for (int part = 0; part < 3; ++part) tc::tma_prefetch_2d(&mapX, 0, y0 + (kc * 3 + part) * Nc);
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % R::DS;
        if (kc >= R::DS && !tc::mbar_wait(&dempty[s], ((kc / R::DS) - 1) & 1, kWaitLimit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag) break;
        tc::mbar_arrive_expect_tx(&dfull[s], 3 * bbytes);
        const int y = y0 + kc * 3 * Nc;
#pragma unroll
        for (int part = 0; part < 3; ++part)
          tc::tma_load_2d(R::dat(tsm, s, part), &mapX, 0, y + part * Nc, &dfull[s]);
        if (kc + kDAhead < nkc)
          for (int part = 0; part < 3; ++part) tc::tma_prefetch_2d(&mapX, 0, y + (kDAhead * 3 + part) * Nc);
        issued = kc + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % R::TS, sd = kc % R::DS, j = kc / kFoldChunks;
        const uint32_t seg = tmem + ((j & 1) ? kColSeg1 : kColSeg0);
        // a segment block is reused once the folding warps have read it
        if (kc % kFoldChunks == 0 && j >= 2 &&
            (*(volatile int *)&abort_flag || !tc::mbar_wait(&segfree[j & 1], ((j - 2) >> 1) & 1, kWaitLimit))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag ||
            !tc::mbar_wait(PRE ? &tfull[s] : &tready[s], (kc / R::TS) & 1, kWaitLimit) ||
            !tc::mbar_wait(&dfull[sd], (kc / R::DS) & 1, kWaitLimit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        tc::tc_fence_after();
        mma_chunk(seg, tmem + kColCorr, R::th(tsm, s), R::tl(tsm, s, kc), R::dat(tsm, sd, 0), R::dat(tsm, sd, 1),
                  R::dat(tsm, sd, 2), idesc, kc % kFoldChunks != 0, kc > 0);
        tc::mma_commit(&tempty[s]);
        tc::mma_commit(&dempty[sd]);
        if (!PRE) tc::mma_commit(&lfree[kc % 2]);
        if (kc % kFoldChunks == kFoldChunks - 1 || kc == nkc - 1) tc::mma_commit(&segf[j & 1]);
      }
    }
    __syncwarp();
  } else if (!PRE && warp >= 3 && warp < 3 + kSplitWarps) {
    const int t = threadIdx.x - 96;
    for (int kc = 0; kc < nkc; ++kc) {
      const int s = kc % R::TS;
      if (tc::warp_flag(&abort_flag) || !tc::mbar_wait_warp(&tfull[s], (kc / R::TS) & 1, kWaitLimit) ||
          (kc >= 2 && !tc::mbar_wait_warp(&lfree[kc % 2], ((kc / 2) - 1) & 1, kWaitLimit))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      split_table(R::th(tsm, s), R::tl(tsm, s, kc), t, 32 * kSplitWarps);
      tc::fence_proxy_async_smem();
      tc::mbar_arrive_warp(&tready[s]);
    }
  }
  // folding warps: chunk sums into (hi in TMEM, lo in registers)
  const int fq = warp & 3, fh = (warp - kFoldWarp0) >> 2;      // lane quadrant, column half
  const uint32_t flanes = (uint32_t)(32 * fq) << 16;
  float lo[64];
#pragma unroll
  for (int e = 0; e < 64; ++e) lo[e] = 0.f;
  if (warp >= kFoldWarp0) {
    {   // the epilogue's state rows into L2 while the GEMM runs
      const int i = i0 + 32 * fq + lane;
      if (i < n_par(m, p, lmax)) {
        const unsigned long long mine = live_slots >> (32 * fh);
        for (int jb = 0; jb < 32; ++jb)
          if ((mine >> jb) & 1ull) tc::prefetch_l2(A.sdf + (size_t)(32 * fh + jb) * A.nalm + rowA + i);
      }
    }
    const int nseg = (nkc + kFoldChunks - 1) / kFoldChunks;
    for (int kc = 0; kc < nseg; ++kc) {   // segment index
      if (tc::warp_flag(&abort_flag) || !tc::mbar_wait_warp(&segf[kc & 1], (kc >> 1) & 1, kWaitLimit)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      tc::tc_fence_after();
      const uint32_t seg = tmem + flanes + ((kc & 1) ? kColSeg1 : kColSeg0);
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) {
        const int cb = 4 * fh + bb;
        if (16 * cb >= Nc) break;
        uint32_t vr[16], hr[16];
        tc::tmem_ld16_issue(seg + 16 * cb, vr);
        if (kc > 0) tc::tmem_ld16_issue(tmem + flanes + kColHi + 16 * cb, hr);
        tc::tmem_ld_wait(vr);
        if (kc > 0) tc::tmem_ld_wait(hr);
        float v[16], h[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(vr[e]);
        if (kc == 0) {
#pragma unroll
          for (int e = 0; e < 16; ++e) h[e] = v[e];
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) h[e] = __uint_as_float(hr[e]);
#pragma unroll
          for (int e = 0; e < 16; ++e) {   // two_sum(h, v): the rounding error goes to lo
            const float sum = h[e] + v[e];
            const float bv = sum - h[e];
            lo[16 * bb + e] += (h[e] - (sum - bv)) + (v[e] - bv);
            h[e] = sum;
          }
        }
        tc::tmem_st16(tmem + flanes + kColHi + 16 * cb, h);
      }
      tc::tmem_wait_st();
      tc::tc_fence_before();
      tc::mbar_arrive_warp(&segfree[kc & 1]);
    }
    // the chunk blocks are free now: park lo there for the epilogue (frees the registers)
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int cb = 4 * fh + bb;
      if (16 * cb >= Nc) break;
      float v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = lo[16 * bb + e];
      tc::tmem_st16(tmem + flanes + kColSeg0 + 16 * cb, v);
    }
    tc::tmem_wait_st();
    tc::tc_fence_before();
  }

  // ---- epilogue (all 16 warps: warp w takes TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..)
  __syncthreads();   // every chunk is folded, the stage buffers are free, abort_flag is final
  tc::tc_fence_after();
  const bool ok_acc = abort_flag == 0;   // uniform over the CTA
  float *red = reinterpret_cast<float *>(tsm);    // [3][Bp][129] partials (row stride 129: no bank conflicts)
  {
    const int eq = warp & 3, ec = warp >> 2;
    const uint32_t elanes = (uint32_t)(32 * eq) << 16;
    const int r = 32 * eq + lane;
    const int i = i0 + r;
    const int np = n_par(m, p, lmax);
    const bool row_ok = i < np;
    const int l = m + p + 2 * i;
    const size_t idx = (size_t)rowA + (row_ok ? i : 0);   // state row (the analysis table's row order)
    const float wgt = (m == 0) ? 1.f : 2.f;
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int cb = 2 * ec + bb;
      if (16 * cb >= Nc) break;
      float th[16], tl[16];
      if (ok_acc) {   // t = hi + (lo + corrections)
        uint32_t hr[16], cr[16], lr[16];
        tc::tmem_ld16_issue(tmem + elanes + kColHi + 16 * cb, hr);
        tc::tmem_ld16_issue(tmem + elanes + kColCorr + 16 * cb, cr);
        tc::tmem_ld16_issue(tmem + elanes + kColSeg0 + 16 * cb, lr);
        tc::tmem_ld_wait(hr);
        tc::tmem_ld_wait(cr);
        tc::tmem_ld_wait(lr);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          th[e] = __uint_as_float(hr[e]);
          tl[e] = __uint_as_float(cr[e]) + __uint_as_float(lr[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) { th[e] = 0.f; tl[e] = 0.f; }
      }
      // every load of the eight slots first (independent), then the updates
      const unsigned live8 = row_ok ? (unsigned)(live_slots >> (8 * cb)) & 0xffu : 0u;
      float4 so[8], fv[4], iv[2];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        so[jj] = (live8 >> jj) & 1u ? A.sdf[(size_t)(8 * cb + jj) * A.nalm + idx] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (live8) {   // filter and 1 / C_l of the eight slots: [l][slot], 16-byte aligned runs
        const float4 *f4 = reinterpret_cast<const float4 *>(A.fdf + (size_t)l * B + 8 * cb);
        const float4 *c4 = reinterpret_cast<const float4 *>(A.icl + (size_t)l * B + 8 * cb);
#pragma unroll
        for (int e = 0; e < 4; ++e) fv[e] = f4[e];
        iv[0] = c4[0];
        iv[1] = c4[1];
      }
      // the next synthesis operand, split into its tf32 parts (part-major within the chunk)
      float *spt = T.SPT + (((size_t)T.offTc[2 * m + p] + (i >> 5)) * 3 * Nc + 16 * cb) * 32 + (i & 31);
      const size_t spart = (size_t)Nc * 32;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int b = 8 * cb + jj;
        float c2 = 0.f, inc = 0.f, nrm = 0.f;
        if ((live8 >> jj) & 1u) {
          const float4 fq4 = fv[jj >> 1];
          const dfl f = (jj & 1) ? dfl{fq4.z, fq4.w} : dfl{fq4.x, fq4.y};
          const float icl = (jj < 4) ? ((jj & 2) ? ((jj & 1) ? iv[0].w : iv[0].z) : ((jj & 1) ? iv[0].y : iv[0].x))
                                     : ((jj & 2) ? ((jj & 1) ? iv[1].w : iv[1].z) : ((jj & 1) ? iv[1].y : iv[1].x));
          const float4 o = so[jj];
          const dfl re = df_mul(f, df_add(dfl{o.x, o.y}, dfl{th[2 * jj], tl[2 * jj]}));
          const dfl im = df_mul(f, df_add(dfl{o.z, o.w}, dfl{th[2 * jj + 1], tl[2 * jj + 1]}));
          const float4 sn = make_float4(re.h, re.l, im.h, im.l);
          c2 = wgt * (o.x * o.x + o.z * o.z) * icl;
          const float dx = (sn.x - o.x) + (sn.y - o.y), dy = (sn.z - o.z) + (sn.w - o.w);
          inc = wgt * (dx * dx + dy * dy);
          nrm = wgt * (sn.x * sn.x + sn.z * sn.z);
          A.sdf[(size_t)b * A.nalm + idx] = sn;
          float h, mid, lw;
          split3(sn.x, h, mid, lw);
          spt[(2 * jj) * 32] = h;
          spt[spart + (2 * jj) * 32] = mid;
          spt[2 * spart + (2 * jj) * 32] = lw;
          split3(sn.z, h, mid, lw);
          spt[(2 * jj + 1) * 32] = h;
          spt[spart + (2 * jj + 1) * 32] = mid;
          spt[2 * spart + (2 * jj + 1) * 32] = lw;
        }
        red[(0 * B + b) * 129 + r] = c2;
        red[(1 * B + b) * 129 + r] = inc;
        red[(2 * B + b) * 129 + r] = nrm;
      }
    }
  }
  __syncthreads();
  // sums over the 128 rows, one (quantity, slot) per warp: each lane adds its
  // four rows, then a butterfly of double-float pairs (the same order on every
  // lane and in every run: the sums are reproducible)
  for (int qb = warp; qb < 3 * B; qb += kAnaThreads / 32) {
    const float *rw = red + qb * 129;
    float h = rw[lane], l = 0.f;
#pragma unroll
    for (int e = 1; e < 4; ++e) two_sum_acc(h, l, rw[lane + 32 * e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
      df_pair_add(h, l, h2, l2);
    }
    if (lane == 0) A.m_part[((size_t)(qb % B) * A.ntiles + blockIdx.x) * 3 + qb / B] = (double)h + (double)l;
  }
  // drain: every TMA this CTA issued has landed before its shared memory is released
  if (warp == 0 || warp == 2) {
    if (lane == 0 && *(volatile int *)&abort_flag) {
      const int ns = warp == 0 ? R::TS : R::DS;
      uint64_t *bar = warp == 0 ? tfull : dfull;
      for (int kc = max(0, issued - ns); kc < issued; ++kc) tc::mbar_wait(&bar[kc % ns], (kc / ns) & 1, kWaitLimit);
    }
    __syncwarp();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc::tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(T.err, 1);
}

// ---------------------------------------------------------------- synthesis GEMM
// One CTA per (m, 128 ring pairs): E and O accumulate in two tensor-memory
// blocks over the chunks of 32 values of i of each parity up to the live band
// limit; the epilogue writes FS = (E + O, E - O) for every slot. Warps: 0 table
// TMA, 1 MMA, 2 data TMA, 3-6 table split (when the table is not split already)
// and the epilogue.
template <bool PRE>
__global__ void __launch_bounds__(kSynThreads, 1)
    bsyn_tc_kernel(const __grid_constant__ CUtensorMap mapT, const __grid_constant__ CUtensorMap mapS,
                   const BatchArgs A, const TcArgs T) {
  extern __shared__ __align__(1024) uint8_t tsm_raw[];
  uint8_t *tsm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~(uintptr_t)1023);
  using R = Ring<PRE>;
  __shared__ uint64_t tfull[kRingMax], tready[kRingMax], tempty[kRingMax], dfull[kRingMax], dempty[kRingMax];
  __shared__ uint64_t lfree[2], accf;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 tile = T.stiles[T.tile0 + blockIdx.x];
  const int m = tile.x, k0 = tile.y;
  const int B = A.B, RP = A.RP, Nc = T.Nc;
  const int Lact = A.bstate[0];
  if (m > Lact) return;
  const int nc0 = (n_par(m, 0, Lact) + 31) / 32, nc1 = (n_par(m, 1, Lact) + 31) / 32;
  const int nq = nc0 + nc1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < R::TS; ++s) {
      tc::mbar_init(&tfull[s], 1);
      tc::mbar_init(&tready[s], kSplitWarps);   // one arrival per splitting warp
      tc::mbar_init(&tempty[s], 1);
    }
    for (int s = 0; s < R::DS; ++s) {
      tc::mbar_init(&dfull[s], 1);
      tc::mbar_init(&dempty[s], 1);
    }
    for (int s = 0; s < 2; ++s) tc::mbar_init(&lfree[s], 1);
    tc::mbar_init(&accf, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  if (warp == 1) tc::tmem_alloc(&tmem_slot, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc::tf32_idesc(kTileRows, Nc);
  const uint32_t bbytes = (uint32_t)Nc * 128;
  int issued = 0;
  // within a parity the chunks run from high l to low l: the large low-l
  // terms enter the fp32 accumulator last
  auto chunk_of = [&](int qi) {
    const int p = qi < nc0 ? 0 : 1, ic = p ? nc0 + nc1 - 1 - qi : nc0 - 1 - qi;
    return (long long)T.offTc[2 * m + p] + ic;
  };

  // Each role branch is taken by a whole warp (lane 0 does the work) and ends in
  // __syncwarp, so that every warp reaches the block barriers below converged.
  if (warp == 0) {   // table ring
    if (lane == 0) {
      if (nq > 0) tc::prefetch_tensormap(&mapT);
      for (int qi = 0; qi < nq; ++qi) {
        const int s = qi % R::TS;
        if (qi >= R::TS && !tc::mbar_wait(&tempty[s], ((qi / R::TS) - 1) & 1, kWaitLimit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag) break;
        const int y = (int)((chunk_of(qi) - T.qbase) * T.RPp + k0);
        tc::mbar_arrive_expect_tx(&tfull[s], PRE ? 2 * kTileBytes : kTileBytes);
        tc::tma_load_2d(R::th(tsm, s), &mapT, 0, y, &tfull[s]);
        if (PRE) tc::tma_load_2d(R::tl(tsm, s, qi), &mapT, 0, T.loT + y, &tfull[s]);
        issued = qi + 1;
      }
    }
    __syncwarp();
  } else if (warp == 2) {   // data ring: the three parts of the state chunk, brought into L2 kDAhead chunks early
    if (lane == 0) {
      if (nq > 0) tc::prefetch_tensormap(&mapS);
      for (int qi = R::DS; qi < kDAhead && qi < nq; ++qi)
        for (int part = 0; part < 3; ++part) tc::tma_prefetch_2d(&mapS, 0, (int)((chunk_of(qi) * 3 + part) * Nc));
      for (int qi = 0; qi < nq; ++qi) {
        const int s = qi % R::DS;
        if (qi >= R::DS && !tc::mbar_wait(&dempty[s], ((qi / R::DS) - 1) & 1, kWaitLimit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag) break;
        const int y = (int)(chunk_of(qi) * 3 * Nc);
        tc::mbar_arrive_expect_tx(&dfull[s], 3 * bbytes);
#pragma unroll
        for (int part = 0; part < 3; ++part)
          tc::tma_load_2d(R::dat(tsm, s, part), &mapS, 0, y + part * Nc, &dfull[s]);
        if (qi + kDAhead < nq)
          for (int part = 0; part < 3; ++part)
            tc::tma_prefetch_2d(&mapS, 0, (int)((chunk_of(qi + kDAhead) * 3 + part) * Nc));
        issued = qi + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      for (int qi = 0; qi < nq; ++qi) {
        const int s = qi % R::TS, sd = qi % R::DS;
        if (*(volatile int *)&abort_flag ||
            !tc::mbar_wait(PRE ? &tfull[s] : &tready[s], (qi / R::TS) & 1, kWaitLimit) ||
            !tc::mbar_wait(&dfull[sd], (qi / R::DS) & 1, kWaitLimit)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        tc::tc_fence_after();
        const int p = qi < nc0 ? 0 : 1, first = p ? qi == nc0 : qi == 0;
        // leading products of parity p in columns 128 p, corrections in 256 + 128 p
        mma_chunk<true>(tmem + (uint32_t)(128 * p), tmem + (uint32_t)(256 + 128 * p), R::th(tsm, s),
                        R::tl(tsm, s, qi), R::dat(tsm, sd, 0), R::dat(tsm, sd, 1), R::dat(tsm, sd, 2), idesc, !first,
                        !first);
        tc::mma_commit(&tempty[s]);
        tc::mma_commit(&dempty[sd]);
        if (!PRE) tc::mma_commit(&lfree[qi % 2]);
      }
      if (nq > 0) tc::mma_commit(&accf);
    }
    __syncwarp();
  } else if (!PRE && warp >= 3) {
    const int t = threadIdx.x - 96;
    for (int qi = 0; qi < nq; ++qi) {
      const int s = qi % R::TS;
      if (tc::warp_flag(&abort_flag) || !tc::mbar_wait_warp(&tfull[s], (qi / R::TS) & 1, kWaitLimit) ||
          (qi >= 2 && !tc::mbar_wait_warp(&lfree[qi % 2], ((qi / 2) - 1) & 1, kWaitLimit))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      split_table(R::th(tsm, s), R::tl(tsm, s, qi), t, 32 * kSplitWarps);
      tc::fence_proxy_async_smem();
      tc::mbar_arrive_warp(&tready[s]);
    }
  }
  // ---- epilogue (warps 3-6): row k0 + r of E (columns 0 .. Nc) and O (Nc .. 2 Nc)
  if (warp >= 3 && nq > 0 && !tc::warp_flag(&abort_flag) && !tc::mbar_wait_warp(&accf, 0, kWaitLimit))
    atomicExch(&abort_flag, 1);
  __syncthreads();   // abort_flag is final from here on
  tc::tc_fence_after();
  const bool have = nq > 0 && abort_flag == 0;   // uniform over the CTA
  if (warp >= 3) {
    const int qd = warp & 3;
    const int k = k0 + 32 * qd + lane;
    const uint32_t lanes = (uint32_t)(32 * qd) << 16;
    for (int cb = 0; cb < Nc / 16; ++cb) {
      float e[16], o[16];
      uint32_t er[16], cer[16], orr[16], cor[16];
      if (have && nc0 > 0) {
        tc::tmem_ld16_issue(tmem + lanes + 16 * cb, er);
        tc::tmem_ld16_issue(tmem + lanes + 256 + 16 * cb, cer);
      }
      if (have && nc1 > 0) {
        tc::tmem_ld16_issue(tmem + lanes + 128 + 16 * cb, orr);
        tc::tmem_ld16_issue(tmem + lanes + 384 + 16 * cb, cor);
      }
      if (have && nc0 > 0) {
        tc::tmem_ld_wait(er);
        tc::tmem_ld_wait(cer);
#pragma unroll
        for (int j = 0; j < 16; ++j) e[j] = __uint_as_float(er[j]) + __uint_as_float(cer[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) e[j] = 0.f;
      }
      if (have && nc1 > 0) {
        tc::tmem_ld_wait(orr);
        tc::tmem_ld_wait(cor);
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = __uint_as_float(orr[j]) + __uint_as_float(cor[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = 0.f;
      }
      if (k < RP) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int b = 8 * cb + jj;
          if (b < B)
            A.FS[((size_t)m * RP + k) * B + b] = make_float4(e[2 * jj] + o[2 * jj], e[2 * jj + 1] + o[2 * jj + 1],
                                                             e[2 * jj] - o[2 * jj], e[2 * jj + 1] - o[2 * jj + 1]);
        }
      }
    }
  }
  if (warp == 0 || warp == 2) {
    if (lane == 0 && *(volatile int *)&abort_flag) {
      const int ns = warp == 0 ? R::TS : R::DS;
      uint64_t *bar = warp == 0 ? tfull : dfull;
      for (int qi = max(0, issued - ns); qi < issued; ++qi) tc::mbar_wait(&bar[qi % ns], (qi / ns) & 1, kWaitLimit);
    }
    __syncwarp();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc::tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(T.err, 1);
}

// ---------------------------------------------------------------- host side
static size_t gemm_smem() { return (size_t)kSmemTiles * kTileBytes + 1024; }

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D fp32 tensor of `rows` rows of `inner` values (inner * 4 bytes apart),
// boxes of box_rows x 32 values, 128-byte swizzle
bool make_tc_map(CUtensorMap *map, const float *base, unsigned long long inner, unsigned long long rows,
                 unsigned box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * sizeof(float)};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_lam_tc_tables(const double *x, const LegDfArgs &D, int lmax, int RP, int RPp, const int *offTc,
                          float *lamA, float *lamT, bool split, size_t loA, size_t loT, cudaStream_t s) {
  // lamT nullptr: analysis table only
  const long long n = (long long)(lmax + 1) * RPp;
  lam_tc_tables_kernel<<<(int)((n + 127) / 128), 128, 0, s>>>(x, D, lmax, RP, RPp, offTc, lamA, lamT, split ? 1 : 0,
                                                               loA, loT);
}

template <bool PRE>
static void launch_gemms(const BatchArgs &a, const TcArgs &t, const TcMaps &maps, cudaStream_t s, int which,
                         const SynBand *bands, int nbands) {
  raise_smem_cap(reinterpret_cast<const void *>(bana_tc_kernel<PRE>));
  raise_smem_cap(reinterpret_cast<const void *>(bsyn_tc_kernel<PRE>));
  if (which == 0) {
    xt_kernel<<<dim3(t.nkc, a.lmax + 1), 256, 0, s>>>(a, t);
    bana_tc_kernel<PRE><<<t.natiles, kAnaThreads, gemm_smem(), s>>>(maps.A, maps.X, a, t);
  } else if (!t.lamTs) {
    bsyn_tc_kernel<PRE><<<t.nstiles, kSynThreads, gemm_smem(), s>>>(maps.T, maps.S, a, t);
  } else {
    // band by band: rebuild the band's synthesis-ordered rows, then its GEMM tiles
    for (int i = 0; i < nbands; ++i) {
      const SynBand &b = bands[i];
      TcArgs tb = t;
      tb.qbase = b.q0;
      tb.tile0 = b.tile0;
      lamt_band_kernel<<<dim3(b.q1 - b.q0, t.nkc), 256, 0, s>>>(tb, b.q0, a.bstate);
      bsyn_tc_kernel<PRE><<<b.tile1 - b.tile0, kSynThreads, gemm_smem(), s>>>(maps.T, maps.S, a, tb);
    }
  }
}

void launch_batch_gemms_tc(const BatchArgs &a, const TcArgs &t, const TcMaps &maps, cudaStream_t s, int which,
                           const SynBand *bands, int nbands) {
  if (t.pre) launch_gemms<true>(a, t, maps, s, which, bands, nbands);
  else launch_gemms<false>(a, t, maps, s, which, bands, nbands);
}

}  // namespace wfk
