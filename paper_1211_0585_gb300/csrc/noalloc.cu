// Allocation-free map2alm.
//
// Some callers cannot call cudaMalloc on their call path: code that runs
// under a device-memory budget owned by another allocator (a framework's
// caching allocator or a fixed pool), and latency-critical loops that cannot
// afford cudaMalloc's implicit device synchronisation. wf_map2alm_noalloc
// serves them: it needs no plan and allocates nothing. Its working memory --
// the ring geometry, FFT and Legendre tables it builds for the requested
// (nside, lmax), and the Fourier coefficients between the ring and Legendre
// stages -- lives in one file-scope device array of kNoAllocScratchBytes
// (16 MiB), which every GPU that loads this library holds until the process
// exits (every lmax <= 4 nside fits it for nside <= 128, lmax <= 243 for
// nside 256). The kernels are the native FP64 ring and Legendre kernels that
// wf_map2alm runs for a WF_PREC_FP64_NATIVE plan, so the two agree to
// rounding (the tables here are built on the device, one ring class over all
// rings); a default (double-float) plan's wf_map2alm agrees to about 1e-12.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "wf_internal.h"

namespace wfk {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

int ilog2_up(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

__device__ __forceinline__ int ilog2_dev(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte offsets of every table inside the scratch array (host arithmetic only).
struct Layout {
  size_t rings, hs, chirp, B, tw, x, rec, ls, sv, FT, total;
  long long hs_n, ch_n, B_n;
  int maxM;
};

Layout layout_for(int nside, int lmax) {
  Layout L{};
  long long hs = 0, ch = 0, B = 0;
  int maxM = 1;
  for (int i = 1; i <= nside; ++i) {
    const long long n = 4LL * i;
    hs += n;
    const bool pow2 = (n & (n - 1)) == 0;
    const int lg = pow2 ? ilog2_up(n) : ilog2_up(2 * n - 1);
    if (!pow2) { ch += n; B += 1LL << lg; }
    if ((1 << lg) > maxM) maxM = 1 << lg;
  }
  const int R = 4 * nside - 1, RP = 2 * nside;
  const size_t nalm = (size_t)(lmax + 1) * (lmax + 2) / 2, nmk = (size_t)(lmax + 1) * RP;
  size_t o = 0;
  L.rings = o; o = align256(o + sizeof(RingDev) * R);
  L.hs = o;    o = align256(o + sizeof(double2) * hs);
  L.chirp = o; o = align256(o + sizeof(double2) * (ch > 4LL * nside ? ch : 4LL * nside));
  L.B = o;     o = align256(o + sizeof(double2) * (B > 0 ? B : 1));
  L.tw = o;    o = align256(o + sizeof(double2) * maxM);
  L.x = o;     o = align256(o + sizeof(double) * RP);
  L.rec = o;   o = align256(o + sizeof(double2) * nalm);
  L.ls = o;    o = align256(o + sizeof(int) * nmk);
  L.sv = o;    o = align256(o + sizeof(double2) * nmk);
  L.FT = o;    o = align256(o + sizeof(double4_32a) * nmk);
  L.total = o;
  L.hs_n = hs; L.ch_n = ch; L.B_n = B; L.maxM = maxM;
  return L;
}

// Ring geometry, per-length FFT tables and ring-pair latitudes for one nside,
// in the layout the ring and Legendre kernels read.
__global__ void noalloc_geometry_kernel(int nside, int maxM, RingDev *rings, double2 *hs, double2 *chirp,
                                        double2 *tw, double *x) {
  const int R = 4 * nside - 1;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // per-length offsets by prefix sums over lengths 4i, i = 1 .. nside
  for (long long r = gid; r < R; r += stride) {
    const int i = (int)r + 1;
    const int ip = i < 4 * nside - i ? i : 4 * nside - i;
    const int cls = ip < nside ? ip : nside;
    long long hs_off = 0, ch_off = 0, B_off = 0;
    for (int c = 1; c < cls; ++c) {
      const long long n = 4LL * c;
      hs_off += n;
      if ((n & (n - 1)) != 0) { ch_off += n; B_off += 1LL << ilog2_dev(2 * n - 1); }
    }
    const long long n = 4LL * cls;
    const bool pow2 = (n & (n - 1)) == 0;
    RingDev g{};
    g.n = (int)n;
    const long long npix = 12LL * nside * nside;
    if (i < nside) g.off = 2LL * i * (i - 1);
    else if (i <= 3 * nside) g.off = 2LL * nside * (nside - 1) + (long long)(i - nside) * 4 * nside;
    else g.off = npix - 2LL * ip * (ip + 1);
    g.shifted = ip < nside ? 1 : (((i - nside) % 2) == 0 ? 1 : 0);
    g.pair = (int)(r < R - 1 - r ? r : R - 1 - r);
    g.side = r > R - 1 - r ? 1 : 0;
    g.logM = pow2 ? ilog2_dev(n) : ilog2_dev(2 * n - 1);
    g.blue = pow2 ? 0 : 1;
    g.hs_off = hs_off;
    g.ch_off = pow2 ? 0 : ch_off;
    g.B_off = pow2 ? 0 : B_off;
    rings[r] = g;
  }
  // half-shift and chirp tables, length by length
  long long hs_off = 0, ch_off = 0;
  for (int c = 1; c <= nside; ++c) {
    const long long n = 4LL * c;
    const bool pow2 = (n & (n - 1)) == 0;
    for (long long q = gid; q < n; q += stride) {
      double s, co;
      sincospi((double)q / (double)n, &s, &co);
      hs[hs_off + q] = make_double2(co, s);
      if (!pow2) {
        const long long jj = (q * q) % (2 * n);
        sincospi((double)jj / (double)n, &s, &co);
        chirp[ch_off + q] = make_double2(co, -s);
      }
    }
    hs_off += n;
    if (!pow2) ch_off += n;
  }
  for (long long k = gid; k < maxM; k += stride) {
    double s, co;
    sincospi(2.0 * (double)k / (double)maxM, &s, &co);
    tw[k] = make_double2(co, -s);
  }
  for (long long k = gid; k < 2 * nside; k += stride) {
    const int i = (int)k + 1;
    x[k] = (i < nside) ? 1.0 - (double)i * i / (3.0 * (double)nside * nside)
                       : 4.0 / 3.0 - 2.0 * i / (3.0 * nside);
  }
}

// Recurrence coefficients a_l, b_l of the orthonormal Legendre functions.
__global__ void noalloc_rec_kernel(int lmax, double2 *rec) {
  const int m = blockIdx.x;
  const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
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

}  // namespace
}  // namespace wfk

using namespace wfk;

extern "C" wf_status wf_map2alm_noalloc(int nside, int lmax, const double *map_dev, double *alm_dev, void *stream) {
  if (!map_dev || !alm_dev) { set_error("wf_map2alm_noalloc: NULL argument"); return WF_EINVAL; }
  if (nside < 1 || nside > 1024 || (nside & (nside - 1)) != 0 || lmax < 0 || lmax > 4 * nside) {
    set_error("wf_map2alm_noalloc: nside must be a power of two in [1, 1024] and 0 <= lmax <= 4 nside");
    return WF_EINVAL;
  }
  const Layout L = layout_for(nside, lmax);
  if (L.total > kNoAllocScratchBytes) {
    set_error("wf_map2alm_noalloc: this (nside, lmax) needs " + std::to_string(L.total) +
              " bytes of scratch; the static scratch holds " + std::to_string(kNoAllocScratchBytes) +
              " bytes (use wf_plan_create + wf_map2alm)");
    return WF_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) { set_error("wf_map2alm_noalloc: device index out of range"); return WF_EINVAL; }
  unsigned char *base = nullptr;
  {
    // once per device, with that device current: the device address of the static array
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress");
      g_noalloc_ptr[dev] = p;
    }
    base = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RingDev *rings = reinterpret_cast<RingDev *>(base + L.rings);
  double2 *hs = reinterpret_cast<double2 *>(base + L.hs);
  double2 *chirp = reinterpret_cast<double2 *>(base + L.chirp);
  double2 *B = reinterpret_cast<double2 *>(base + L.B);
  double2 *tw = reinterpret_cast<double2 *>(base + L.tw);
  double *x = reinterpret_cast<double *>(base + L.x);
  double2 *rec = reinterpret_cast<double2 *>(base + L.rec);
  int *ls = reinterpret_cast<int *>(base + L.ls);
  double2 *sv = reinterpret_cast<double2 *>(base + L.sv);
  double4_32a *FT = reinterpret_cast<double4_32a *>(base + L.FT);
  const int R = 4 * nside - 1, RP = 2 * nside;
  // the ring stage never writes the equator pair's south slot: it must read as zero
  e = cudaMemsetAsync(FT, 0, sizeof(double4_32a) * (size_t)(lmax + 1) * RP, s);
  if (e != cudaSuccess) return cuda_status(e, "cudaMemsetAsync");
  noalloc_geometry_kernel<<<64, 256, 0, s>>>(nside, L.maxM, rings, hs, chirp, tw, x);
  noalloc_rec_kernel<<<lmax + 1, 128, 0, s>>>(lmax, rec);
  const RingClass all{ilog2_up(L.maxM), 0, R, 0};   // one launch over every ring, in ring order
  if (L.B_n > 0) launch_bluestein_setup(rings, nullptr, &all, 1, nullptr, tw, ilog2_up(L.maxM), chirp, B, s);
  launch_start_values(x, rec, lmax, RP, ls, sv, s);
  RingArgs ra{};
  ra.rings = rings; ra.tw = tw; ra.logMmax = ilog2_up(L.maxM); ra.hs = hs; ra.chirp = chirp; ra.B = B;
  ra.FT = FT; ra.RP = RP; ra.map_in = map_dev; ra.lsht = lmax;
  ra.omega = 4.0 * M_PI / (double)(12LL * nside * nside);
  launch_ring(ra, &all, 1, s, RING_ANALYSIS);
  LegArgs la{};
  la.x = x; la.rec = rec; la.ls = ls; la.sv = sv; la.FT = FT; la.alm = reinterpret_cast<double2 *>(alm_dev);
  la.lsht = lmax; la.lmax = lmax; la.RP = RP;
  launch_legendre(la, s, LEG_ANALYSIS);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "wf_map2alm_noalloc launch");
  return WF_OK;
}
