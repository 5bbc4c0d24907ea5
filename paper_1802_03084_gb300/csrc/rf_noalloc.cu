// rf_noalloc.cu -- rf_image_stats_noalloc: image one caller-supplied uv
// half-plane and measure its peak, noise and S/N without allocating any
// memory.
//
// Who needs it: code that must not call cudaMalloc -- a caller recording
// work into a CUDA graph (cudaMalloc cannot be captured), a real-time loop
// that cannot take the latency or the failure modes of the allocator, or a
// host framework that owns the device memory pool and forbids allocations by
// libraries it hosts.  Such a caller passes device pointers for the input
// and the output; the column-FFT intermediate and the row-block partials this
// imaging needs live in one file-scope __device__ array, sized for images up
// to RF_NOALLOC_MAX_NPIX pixels a side, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "realfast_gb300.h"
#include "rf_engine.h"
#include "rf_image.cuh"

namespace rf {
namespace {

constexpr int kMaxN = RF_NOALLOC_MAX_NPIX;
constexpr int kMaxDevices = 64;

// Scratch: column-FFT output T[u][y] (u < N/2), the row-pair partials of
// the statistics kernel, the per-column Parseval sums and the (0, 0) term.  Every byte a call reads is written by
// the same call first, so nothing has to start at zero.
constexpr size_t kTBytes = (size_t)kMaxN * (kMaxN / 2) * sizeof(float2);
constexpr size_t kPartialBytes = (size_t)ImgCfg<kMaxN>::PARTIALS * sizeof(StatPartial);
constexpr size_t kColsqBytes = (kMaxN / 2 + 64) * sizeof(float);  // Parseval column sums + mean term
static __device__ __align__(256) unsigned char g_noalloc_scratch[kTBytes + kPartialBytes + kColsqBytes];

// Twiddle tables of the length-N transforms (fft_twiddle_table) for N = 16,
// 32, ..., kMaxN, back to back (constants written once per device at
// set-up, not scratch).
constexpr int twiddle_offset(int n) { return n <= 16 ? 0 : twiddle_offset(n >> 1) + fft_twiddle_len(n >> 1); }
constexpr int kTwiddleElems = twiddle_offset(kMaxN) + fft_twiddle_len(kMaxN);
static __device__ __align__(256) float2 g_noalloc_twiddle[kTwiddleElems];

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;
  float2* twiddle = nullptr;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

rf_status setup_error(rf_status s, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof(buf), "rf_image_stats_noalloc set-up: %s: %s", what, cudaGetErrorString(e));
  set_last_error(buf);
  return s;
}

// Once per device, with that device current: resolve the device addresses
// of the two arrays (host code cannot use the symbols themselves) and write
// the twiddle tables.
rf_status ensure_setup(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return setup_error(RF_ERR_CUDA, "cudaGetSymbolAddress(scratch)", e);
    d.scratch = static_cast<unsigned char*>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_twiddle);
    if (e != cudaSuccess) return setup_error(RF_ERR_CUDA, "cudaGetSymbolAddress(twiddle)", e);
    d.twiddle = static_cast<float2*>(p);
    std::vector<float2> tw(kTwiddleElems);
    for (int n = 16; n <= kMaxN; n <<= 1) fft_twiddle_table(n, tw.data() + twiddle_offset(n));
    e = cudaMemcpy(d.twiddle, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return setup_error(RF_ERR_CUDA, "twiddle upload", e);
    d.ready = true;
  }
  *out = &d;
  return RF_OK;
}

// Column pass of the imaging kernels, reading a dense half-plane grid
// H[v][u] (row length N/2 + 1) instead of gathering visibilities: each of the
// XA transforms of a CTA takes one column u < N/2, applies the
// (-1)^(u + v) phase-centre shift and inverse-FFTs it along v.
template <int N>
__global__ void __launch_bounds__(ImgCfg<N>::T * ImgCfg<N>::XA)
    k_colfft_dense(const float2* __restrict__ grid, float2* __restrict__ T, const float2* __restrict__ tw,
                   float* __restrict__ colsq, float* __restrict__ mean0) {
  using K = ImgCfg<N>;
  constexpr int W = N / 2 + 1;
  constexpr int NC = N / 2;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int col0 = blockIdx.x * K::XA;
  constexpr int THREADS = K::T * K::XA;
  for (int i = tid; i < N * K::XA; i += THREADS) {
    const int c = i % K::XA;
    const int v = i / K::XA;
    const int u = col0 + c;
    float2 h = make_float2(0.f, 0.f);
    if (u < NC) {
      h = __ldg(grid + (size_t)v * W + u);
      if ((u + v) & 1) h = make_float2(-h.x, -h.y);
    }
    sm[c * K::STRIDE + padx(v)] = h;
  }
  __syncthreads();
  const int xf = tid / K::T;
  const int t = tid - xf * K::T;
  const int u = col0 + xf;
  {
    // Parseval: weighted sum of |H|^2 down the column (twice for u > 0)
    float acc = 0.f;
    for (int v = t; v < N; v += K::T) {
      const float2 h = sm[xf * K::STRIDE + padx(v)];
      acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
    }
    constexpr int WL = K::T < 32 ? K::T : 32;
#pragma unroll
    for (int off = WL / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (t == 0 && u < NC) {
      colsq[u] = (u == 0 ? 1.f : 2.f) * acc;
      if (u == 0) *mean0 = sm[xf * K::STRIDE].x;
    }
  }
  float2 v[K::E];
  fft_inverse_to_regs<N>(v, sm + xf * K::STRIDE, tw, t, xf);
  if (u < NC) {
    float2* dst = T + (size_t)u * N;
    constexpr int LP = FftShape<N>::LAST_P;
#pragma unroll
    for (int m = 0; m < K::E / LP; ++m)
#pragma unroll
      for (int q = 0; q < LP; ++q) dst[fft_out_index<N>(t, m, q)] = v[m * LP + dft_perm<LP>(q)];
  }
}

// Reduce the row-block partials of one image into an rf_image_stat.
__global__ void k_noalloc_finalize(const StatPartial* __restrict__ partials, int nrb, const float* __restrict__ colsq,
                                   const float* __restrict__ mean0, int npix, double weight,
                                   rf_image_stat* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sq = 0.0;
  float mx = -FLT_MAX;
  int mi = INT_MAX;
  for (int r = 0; r < nrb; ++r) {
    const StatPartial p = partials[r];
    if (p.max > mx || (p.max == mx && p.idx < mi)) {
      mx = p.max;
      mi = p.idx;
    }
  }
  for (int c = 0; c < npix / 2; ++c) sq += (double)colsq[c];
  // mean = G(0,0) / 2W; mean of I^2 = sum_full |G|^2 / 4W^2 (Parseval)
  const double inv = 0.5 / weight;
  const double mean = (double)*mean0 * inv;
  double var = sq * inv * inv - mean * mean;
  var = var > 0.0 ? var : 0.0;
  const double sigma = sqrt(var);
  const double peak = (double)mx * inv;
  rf_image_stat o;
  o.dm_idx = 0;
  o.dt_idx = 0;
  o.t_idx = 0;
  o.y = mi / npix;
  o.x = mi - o.y * npix;
  o.peak = (float)peak;
  o.sigma = (float)sigma;
  o.snr = (float)(sigma > 0.0 ? peak / sigma : 0.0);
  o.mean = mean;
  o.weight = weight;
  *out = o;
}

template <int N>
cudaError_t run_noalloc(const float2* grid, double weight, const DeviceSetup& d, cudaStream_t st,
                        rf_image_stat* out) {
  using K = ImgCfg<N>;
  // The column-FFT scratch holds one image of at most kMaxN, the partials
  // area ImgCfg<kMaxN>::PARTIALS records; the Parseval sum of k_colfft_dense
  // and the finalisation reduce within one warp per column, which holds
  // while a transform fits one warp.
  static_assert(N <= kMaxN, "image larger than the static scratch");
  static_assert(K::PARTIALS <= ImgCfg<kMaxN>::PARTIALS, "partials area too small");
  static_assert(K::T <= 32, "the Parseval reduction of k_colfft_dense spans one warp");
  // set on every call: the attribute belongs to the current device's context
  const cudaError_t attr =
      cudaFuncSetAttribute(k_colfft_dense<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM_A_FIXED);
  if (attr != cudaSuccess) return attr;
  float2* T = reinterpret_cast<float2*>(d.scratch);
  StatPartial* partials = reinterpret_cast<StatPartial*>(d.scratch + kTBytes);
  float* colsq = reinterpret_cast<float*>(d.scratch + kTBytes + kPartialBytes);
  float* mean0 = colsq + kMaxN / 2;
  const float2* tw = d.twiddle + twiddle_offset(N);
  constexpr int NC = N / 2;
  k_colfft_dense<N><<<(NC + K::XA - 1) / K::XA, K::T * K::XA, K::SMEM_A_FIXED, st>>>(grid, T, tw, colsq, mean0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SegmentGeom g{};
  g.npix = N;
  g.ncol = NC;
  g.tsplit = 1;  // k_colfft_dense stores T in natural row order
  DevTables tb{};
  tb.twiddle = tw;
  tb.twiddle_col = tw;
  e = launch_rowfft_stats(g, tb, T, 1, 0, nullptr, partials, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  k_noalloc_finalize<<<1, 32, 0, st>>>(partials, K::PARTIALS, colsq, mean0, N, weight, out);
  return cudaGetLastError();
}


}  // namespace
}  // namespace rf

extern "C" rf_status rf_image_stats_noalloc(const void* half_plane, int32_t npix, double weight, void* stream,
                                            rf_image_stat* stat) {
  using namespace rf;
  char buf[256];
  if (!half_plane || !stat) {
    set_last_error("rf_image_stats_noalloc: half_plane and stat must be device pointers");
    return RF_ERR_INVALID_ARG;
  }
  if (npix < 16 || (npix & (npix - 1)) || npix > RF_NOALLOC_MAX_NPIX) {
    snprintf(buf, sizeof(buf),
             "rf_image_stats_noalloc: npix %d must be a power of two in [16, %d] (the size of its static scratch)",
             npix, RF_NOALLOC_MAX_NPIX);
    set_last_error(buf);
    return RF_ERR_INVALID_ARG;
  }
  if (!(weight > 0.0) || !std::isfinite(weight)) {
    set_last_error("rf_image_stats_noalloc: weight must be > 0");
    return RF_ERR_INVALID_ARG;
  }
  if ((uintptr_t)half_plane % 8 != 0 || (uintptr_t)stat % alignof(rf_image_stat) != 0) {
    snprintf(buf, sizeof(buf), "rf_image_stats_noalloc: half_plane must be 8-byte and stat %zu-byte aligned",
             alignof(rf_image_stat));
    set_last_error(buf);
    return RF_ERR_INVALID_ARG;
  }
  // Both pointers must be device memory of the current device: a kernel
  // given host memory would fault (or, where the device can reach host
  // memory, silently read and write it).  The query allocates nothing.
  int dev = -1;
  const bool have_dev = cudaGetDevice(&dev) == cudaSuccess && dev >= 0;
  for (const void* ptr : {half_plane, static_cast<const void*>(stat)}) {
    cudaPointerAttributes attr;
    const bool ok = have_dev && cudaPointerGetAttributes(&attr, ptr) == cudaSuccess &&
                    (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == dev;
    if (!ok) {
      cudaGetLastError();
      set_last_error("rf_image_stats_noalloc: half_plane and stat must be device memory of the current device");
      return RF_ERR_INVALID_ARG;
    }
  }
  cudaError_t e = cudaSuccess;
  if (dev >= kMaxDevices) {
    set_last_error("rf_image_stats_noalloc: device ordinal beyond the set-up table");
    return RF_ERR_NO_DEVICE;
  }
  DeviceSetup* d = nullptr;
  rf_status s = ensure_setup(dev, &d);
  if (s != RF_OK) return s;
  const float2* grid = static_cast<const float2*>(half_plane);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (npix) {
    case 16: e = run_noalloc<16>(grid, weight, *d, st, stat); break;
    case 32: e = run_noalloc<32>(grid, weight, *d, st, stat); break;
    case 64: e = run_noalloc<64>(grid, weight, *d, st, stat); break;
    case 128: e = run_noalloc<128>(grid, weight, *d, st, stat); break;
    case 256: e = run_noalloc<256>(grid, weight, *d, st, stat); break;
    case 512: e = run_noalloc<512>(grid, weight, *d, st, stat); break;
    case 1024: e = run_noalloc<1024>(grid, weight, *d, st, stat); break;
    default: e = cudaErrorInvalidValue; break;
  }
  if (e != cudaSuccess) {
    snprintf(buf, sizeof(buf), "rf_image_stats_noalloc: launch failed: %s", cudaGetErrorString(e));
    set_last_error(buf);
    return RF_ERR_CUDA;
  }
  return RF_OK;
}
