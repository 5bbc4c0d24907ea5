// rf_kernels.cu -- Stokes-I ingest, per-image weights, per-image finalisation
// (noise, S/N, threshold, candidate append) and the launch dispatch by image
// size for the imaging kernels.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <type_traits>

#include "rf_async.cuh"
#include "rf_engine.h"

namespace rf {

void fft_twiddle_table(int n, float2* out) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < n; ++m) {
    const double a = two_pi * (double)m / (double)n;
    out[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  const int p2 = fft_pass2_radix(n);
  const int len = 32 * p2;
  for (int r = 0; r < p2; ++r)
    for (int k = 0; k < 32; ++k) {
      const double a = two_pi * (double)((k * r) % len) / (double)len;
      out[n + (r >> 1) * 64 + 2 * k + (r & 1)] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  if (n == 2048)
    for (int r = 0; r < 32; ++r)
      for (int k = 0; k < 32; ++k) {
        const double a = two_pi * (double)((r * (2 * k + 1)) % n) / (double)n;
        out[n + len + (r >> 1) * 64 + 2 * k + (r & 1)] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
}

int sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 1;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return 1;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// ----------------------------------------------------------------- ingest --
// Stokes I (Sec. 3.1: a Stokes I image; Table 1: two polarisations) is the
// mean of the polarisations.  The input [t][b][c][p] is transposed through a
// 32x32 shared tile into the time-major S[c * nbl + b][t] so that the
// dedispersion gathers of consecutive t' read consecutive addresses.
template <bool FP16, int NPOL>
__global__ void __launch_bounds__(256) k_ingest(const float2* __restrict__ vis, int nt, int t_begin, int nbl,
                                                int nchan, int nint_pad, void* __restrict__ S) {
  __shared__ float2 tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nq = nbl * nchan;
  const int q0 = blockIdx.x * 32;
  const int t0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int tt = t0 + ty + 8 * k;
    const int q = q0 + tx;
    float2 s = make_float2(0.f, 0.f);
    if (tt < nt && q < nq) {
      if (NPOL == 2) {
        const float4 p = __ldg(reinterpret_cast<const float4*>(vis) + (size_t)tt * nq + q);
        s = make_float2(0.5f * (p.x + p.z), 0.5f * (p.y + p.w));
      } else {
        s = __ldg(vis + (size_t)tt * nq + q);
      }
    }
    tile[ty + 8 * k][tx] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = q0 + ty + 8 * k;
    const int tt = t0 + tx;
    if (q < nq && tt < nt) {
      const int b = q / nchan;
      const int c = q - b * nchan;
      const size_t o = (size_t)(c * nbl + b) * nint_pad + t_begin + tt;
      const float2 v = tile[tx][ty + 8 * k];
      if (FP16)
        reinterpret_cast<__half2*>(S)[o] = __floats2half2_rn(v.x, v.y);
      else
        reinterpret_cast<float2*>(S)[o] = v;
    }
  }
}

cudaError_t launch_ingest(const float2* vis, int nt, int t_begin, int npol, const SegmentGeom& g, void* S,
                          cudaStream_t st) {
  if (nt <= 0) return cudaSuccess;
  const int nq = g.nbl * g.nchan;
  dim3 grid((nq + 31) / 32, (nt + 31) / 32);
  dim3 block(32, 8);
  if (npol == 2) {
    if (g.fp16)
      k_ingest<true, 2><<<grid, block, 0, st>>>(vis, nt, t_begin, g.nbl, g.nchan, g.nint_pad, S);
    else
      k_ingest<false, 2><<<grid, block, 0, st>>>(vis, nt, t_begin, g.nbl, g.nchan, g.nint_pad, S);
  } else {
    if (g.fp16)
      k_ingest<true, 1><<<grid, block, 0, st>>>(vis, nt, t_begin, g.nbl, g.nchan, g.nint_pad, S);
    else
      k_ingest<false, 1><<<grid, block, 0, st>>>(vis, nt, t_begin, g.nbl, g.nchan, g.nint_pad, S);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------- mean subtract --
// Mean-visibility subtraction over the segment (Sec. 3.1): every row of S
// (one baseline and channel) loses its mean over t < nint, which removes
// sources that are constant over the segment.  One warp per row; lane l sums
// t = l, l + 32, ... (FP32 over runs of 32 samples, FP64 above) and a fixed
// xor-shuffle tree combines the lanes in FP64,
// so the mean does not depend on scheduling.  The difference is formed in
// FP32 and stored back in the storage precision.
template <bool FP16>
__global__ void __launch_bounds__(256) k_mean_subtract(void* __restrict__ S, int nrows, int nint, int nint_pad) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;
  const size_t base = (size_t)row * nint_pad;
  // FP32 over each lane's runs of 32 samples, FP64 above (the FP64 pipe is
  // narrow on this part)
  double sr = 0.0, si = 0.0;
  for (int t0 = lane; t0 < nint; t0 += 32 * 32) {
    float fr = 0.f, fi = 0.f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const int t = t0 + 32 * j;
      if (t < nint) {
        float2 v;
        if (FP16)
          v = __half22float2(reinterpret_cast<const __half2*>(S)[base + t]);
        else
          v = reinterpret_cast<const float2*>(S)[base + t];
        fr += v.x;
        fi += v.y;
      }
    }
    sr += (double)fr;
    si += (double)fi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  const float mr = (float)(sr / (double)nint);
  const float mi = (float)(si / (double)nint);
  for (int t = lane; t < nint; t += 32) {
    if (FP16) {
      __half2* q = reinterpret_cast<__half2*>(S) + base + t;
      const float2 v = __half22float2(*q);
      *q = __floats2half2_rn(v.x - mr, v.y - mi);
    } else {
      float2* q = reinterpret_cast<float2*>(S) + base + t;
      const float2 v = *q;
      *q = make_float2(v.x - mr, v.y - mi);
    }
  }
}

cudaError_t launch_mean_subtract(const SegmentGeom& g, void* S, cudaStream_t st) {
  const int nrows = g.nbl * g.nchan;
  if (nrows <= 0 || g.nint <= 0) return cudaSuccess;
  if (g.fp16)
    k_mean_subtract<true><<<(nrows + 7) / 8, 256, 0, st>>>(S, nrows, g.nint, g.nint_pad);
  else
    k_mean_subtract<false><<<(nrows + 7) / 8, 256, 0, st>>>(S, nrows, g.nint, g.nint_pad);
  return cudaGetLastError();
}

// --------------------------------------------------------------- resample --
// Boxcar resampling over dt integrations (Sec. 2.2: matched filters over
// pulse width; Fig. 2: the loop over sampling time), computed once per
// segment and width: out[row][p][i] = sum_{j<dt} S[row][i dt + p + j], the
// j in order, samples at or past nint counted as absent.  The phase-split
// layout makes the dedispersion gather of consecutive t' read consecutive
// addresses for every dt: sample t' dt + delta lives at phase delta mod dt,
// index t' + delta div dt.  The sums are FP32 and stored as FP32 whatever
// the storage of S (FP16 storage applies to the visibilities only).
template <bool FP16>
__global__ void __launch_bounds__(256) k_resample(const void* __restrict__ S, void* __restrict__ out, int nrows,
                                                  int nint, int nint_pad, int dt, int lp) {
  const size_t pitch = (size_t)dt * lp;
  const size_t total = (size_t)nrows * pitch;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
    const size_t row = o / pitch;
    const int rem = (int)(o - row * pitch);
    const int p = rem / lp;
    const int i = rem - p * lp;
    const int t = i * dt + p;
    float2 a = make_float2(0.f, 0.f);
    const size_t base = row * (size_t)nint_pad;
    for (int j = 0; j < dt; ++j) {
      if (t + j < nint) {
        float2 v;
        if (FP16)
          v = __half22float2(reinterpret_cast<const __half2*>(S)[base + t + j]);
        else
          v = reinterpret_cast<const float2*>(S)[base + t + j];
        a.x += v.x;
        a.y += v.y;
      }
    }
    reinterpret_cast<float2*>(out)[o] = a;
  }
}

cudaError_t launch_resample(const SegmentGeom& g, const void* S, void* Sdt, int dt, int lp, cudaStream_t st) {
  const int nrows = g.nbl * g.nchan;
  const size_t total = (size_t)nrows * dt * lp;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)sm_count() * 16);
  if (g.fp16)
    k_resample<true><<<blocks, 256, 0, st>>>(S, Sdt, nrows, g.nint, g.nint_pad, dt, lp);
  else
    k_resample<false><<<blocks, 256, 0, st>>>(S, Sdt, nrows, g.nint, g.nint_pad, dt, lp);
  return cudaGetLastError();
}

// --------------------------------------------------------------- gridding --
// Dedispersion + resampling + nearest-neighbour gridding (Sec. 2.2, 3.1) of
// a group of up to 32 consecutive output integrations t0 .. t0+31 of one
// (DM, dt) trial.  Lane k of every warp is image t0 + k: it reads sample
// t' dt + delta[d][c] of the dt-resampled series (phase delta mod dt, index
// t' + delta div dt), so one load instruction reads 32 consecutive samples.
// Each warp walks one host-made, cell-aligned range of gridding entries
// (sorted by cell), 32 entries at a time: lane l turns entry l into the
// series offset of its sample for t' = 0 and a word holding its cell and
// flags (and, under the PARTIAL edge rule, how many lanes have the sample);
// those are broadcast by shuffle, with kGatherBatch sample loads in flight
// per lane.  Every cell is summed in registers in a fixed order
//   H[cell] = sum_entries (-1)^(iu+iv) R  (or conj R for folded entries)
// and its 32 values are written to cellbuf[group][cell][k] (one 256-byte
// row).  No atomics: the grid is bitwise reproducible.
template <bool FP16>
__device__ __forceinline__ float2 load_s(const unsigned char* __restrict__ S, size_t i) {
  if (FP16) return __half22float2(__ldg(reinterpret_cast<const __half2*>(S) + i));
  return __ldg(reinterpret_cast<const float2*>(S) + i);
}

constexpr int kGatherBatch = 4;  // samples each lane has in flight (swept: 4 at 6 blocks per SM beat 8-32 at 2-5)

// Cell index and entry flags in one word: cells < 2^30 (at most (N/2 + 1) N
// for N <= 8192); bit 30 = ENT_CONJ, bit 31 = ENT_NEG.
constexpr unsigned kCellMask = (1u << 30) - 1u;

// One warp's range r of gridding entries for group gr; FP16 is the sample
// type of the series the group reads (S itself at dt = 1 under FP16 storage;
// the resampled series are FP32).
template <bool FP16, bool IDX32, bool PARTIAL>
__device__ __forceinline__ void grid_range(const SegmentGeom& g, const DevTables& tb, const Group& gr,
                                           const int* __restrict__ sdel, int lane, int r,
                                           float2* __restrict__ cellbuf) {
  using Off = typename std::conditional<IDX32, unsigned, unsigned long long>::type;
  const int2 rg = tb.ranges[r];
  const int ebeg = rg.x, eend = rg.y;
  const int dt = tb.dt_list[gr.s];
  const int lp = tb.sdt_lp[gr.s];
  const unsigned char* __restrict__ Sd = reinterpret_cast<const unsigned char*>(tb.sdt_ptr[gr.s]);
  const Off rowpitch = (Off)dt * (Off)lp;
  const bool active = lane < gr.nimg;
  const Off tq = (Off)(gr.t0 + lane);
  float2* __restrict__ out = cellbuf + (size_t)blockIdx.x * g.ncells * 32 + lane;
  float2 acc = make_float2(0.f, 0.f);
  unsigned cur = 0xffffffffu;
  GridEntry nxt = {0, 0, 0, -1};
  if (ebeg + lane < eend) nxt = tb.ent[ebeg + lane];
  for (int base = ebeg; base < eend; base += 32) {
    const GridEntry my = nxt;
    const bool mine = base + lane < eend;
    if (base + 32 + lane < eend) nxt = tb.ent[base + 32 + lane];
    const int mydel = mine ? sdel[my.cflags >> 2] : 0;
    // sample t' dt + delta lives at phase delta mod dt, index t' + delta div dt
    const Off myoff = (Off)my.bc * rowpitch + (Off)((mydel % dt) * lp + mydel / dt);
    const unsigned mycf = ((unsigned)my.cell & kCellMask) | ((unsigned)(my.cflags & 3) << 30);
    // PARTIAL: lanes k with (t0 + k) dt + delta < nint have the sample
    int mylim = 32;
    if (PARTIAL) {
      const int rem = g.nint - mydel - 1;
      mylim = rem < 0 ? 0 : max(0, min(32, rem / dt - gr.t0 + 1));
    }
    const int n = min(32, eend - base);
    for (int i0 = 0; i0 < n; i0 += kGatherBatch) {
      float2 a[kGatherBatch];
#pragma unroll
      for (int q = 0; q < kGatherBatch; ++q) {
        const int i = (i0 + q) & 31;
        Off off;
        if (IDX32)
          off = __shfl_sync(0xffffffffu, myoff, i);
        else
          off = (Off)__shfl_sync(0xffffffffu, (unsigned long long)myoff, i);
        bool ok = active && i0 + q < n;
        if (PARTIAL) {
          const int lim = __shfl_sync(0xffffffffu, mylim, i);  // every lane takes part in the shuffle
          ok = ok && lane < lim;
        }
        a[q] = make_float2(0.f, 0.f);
        if (ok) a[q] = load_s<FP16>(Sd, (size_t)(off + tq));
      }
#pragma unroll
      for (int q = 0; q < kGatherBatch; ++q) {
        const unsigned cf = __shfl_sync(0xffffffffu, mycf, (i0 + q) & 31);
        if (i0 + q < n) {
          const unsigned cell = cf & kCellMask;
          const bool flush = cell != cur;  // the same on every lane
          if (flush && cur != 0xffffffffu) out[(size_t)cur * 32] = acc;
          acc.x = flush ? 0.f : acc.x;
          acc.y = flush ? 0.f : acc.y;
          cur = cell;
          // sign of the real part: ENT_NEG; of the imaginary part: ENT_NEG ^ ENT_CONJ
          const unsigned sx = cf & 0x80000000u;
          const unsigned sy = (cf ^ (cf << 1)) & 0x80000000u;
          acc.x += __uint_as_float(__float_as_uint(a[q].x) ^ sx);
          acc.y += __uint_as_float(__float_as_uint(a[q].y) ^ sy);
        }
      }
    }
  }
  if (cur != 0xffffffffu) out[(size_t)cur * 32] = acc;
}

// FP16: the plan stores S in FP16 (the dt = 1 series); every resampled
// series (dt > 1) is FP32.
template <bool FP16, bool IDX32, bool PARTIAL>
__global__ void __launch_bounds__(256, 6) k_grid_cells(SegmentGeom g, DevTables tb, const Group* __restrict__ groups,
                                                    int g_begin, float2* __restrict__ cellbuf) {
  extern __shared__ int sdel[];  // [nchan] delays of this group's DM
  const int tid = threadIdx.x;
  const Group gr = groups[g_begin + blockIdx.x];
  {
    const int* __restrict__ dl = tb.delays + (size_t)gr.d * g.nchan;
    for (int c = tid; c < g.nchan; c += blockDim.x) sdel[c] = dl[c];
  }
  __syncthreads();
  const int r = blockIdx.y * (blockDim.x >> 5) + (tid >> 5);
  if (r >= g.nranges) return;
  if constexpr (FP16) {
    if (tb.dt_list[gr.s] == 1) {
      grid_range<true, IDX32, PARTIAL>(g, tb, gr, sdel, tid & 31, r, cellbuf);
      return;
    }
  }
  grid_range<false, IDX32, PARTIAL>(g, tb, gr, sdel, tid & 31, r, cellbuf);
}

cudaError_t launch_grid_cells(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                              int ngroups, float2* cellbuf, cudaStream_t st) {
  if (ngroups <= 0 || g.nranges <= 0) return cudaSuccess;
  dim3 grid(ngroups, (g.nranges + 7) / 8);
  const int smem = g.nchan * 4;
#define RF_GRID(F16, I32, PART) \
  k_grid_cells<F16, I32, PART><<<grid, 256, smem, st>>>(g, tb, groups, g_begin, cellbuf)
  if (g.fp16) {
    if (g.idx32) {
      if (g.partial) RF_GRID(true, true, true); else RF_GRID(true, true, false);
    } else {
      if (g.partial) RF_GRID(true, false, true); else RF_GRID(true, false, false);
    }
  } else {
    if (g.idx32) {
      if (g.partial) RF_GRID(false, true, true); else RF_GRID(false, true, false);
    } else {
      if (g.partial) RF_GRID(false, false, true); else RF_GRID(false, false, false);
    }
  }
#undef RF_GRID
  return cudaGetLastError();
}

// ---------------------------------------------------------------- weights --
// W = sum over on-grid (b, c) of the samples summed into R[b, c].  Under the
// FULL edge rule every channel sums dt samples; under PARTIAL channel c sums
// clamp(nint - (t dt + delta[d][c]), 0, dt) of them.
__global__ void k_weights(const int4* __restrict__ img_info, int nimg, int partial, int nint, int nchan,
                          const int* __restrict__ delays, const int* __restrict__ dt_list,
                          const int* __restrict__ ongrid_chan, double n_on, double* __restrict__ weight) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nimg) return;
  const int4 info = img_info[i];
  const int dt = dt_list[info.y];
  if (!partial) {
    weight[i] = (double)dt * n_on;
    return;
  }
  const int* dl = delays + (size_t)info.x * nchan;
  const int tb = info.z * dt;
  long long w = 0;
  for (int c = 0; c < nchan; ++c) {
    int n = nint - (tb + dl[c]);
    n = n < 0 ? 0 : (n > dt ? dt : n);
    w += (long long)n * ongrid_chan[c];
  }
  weight[i] = (double)w;
}

cudaError_t launch_weights(const int4* img_info, int nimg, bool partial, const SegmentGeom& g,
                           const DevTables& tb, double n_on, double* weight, cudaStream_t st) {
  if (nimg <= 0) return cudaSuccess;
  k_weights<<<(nimg + 255) / 256, 256, 0, st>>>(img_info, nimg, partial ? 1 : 0, g.nint, g.nchan, tb.delays,
                                                 tb.dt_list, tb.ongrid_chan, n_on, weight);
  return cudaGetLastError();
}

// --------------------------------------------------------------- finalize --
// Per image: reduce the row-block partials (FP64), then
//   mean = sum / N^2,  sigma = sqrt(sum_sq / N^2 - mean^2)  (population),
//   peak = max pixel (lowest y N + x on ties),  snr = peak / sigma,
// and append a candidate iff snr >= threshold (Sec. 3.1).  Raw pixel sums are
// scaled by 1 / (2 W) here.
__device__ __forceinline__ void fmax_merge(float& m, int& i, float m2, int i2) {
  if (m2 > m || (m2 == m && i2 < i)) {
    m = m2;
    i = i2;
  }
}

// Sum over the ncol Parseval column sums of one image, lanes strided and an
// xor tree (fixed order); every lane holds the result.
__device__ __forceinline__ double parseval_sum(const float* __restrict__ cs, int ncol, int lane) {
  double sq = 0.0;
  for (int c = lane; c < ncol; c += 32) sq += (double)cs[c];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
  return sq;
}

// One warp per image slot: the clipping window {mean, kClipSigmas sigma} of
// the raw image J = 2W I.  mean(J) = Re G(0, 0) and mean(J^2) = the sum of
// |G|^2 over the full plane (Parseval), so var(J) = sum - mean^2.
__global__ void k_clip_window(int ncol, const float* __restrict__ colsq, const float* __restrict__ mean0, int nimg,
                              float2* __restrict__ clip) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= nimg) return;
  const double sq = parseval_sum(colsq + (size_t)i * ncol, ncol, lane);
  if (lane != 0) return;
  const float m = mean0[i];
  double var = sq - (double)m * (double)m;
  var = var > 0.0 ? var : 0.0;
  clip[i] = make_float2(m, (float)(kClipSigmas * sqrt(var)));
}

cudaError_t launch_clip_window(const SegmentGeom& g, const float* colsq, const float* mean0, int nimg, float2* clip,
                               cudaStream_t st) {
  if (nimg <= 0) return cudaSuccess;
  k_clip_window<<<(nimg + 7) / 8, 256, 0, st>>>(g.ncol, colsq, mean0, nimg, clip);
  return cudaGetLastError();
}

__global__ void k_finalize(int npix, int nrb, int ncol, const StatPartial* __restrict__ partials,
                           const float* __restrict__ colsq, const float* __restrict__ mean0,
                           const int4* __restrict__ img_info, const double* __restrict__ weight, int nimg,
                           int img_base, double threshold, DevCand* __restrict__ cands, int* __restrict__ ncand,
                           int cand_cap, DevStat* __restrict__ stats, int clip) {
  // one warp per image; lanes stride over the row-pair partials (peak, and
  // the kept-pixel sums of the clipped noise) and the per-column Parseval
  // sums (FP64), then an xor-tree (fixed order) combines them
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= nimg) return;
  const int img = img_base + i;
  const StatPartial* pp = partials + (size_t)i * nrb;
  float mx = -FLT_MAX;
  int mi = INT_MAX;
  double ks1 = 0.0, ks2 = 0.0;
  long long kn = 0;
  for (int r = lane; r < nrb; r += 32) {
    const StatPartial p = pp[r];
    fmax_merge(mx, mi, p.max, p.idx);
    if (clip) {
      ks1 += p.sum;
      ks2 += p.sumsq;
      kn += p.kept;
    }
  }
  const double sq = parseval_sum(colsq + (size_t)i * ncol, ncol, lane);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float om = __shfl_xor_sync(0xffffffffu, mx, off);
    const int oi = __shfl_xor_sync(0xffffffffu, mi, off);
    fmax_merge(mx, mi, om, oi);
    if (clip) {
      ks1 += __shfl_xor_sync(0xffffffffu, ks1, off);
      ks2 += __shfl_xor_sync(0xffffffffu, ks2, off);
      kn += __shfl_xor_sync(0xffffffffu, kn, off);
    }
  }
  if (lane != 0) return;
  const double W = weight[img];
  const int4 info = img_info[img];
  DevStat ds;
  ds.pad = 0;
  ds.weight = W;
  if (!(W > 0.0)) {
    ds.peak = 0.f;
    ds.sigma = 0.f;
    ds.snr = 0.f;
    ds.x = 0;
    ds.y = 0;
    ds.mean = 0.0;
    if (stats) stats[img] = ds;
    return;
  }
  // mean = G(0,0) / 2W; mean of I^2 = sum_full |G|^2 / 4W^2 (Parseval)
  const double inv = 0.5 / W;
  double mean = (double)mean0[i] * inv;
  double var = sq * inv * inv - mean * mean;
  if (clip) {
    // clipped noise: the kept pixels' deviations d from mean0 (raw units)
    const double n = kn > 0 ? (double)kn : 1.0;
    const double m1 = ks1 / n;
    mean = ((double)mean0[i] + m1) * inv;
    var = (ks2 / n - m1 * m1) * inv * inv;
  }
  var = var > 0.0 ? var : 0.0;
  const double sigma = sqrt(var);
  const double peak = (double)mx * inv;
  const double snr = sigma > 0.0 ? peak / sigma : 0.0;
  const int y = mi / npix;
  const int x = mi - y * npix;
  ds.peak = (float)peak;
  ds.sigma = (float)sigma;
  ds.snr = (float)snr;
  ds.x = x;
  ds.y = y;
  ds.mean = mean;
  if (stats) stats[img] = ds;
  if (sigma > 0.0 && snr >= threshold) {
    const int k = atomicAdd(ncand, 1);
    if (k < cand_cap) {
      DevCand c;
      c.d = info.x;
      c.s = info.y;
      c.t = info.z;
      c.x = x;
      c.y = y;
      c.snr = (float)snr;
      c.peak = (float)peak;
      c.sigma = (float)sigma;
      cands[k] = c;
    }
  }
}

cudaError_t launch_finalize(const SegmentGeom& g, const StatPartial* partials, const float* colsq,
                            const float* mean0, const int4* img_info, const double* weight, int nimg, int img_base,
                            double threshold, DevCand* cands, int* ncand, int cand_cap, DevStat* stats,
                            cudaStream_t st, bool clip) {
  if (nimg <= 0) return cudaSuccess;
  ImageKernelShape sh;
  if (!image_kernel_shape(g.npix, &sh)) return cudaErrorInvalidValue;
  const int nrb = sh.partials_per_image;
  k_finalize<<<(nimg + 7) / 8, 256, 0, st>>>(g.npix, nrb, g.ncol, partials, colsq, mean0, img_info, weight, nimg,
                                              img_base, threshold, cands, ncand, cand_cap, stats, clip ? 1 : 0);
  return cudaGetLastError();
}

// --------------------------------------------------------------- dispatch --
template <int N>
cudaError_t run_colfft(const SegmentGeom&, const DevTables&, const Group*, int, int, int, const float2*, float2*,
                       float*, float*, cudaStream_t, const PassLaunch*);
template <int N>
cudaError_t run_rowfft_stats(const SegmentGeom&, const DevTables&, const float2*, int, int, const double*,
                             StatPartial*, float*, const TileMap*, int*, cudaStream_t, const float2*,
                             const PassLaunch*);
template <int N>
void fill_shape(ImageKernelShape*);
template <int N>
cudaError_t run_rowfft_power(const SegmentGeom&, const DevTables&, const float2*, const int4*, int, StatPartial*,
                             const TileMap*, int*, cudaStream_t);

template <int N>
cudaError_t run_image_fused(const SegmentGeom&, const DevTables&, const Group*, int, const FusedChunk*, int, int,
                            const float2*, float2*, int, const TileMap&, float*, float*, StatPartial*, int*, int*,
                            cudaStream_t);

#define RF_FOR_EACH_N(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

int fused_chunk_images(int npix) {
  switch (npix) {
    case 1024: return 8;
    case 2048: return RF_ROW_VALUES_2048 == 32 ? 4 : 0;
    case 4096: return 2;
    default: return 0;
  }
}

cudaError_t launch_image_fused(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                               const FusedChunk* chunks, int nchunks, int img_base, const float2* cellbuf,
                               float2* Tring, int ring, const TileMap& tm, float* colsq, float* mean0,
                               StatPartial* partials, int* counters, int* err, cudaStream_t st) {
  switch (g.npix) {
#define RF_CASE(N)                                                                                               \
  case N:                                                                                                        \
    return run_image_fused<N>(g, tb, groups, g_begin, chunks, nchunks, img_base, cellbuf, Tring, ring, tm, colsq, \
                              mean0, partials, counters, err, st);
    RF_CASE(1024) RF_CASE(4096)
#if RF_ROW_VALUES_2048 == 32
    RF_CASE(2048)
#endif
#undef RF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_colfft(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                          int ngroups, int img_base, const float2* cellbuf, float2* Tbuf, float* colsq,
                          float* mean0, cudaStream_t st, const PassLaunch* pl) {
  switch (g.npix) {
#define RF_CASE(N) \
  case N:          \
    return run_colfft<N>(g, tb, groups, g_begin, ngroups, img_base, cellbuf, Tbuf, colsq, mean0, st, pl);
    RF_FOR_EACH_N(RF_CASE)
#undef RF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rowfft_stats(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, int nimg,
                                int img_base, const double* weight, StatPartial* partials, float* images,
                                const TileMap* tm, int* err, cudaStream_t st, const float2* clip,
                                const PassLaunch* pl) {
  switch (g.npix) {
#define RF_CASE(N) \
  case N:          \
    return run_rowfft_stats<N>(g, tb, Tbuf, nimg, img_base, weight, partials, images, tm, err, st, clip, pl);
    RF_FOR_EACH_N(RF_CASE)
#undef RF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rowfft_power(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, const int4* pairs,
                                int npairs, StatPartial* partials, const TileMap* tm, int* err, cudaStream_t st) {
  switch (g.npix) {
#define RF_CASE(N) \
  case N:          \
    return run_rowfft_power<N>(g, tb, Tbuf, pairs, npairs, partials, tm, err, st);
    RF_FOR_EACH_N(RF_CASE)
#undef RF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

bool image_kernel_shape(int npix, ImageKernelShape* out) {
  switch (npix) {
#define RF_CASE(N)      \
  case N:               \
    fill_shape<N>(out); \
    return true;
    RF_FOR_EACH_N(RF_CASE)
#undef RF_CASE
    default:
      return false;
  }
}

}  // namespace rf

// ------------------------------------------------------ bounded-wait check --
namespace rf {
namespace {
// The two kinds of bounded device-side wait, each on something that never
// comes: the row pass's mbarrier wait for a tile copy (on a barrier that
// nothing arrives at) and the fused pass's wait for a global count (on
// status[1], which stays 0).  Each must give up and report it instead of
// hanging: status[0] gets bit 0 for the first, bit 1 for the second.
__global__ void k_wait_selftest(int polls, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, polls);
  const bool gave_up_bar = __syncthreads_or(!ok);
  if (threadIdx.x == 0) {
    const bool gave_up_count = !wait_count(status + 1, 1, status + 1, polls);
    *status = (gave_up_bar ? 1 : 0) | (gave_up_count ? 2 : 0);
  }
}
}  // namespace

cudaError_t launch_wait_selftest(int polls, int* status, cudaStream_t st) {
  k_wait_selftest<<<1, 64, 0, st>>>(polls, status);
  return cudaGetLastError();
}
}  // namespace rf
