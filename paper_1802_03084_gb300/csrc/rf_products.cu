// rf_products.cu -- candidate products (Sec. 3.3): statistics measured from
// each candidate's image and spectrum, and the spectrum itself for plots.
//
// Spectrum of candidate (d, s, t', x, y): per channel c, the dedispersed,
// resampled visibilities R[b,c] phased to pixel (x, y) with the image's own
// cell phases exp(+2 pi i (iu (x - N/2) + iv (y - N/2)) / N), summed over
// the on-grid baselines and divided by w_c = (on-grid baselines at c) n_c,
// n_c = samples present.  The w-weighted mean of its real part is the image
// value at (x, y).  Image moments are over the N^2 pixels, spectrum moments
// over Re(spec) at the channels with w_c > 0; both in FP64 with a fixed
// reduction order.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rf_engine.h"

namespace rf {

namespace {

template <bool FP16>
__device__ __forceinline__ float2 load_resampled(const unsigned char* base, size_t i) {
  if (FP16) return __half22float2(reinterpret_cast<const __half2*>(base)[i]);
  return reinterpret_cast<const float2*>(base)[i];
}

// One warp per (candidate, channel); lanes stride over the baselines.
template <bool FP16>
__global__ void __launch_bounds__(256) k_cand_spectrum(SegmentGeom g, DevTables tb, const int2* __restrict__ cellbc,
                                                       const CandRef* __restrict__ refs, int n,
                                                       double2* __restrict__ spec, double* __restrict__ wch,
                                                       float2* __restrict__ spec_out) {
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= n * g.nchan) return;
  const int k = warp / g.nchan;
  const int c = warp - k * g.nchan;
  const CandRef r = refs[k];
  const int N = g.npix;
  const int dt = tb.dt_list[r.s];
  const int lp = tb.sdt_lp[r.s];
  const unsigned char* Sd = reinterpret_cast<const unsigned char*>(tb.sdt_ptr[r.s]);
  const size_t rowpitch = (size_t)dt * lp;
  const int del = tb.delays[(size_t)r.d * g.nchan + c];
  const int first = r.t * dt + del;                         // first sample of the boxcar
  const int nc = max(0, min(dt, g.nint - first));           // samples present
  const size_t part = (size_t)(del % dt) * lp + del / dt + r.t;
  const int dx = r.x - N / 2, dy = r.y - N / 2;
  double sr = 0.0, si = 0.0;
  if (nc > 0) {
    for (int b = lane; b < g.nbl; b += 32) {
      const int row = c * g.nbl + b;
      const int2 cv = cellbc[row];
      if (cv.x == kOffGrid) continue;
      const float2 v = load_resampled<FP16>(Sd, (size_t)row * rowpitch + part);
      long long kk = (long long)cv.x * dx + (long long)cv.y * dy;
      int m = (int)(kk % N);
      if (m < 0) m += N;
      const float2 w = tb.twiddle[m];
      sr += (double)v.x * w.x - (double)v.y * w.y;
      si += (double)v.x * w.y + (double)v.y * w.x;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    const double wc = (double)tb.ongrid_chan[c] * nc;
    const double2 sp = wc > 0 ? make_double2(sr / wc, si / wc) : make_double2(0.0, 0.0);
    spec[(size_t)k * g.nchan + c] = sp;
    wch[(size_t)k * g.nchan + c] = wc;
    if (spec_out) spec_out[(size_t)k * g.nchan + c] = make_float2((float)sp.x, (float)sp.y);
  }
}

// Population moments of Re(spec) over the channels with data, and the
// w-weighted mean of Re(spec); one warp per candidate.
// out[k] = {mean, std, skew, excess kurtosis, weighted mean, channels used}.
__global__ void k_spec_moments(const double2* __restrict__ spec, const double* __restrict__ wch, int nchan, int n,
                               double* __restrict__ out) {
  const int k = blockIdx.x;
  const int lane = threadIdx.x;
  if (k >= n) return;
  const double2* sp = spec + (size_t)k * nchan;
  const double* w = wch + (size_t)k * nchan;
  double s = 0.0, cnt = 0.0, sw = 0.0, swr = 0.0;
  for (int c = lane; c < nchan; c += 32)
    if (w[c] > 0) {
      s += sp[c].x;
      cnt += 1.0;
      sw += w[c];
      swr += w[c] * sp[c].x;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    swr += __shfl_xor_sync(0xffffffffu, swr, o);
  }
  const double mu = cnt > 0 ? s / cnt : 0.0;
  double m2 = 0.0, m3 = 0.0, m4 = 0.0;
  for (int c = lane; c < nchan; c += 32)
    if (w[c] > 0) {
      const double d = sp[c].x - mu;
      const double d2 = d * d;
      m2 += d2;
      m3 += d2 * d;
      m4 += d2 * d2;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m2 += __shfl_xor_sync(0xffffffffu, m2, o);
    m3 += __shfl_xor_sync(0xffffffffu, m3, o);
    m4 += __shfl_xor_sync(0xffffffffu, m4, o);
  }
  if (lane == 0) {
    double* o = out + (size_t)k * 6;
    if (cnt > 0) {
      m2 /= cnt;
      m3 /= cnt;
      m4 /= cnt;
    }
    o[0] = mu;
    o[1] = sqrt(m2);
    o[2] = m2 > 0 ? m3 / (m2 * sqrt(m2)) : 0.0;
    o[3] = m2 > 0 ? m4 / (m2 * m2) - 3.0 : 0.0;
    o[4] = sw > 0 ? swr / sw : 0.0;
    o[5] = cnt;
  }
}

constexpr int kMomThreads = 256;

// Fixed-order block sum of one double per thread (kMomThreads threads).
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = kMomThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Population moments of all pixels of one image per block.
// out[k] = {mean, std, skew, excess kurtosis}.
__global__ void __launch_bounds__(kMomThreads) k_image_moments(const float* __restrict__ images, size_t npx,
                                                               double* __restrict__ out) {
  __shared__ double sh[kMomThreads];
  const float* im = images + (size_t)blockIdx.x * npx;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < npx; i += kMomThreads) s += (double)im[i];
  const double mu = block_sum(s, sh) / (double)npx;
  double m2 = 0.0, m3 = 0.0, m4 = 0.0;
  for (size_t i = threadIdx.x; i < npx; i += kMomThreads) {
    const double d = (double)im[i] - mu;
    const double d2 = d * d;
    m2 += d2;
    m3 += d2 * d;
    m4 += d2 * d2;
  }
  m2 = block_sum(m2, sh) / (double)npx;
  m3 = block_sum(m3, sh) / (double)npx;
  m4 = block_sum(m4, sh) / (double)npx;
  if (threadIdx.x == 0) {
    double* o = out + (size_t)blockIdx.x * 4;
    o[0] = mu;
    o[1] = sqrt(m2);
    o[2] = m2 > 0 ? m3 / (m2 * sqrt(m2)) : 0.0;
    o[3] = m2 > 0 ? m4 / (m2 * m2) - 3.0 : 0.0;
  }
}

}  // namespace

cudaError_t launch_cand_spectrum(const SegmentGeom& g, const DevTables& tb, const int2* cellbc, const CandRef* refs,
                                 int n, double2* spec, double* wch, float2* spec_out, double* spec_mom,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long warps = (long)n * g.nchan;
  const int blocks = (int)((warps + 7) / 8);
  if (g.fp16)
    k_cand_spectrum<true><<<blocks, 256, 0, st>>>(g, tb, cellbc, refs, n, spec, wch, spec_out);
  else
    k_cand_spectrum<false><<<blocks, 256, 0, st>>>(g, tb, cellbc, refs, n, spec, wch, spec_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_spec_moments<<<n, 32, 0, st>>>(spec, wch, g.nchan, n, spec_mom);
  return cudaGetLastError();
}

cudaError_t launch_image_moments(const float* images, int n, size_t npx, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_image_moments<<<n, kMomThreads, 0, st>>>(images, npx, out);
  return cudaGetLastError();
}

}  // namespace rf
