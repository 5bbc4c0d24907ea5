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

#include <algorithm>

#include "rf_engine.h"

namespace rf {

namespace {

template <bool FP16>
__device__ __forceinline__ float2 load_resampled(const unsigned char* base, size_t i) {
  if (FP16) return __half22float2(reinterpret_cast<const __half2*>(base)[i]);
  return reinterpret_cast<const float2*>(base)[i];
}

// One warp per (candidate, channel); lanes stride over the baselines.
// FP16: S is stored in FP16, which the dt = 1 series reads; the resampled
// series (dt > 1) are FP32.
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
      const float2 v = (FP16 && dt == 1) ? load_resampled<true>(Sd, (size_t)row * rowpitch + part)
                                         : load_resampled<false>(Sd, (size_t)row * rowpitch + part);
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

// Population moments of all pixels of each image, in two passes over slices
// of the image so that every SM takes part: block (slice, image) sums its
// pixels (FP32 over 32 pixels per thread step, FP64 above), then around the
// image mean (combined from the slice sums in a fixed order) the sums of d^2,
// d^3 and d^4, d = pixel - mean, in the same way; a warp per image combines
// the slices in a fixed order.  out[k] = {mean, std, skew, excess kurtosis}.
__device__ __forceinline__ void slice_range(size_t npx, int nslices, int s, size_t* b, size_t* e) {
  const size_t per = (npx + nslices - 1) / nslices;
  *b = min(npx, (size_t)s * per);
  *e = min(npx, *b + per);
}

__global__ void __launch_bounds__(kMomThreads) k_moments_sum(const float* __restrict__ images, size_t npx,
                                                             int nslices, double* __restrict__ part) {
  __shared__ double sh[kMomThreads];
  const int sl = blockIdx.x, k = blockIdx.y;
  const float* im = images + (size_t)k * npx;
  size_t b, e;
  slice_range(npx, nslices, sl, &b, &e);
  double acc = 0.0;
  for (size_t i0 = b + threadIdx.x; i0 < e; i0 += (size_t)kMomThreads * 32) {
    float f = 0.f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const size_t i = i0 + (size_t)j * kMomThreads;
      if (i < e) f += im[i];
    }
    acc += (double)f;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[((size_t)k * nslices + sl) * 4] = acc;
}

__global__ void __launch_bounds__(kMomThreads) k_moments_central(const float* __restrict__ images, size_t npx,
                                                                 int nslices, double* __restrict__ part) {
  __shared__ double sh[kMomThreads];
  const int sl = blockIdx.x, k = blockIdx.y;
  const float* im = images + (size_t)k * npx;
  double* pk = part + (size_t)k * nslices * 4;
  double sum = 0.0;
  for (int q = 0; q < nslices; ++q) sum += pk[(size_t)q * 4];
  const float mu = (float)(sum / (double)npx);
  size_t b, e;
  slice_range(npx, nslices, sl, &b, &e);
  double m2 = 0.0, m3 = 0.0, m4 = 0.0;
  for (size_t i0 = b + threadIdx.x; i0 < e; i0 += (size_t)kMomThreads * 32) {
    float f2 = 0.f, f3 = 0.f, f4 = 0.f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      const size_t i = i0 + (size_t)j * kMomThreads;
      if (i < e) {
        const float d = im[i] - mu;
        const float d2 = d * d;
        f2 += d2;
        f3 = fmaf(d2, d, f3);
        f4 = fmaf(d2, d2, f4);
      }
    }
    m2 += (double)f2;
    m3 += (double)f3;
    m4 += (double)f4;
  }
  m2 = block_sum(m2, sh);
  m3 = block_sum(m3, sh);
  m4 = block_sum(m4, sh);
  if (threadIdx.x == 0) {
    double* o = pk + (size_t)sl * 4;
    o[1] = m2;
    o[2] = m3;
    o[3] = m4;
  }
}

__global__ void k_moments_final(const double* __restrict__ part, size_t npx, int nslices, int n,
                                double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* pk = part + (size_t)k * nslices * 4;
  double sum = 0.0, m2 = 0.0, m3 = 0.0, m4 = 0.0;
  for (int q = 0; q < nslices; ++q) {
    sum += pk[(size_t)q * 4];
    m2 += pk[(size_t)q * 4 + 1];
    m3 += pk[(size_t)q * 4 + 2];
    m4 += pk[(size_t)q * 4 + 3];
  }
  const double np = (double)npx;
  const double mean = sum / np;
  // the central sums were taken about the FP32-rounded mean mu_f; move them to
  // the mean itself (e = mean - mu_f, central moments about mean from those
  // about mu_f)
  const double e = mean - (double)(float)mean;
  const double a2 = m2 / np, a3 = m3 / np, a4 = m4 / np;
  const double c2 = a2 - e * e;
  const double c3 = a3 - 3.0 * e * a2 + 2.0 * e * e * e;
  const double c4 = a4 - 4.0 * e * a3 + 6.0 * e * e * a2 - 3.0 * e * e * e * e;
  double* o = out + (size_t)k * 4;
  o[0] = mean;
  o[1] = c2 > 0 ? sqrt(c2) : 0.0;
  o[2] = c2 > 0 ? c3 / (c2 * sqrt(c2)) : 0.0;
  o[3] = c2 > 0 ? c4 / (c2 * c2) - 3.0 : 0.0;
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

int image_moment_slices(int n, size_t npx) {
  // about four blocks per SM in all, slices of at least 64K pixels
  const long want = (4L * sm_count() + n - 1) / std::max(n, 1);
  const long most = (long)std::max<size_t>(1, npx / 65536);
  return (int)std::max(1L, std::min(std::min(want, most), 256L));
}

cudaError_t launch_image_moments(const float* images, int n, size_t npx, int nslices, double* part, double* out,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid(nslices, n);
  k_moments_sum<<<grid, kMomThreads, 0, st>>>(images, npx, nslices, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_moments_central<<<grid, kMomThreads, 0, st>>>(images, npx, nslices, part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_moments_final<<<(n + 31) / 32, 32, 0, st>>>(part, npx, nslices, n, out);
  return cudaGetLastError();
}

}  // namespace rf
