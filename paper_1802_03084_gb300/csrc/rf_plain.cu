// rf_plain.cu -- the plain form of the search: one unfused launch set per
// (DM, dt) trial, every intermediate stored in HBM.  It computes the same
// images as the batched form (Sec. 3.1: dedisperse, resample, grid, 2D FFT,
// threshold) in the textbook order, and exists as the per-trial baseline the
// batched form is measured against:
//   1. k_plain_dedisperse  R[bc][k] = sum_{j<dt} S[bc][(t0+k) dt + j + delta[d][c]]
//   2. k_plain_grid        dense half-plane grids, one float atomic per
//                          (entry, image) into grid[k][v][u] (u = 0 .. N/2)
//   3. k_plain_colfft      inverse FFT of every column u < N/2 (no pruning)
//   4. row pass            the shared row kernel, writing full N x N images
//   5. k_plain_stats       mean, sigma, peak of each image read back from HBM
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "rf_engine.h"
#include "rf_image.cuh"

namespace rf {

// 1. dedispersion + resampling of `nk` consecutive t' of trial (d, s) into
// R[bc][k] (k fastest); samples at or past nint are absent.
__global__ void k_plain_dedisperse(SegmentGeom g, DevTables tb, const void* __restrict__ S, int d, int s, int t0,
                                   int nk, float2* __restrict__ R) {
  const size_t total = (size_t)g.nbl * g.nchan * nk;
  const int dt = tb.dt_list[s];
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
    const int bc = (int)(o / nk);
    const int k = (int)(o - (size_t)bc * nk);
    const int c = bc / g.nbl;
    const int t = (t0 + k) * dt + tb.delays[(size_t)d * g.nchan + c];
    float2 a = make_float2(0.f, 0.f);
    for (int j = 0; j < dt; ++j) {
      if (t + j < g.nint) {
        float2 v;
        if (g.fp16)
          v = __half22float2(reinterpret_cast<const __half2*>(S)[(size_t)bc * g.nint_pad + t + j]);
        else
          v = reinterpret_cast<const float2*>(S)[(size_t)bc * g.nint_pad + t + j];
        a.x += v.x;
        a.y += v.y;
      }
    }
    R[o] = a;
  }
}

// 2. nearest-neighbour gridding into zeroed dense half planes
// grid[k][row][col] (row length N/2 + 1), checkerboard sign and Hermitian
// fold from the plan's entry table.
__global__ void k_plain_grid(SegmentGeom g, const int4* __restrict__ pent, int nent, const float2* __restrict__ R,
                             int nk, float2* __restrict__ grid) {
  const int W = g.npix / 2 + 1;
  const size_t total = (size_t)nent * nk;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(o / nk);
    const int k = (int)(o - (size_t)e * nk);
    const int4 en = pent[e];  // bc, col, row, flags
    float2 r = R[(size_t)en.x * nk + k];
    if (en.w & ENT_CONJ) r.y = -r.y;
    if (en.w & ENT_NEG) r = make_float2(-r.x, -r.y);
    float* cell = reinterpret_cast<float*>(grid + ((size_t)k * g.npix + en.z) * W + en.y);
    atomicAdd(cell, r.x);
    atomicAdd(cell + 1, r.y);
  }
}

// 3. column FFTs of the dense grids: T[k][u][y] for every u < N/2.
template <int N>
__global__ void __launch_bounds__(ImgCfg<N>::T * ImgCfg<N>::XA)
    k_plain_colfft(const float2* __restrict__ grid, float2* __restrict__ T, const float2* __restrict__ tw) {
  using K = ImgCfg<N>;
  constexpr int W = N / 2 + 1;
  constexpr int NC = N / 2;
  constexpr int THREADS = K::T * K::XA;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int col0 = blockIdx.x * K::XA;
  const int k = blockIdx.y;
  const float2* gk = grid + (size_t)k * N * W;
  for (int i = tid; i < N * K::XA; i += THREADS) {
    const int c = i % K::XA;
    const int v = i / K::XA;
    const int u = col0 + c;
    sm[c * K::STRIDE + padx(v)] = u < NC ? gk[(size_t)v * W + u] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int xf = tid / K::T;
  const int t = tid - xf * K::T;
  float2 v[K::E];
  fft_inverse_to_regs<N>(v, sm + xf * K::STRIDE, tw, t, xf);
  const int u = col0 + xf;
  if (u < NC) {
    float2* dst = T + ((size_t)k * NC + u) * N;
    constexpr int LP = FftShape<N>::LAST_P;
#pragma unroll
    for (int m = 0; m < K::E / LP; ++m)
#pragma unroll
      for (int q = 0; q < LP; ++q) dst[fft_out_index<N>(t, m, q)] = v[m * LP + dft_perm<LP>(q)];
  }
}

// 5. statistics of each stored image: mean, population sigma, max with the
// lowest index; candidate iff peak / sigma >= threshold.  One block per
// image; FP32 sums over 32 pixels per step, FP64 per thread and block.
// With `clip` (the one-pass clipped noise) a second read of the image sums
// the deviations d = I - mean of the pixels with |d| <= kClipSigmas sigma,
// and mean and sigma become those of the kept pixels.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[3 * w] = a;
    sh[3 * w + 1] = b;
    sh[3 * w + 2] = c;
  }
  __syncthreads();
  a = b = c = 0.0;
  for (int i = 0; i < 8; ++i) {
    a += sh[3 * i];
    b += sh[3 * i + 1];
    c += sh[3 * i + 2];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_plain_stats(int npix, const float* __restrict__ images,
                                                     const int4* __restrict__ img_info,
                                                     const double* __restrict__ weight, int img_base,
                                                     double threshold, DevCand* __restrict__ cands,
                                                     int* __restrict__ ncand, int cand_cap,
                                                     DevStat* __restrict__ stats, int clip) {
  __shared__ double s_red[24];
  __shared__ float s_max[8];
  __shared__ int s_idx[8];
  const int k = blockIdx.x;
  const int img = img_base + k;
  const size_t n2 = (size_t)npix * npix;
  const float* im = images + (size_t)k * n2;
  double sum = 0.0, sq = 0.0, unused = 0.0;
  float mx = -FLT_MAX;
  int mi = INT_MAX;
  for (size_t base = 0; base < n2; base += 256 * 32) {
    float ps = 0.f, pq = 0.f;
    for (int j = 0; j < 32; ++j) {
      const size_t i = base + (size_t)j * 256 + threadIdx.x;
      if (i < n2) {
        const float v = im[i];
        ps += v;
        pq = fmaf(v, v, pq);
        if (v > mx || (v == mx && (int)i < mi)) {
          mx = v;
          mi = (int)i;
        }
      }
    }
    sum += ps;
    sq += pq;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float om = __shfl_xor_sync(0xffffffffu, mx, off);
    const int oi = __shfl_xor_sync(0xffffffffu, mi, off);
    if (om > mx || (om == mx && oi < mi)) {
      mx = om;
      mi = oi;
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_max[w] = mx;
    s_idx[w] = mi;
  }
  block_sum3(sum, sq, unused, s_red);
  mx = s_max[0];
  mi = s_idx[0];
  for (int i = 1; i < 8; ++i)
    if (s_max[i] > mx || (s_max[i] == mx && s_idx[i] < mi)) {
      mx = s_max[i];
      mi = s_idx[i];
    }
  double mean = sum / (double)n2;
  double var = sq / (double)n2 - mean * mean;
  var = var > 0.0 ? var : 0.0;
  if (clip) {
    const float mu = (float)mean;
    const float r = (float)(kClipSigmas * sqrt(var));
    double ks1 = 0.0, ks2 = 0.0, kn = 0.0;
    for (size_t base = 0; base < n2; base += 256 * 32) {
      float ps = 0.f, pq = 0.f;
      int pn = 0;
      for (int j = 0; j < 32; ++j) {
        const size_t i = base + (size_t)j * 256 + threadIdx.x;
        if (i < n2) {
          const float dv = im[i] - mu;
          if (fabsf(dv) <= r) {
            ps += dv;
            pq = fmaf(dv, dv, pq);
            ++pn;
          }
        }
      }
      ks1 += ps;
      ks2 += pq;
      kn += pn;
    }
    block_sum3(ks1, ks2, kn, s_red);
    const double nk = kn > 0.0 ? kn : 1.0;
    const double m1 = ks1 / nk;
    mean = (double)mu + m1;
    var = ks2 / nk - m1 * m1;
    var = var > 0.0 ? var : 0.0;
  }
  if (threadIdx.x != 0) return;
  const double W = weight[img];
  const int4 info = img_info[img];
  const double sigma = sqrt(var);
  const double peak = mx;
  const double snr = sigma > 0.0 ? peak / sigma : 0.0;
  DevStat ds;
  ds.pad = 0;
  ds.weight = W;
  ds.mean = mean;
  ds.peak = (float)peak;
  ds.sigma = (float)sigma;
  ds.snr = (float)snr;
  ds.y = mi / npix;
  ds.x = mi - ds.y * npix;
  if (!(W > 0.0)) {
    ds.peak = ds.sigma = ds.snr = 0.f;
    ds.x = ds.y = 0;
    ds.mean = 0.0;
  }
  if (stats) stats[img] = ds;
  if (W > 0.0 && sigma > 0.0 && snr >= threshold) {
    const int c = atomicAdd(ncand, 1);
    if (c < cand_cap) {
      DevCand dc;
      dc.d = info.x;
      dc.s = info.y;
      dc.t = info.z;
      dc.x = ds.x;
      dc.y = ds.y;
      dc.snr = (float)snr;
      dc.peak = (float)peak;
      dc.sigma = (float)sigma;
      cands[c] = dc;
    }
  }
}

template <int N>
cudaError_t run_plain_colfft(const float2* grid, float2* T, const float2* tw, int nk, cudaStream_t st) {
  using K = ImgCfg<N>;
  // set on every call: the attribute belongs to the current device's context
  const cudaError_t attr =
      cudaFuncSetAttribute(k_plain_colfft<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM_A_FIXED);
  if (attr != cudaSuccess) return attr;
  dim3 grid_dim((N / 2 + K::XA - 1) / K::XA, nk);
  k_plain_colfft<N><<<grid_dim, K::T * K::XA, K::SMEM_A_FIXED, st>>>(grid, T, tw);
  return cudaGetLastError();
}

// One launch set for images [img0, img0 + nk) = t' t0 .. t0+nk-1 of trial (d, s).
cudaError_t launch_plain_chunk(const SegmentGeom& g, const DevTables& tb, const PlainBuffers& pb, int d, int s,
                               int t0, int nk, int img0, const int4* img_info, const double* weight,
                               double threshold, DevCand* cands, int* ncand, int cand_cap, DevStat* stats,
                               cudaStream_t st, bool clip) {
  const size_t rows = (size_t)g.nbl * g.nchan;
  const int blocks = (int)std::min<size_t>((rows * nk + 255) / 256, (size_t)sm_count() * 32);
  k_plain_dedisperse<<<blocks, 256, 0, st>>>(g, tb, pb.S, d, s, t0, nk, pb.R);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int W = g.npix / 2 + 1;
  e = cudaMemsetAsync(pb.grid, 0, (size_t)nk * g.npix * W * sizeof(float2), st);
  if (e != cudaSuccess) return e;
  const int gblocks = (int)std::min<size_t>(((size_t)pb.nent * nk + 255) / 256, (size_t)sm_count() * 32);
  k_plain_grid<<<gblocks, 256, 0, st>>>(g, pb.ent, pb.nent, pb.R, nk, pb.grid);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (g.npix) {
#define RF_CASE(NN)                                                        \
  case NN:                                                                 \
    e = run_plain_colfft<NN>(pb.grid, pb.T, tb.twiddle, nk, st);           \
    break;
    RF_CASE(16) RF_CASE(32) RF_CASE(64) RF_CASE(128) RF_CASE(256) RF_CASE(512) RF_CASE(1024) RF_CASE(2048)
    RF_CASE(4096) RF_CASE(8192)
#undef RF_CASE
    default:
      e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  SegmentGeom gr = g;
  gr.ncol = g.npix / 2;
  gr.tsplit = 1;  // k_plain_colfft stores T in natural row order
  e = launch_rowfft_stats(gr, tb, pb.T, nk, img0, weight, pb.partials, pb.images, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  k_plain_stats<<<nk, 256, 0, st>>>(g.npix, pb.images, img_info, weight, img0, threshold, cands, ncand, cand_cap,
                                    stats, clip ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rf
