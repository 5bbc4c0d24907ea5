// rf_periodic.cu -- periodicity search (Sec. 3.1 footnote: a time segment is
// Fourier transformed and each fluctuation frequency imaged; Fig. 2: a change
// of the innermost loop of the search).
//
// For DM trial d and each (baseline, channel) row of the Stokes-I buffer, the
// dedispersed window x[t] = S[row][delta[d][c] + t], t < L, is transformed
// over time with the shared-memory FFT core (length L, a power of two).  With
// Y the inverse DFT (sign +) of x, the cosine and sine sums at fluctuation
// frequency k are
//   U_k = (1/L) sum_t x[t] cos(2 pi k t / L) = (Y[k] + Y[L-k]) / (2L),
//   Q_k = (1/L) sum_t x[t] sin(2 pi k t / L) = -i (Y[k] - Y[L-k]) / (2L).
// They are written as two series of "visibilities" per (DM, k) so that the
// search's gridding and column-FFT kernels image them unchanged; the power row
// pass then pairs the two images of each (DM, k).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "rf_engine.h"
#include "rf_fft.cuh"

namespace rf {

namespace {

template <bool FP16>
__device__ __forceinline__ float2 load_stokes(const void* S, size_t i) {
  if (FP16) return __half22float2(reinterpret_cast<const __half2*>(S)[i]);
  return reinterpret_cast<const float2*>(S)[i];
}

// One transform of T = L/E threads per (DM trial of the batch, row); 256/T
// transforms per block.  out[(2 j + q) nrows + row][kk] (pitch kpad) holds
// U (q = 0) and Q (q = 1) of batch trial j at k = kmin + kk.
template <bool FP16, int L>
__global__ void __launch_bounds__(256) k_period_dft(SegmentGeom g, const void* __restrict__ S,
                                                    const int* __restrict__ delays, const int* __restrict__ dms,
                                                    int nb, const float2* __restrict__ twl, int kmin, int K,
                                                    int kpad, float2* __restrict__ out) {
  using FS = FftShape<L>;
  constexpr int T = FS::T;
  constexpr int E = FS::E;
  constexpr int XT = 256 / T;
  constexpr int P0 = FS::NPASS == 1 ? FS::LAST_P : E;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int xf = threadIdx.x / T;
  const int t = threadIdx.x - xf * T;
  float2* buf = reinterpret_cast<float2*>(smraw) + xf * FS::STRIDE;
  const int nrows = g.nbl * g.nchan;
  // transforms past the end run on zeros and write nothing: several short
  // transforms share a warp and its __syncwarp barriers
  const long tr = (long)blockIdx.x * XT + xf;
  const bool valid = tr < (long)nb * nrows;
  const int j = valid ? (int)(tr / nrows) : 0;
  const int row = valid ? (int)(tr - (long)j * nrows) : 0;
  const int c = row / g.nbl;
  const int del = valid ? delays[(size_t)dms[j] * g.nchan + c] : 0;
  const size_t base = (size_t)row * g.nint_pad + del;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E / P0; ++m)
#pragma unroll
    for (int r = 0; r < P0; ++r)
      v[m * P0 + r] = valid ? load_stokes<FP16>(S, base + t + m * T + r * (L / P0)) : make_float2(0.f, 0.f);
  fft_inverse_from_regs<L>(v, buf, twl, t, xf);
  fft_sync<T>(xf);  // every thread's last-pass loads are done
  constexpr int LP = FS::LAST_P;
#pragma unroll
  for (int m = 0; m < E / LP; ++m)
#pragma unroll
    for (int q = 0; q < LP; ++q) buf[padx(fft_out_index<L>(t, m, q))] = v[m * LP + dft_perm<LP>(q)];
  fft_sync<T>(xf);
  if (!valid) return;  // no barrier follows
  const float h = 0.5f / (float)L;
  float2* ou = out + ((size_t)(2 * j) * nrows + row) * kpad;
  float2* oq = out + ((size_t)(2 * j + 1) * nrows + row) * kpad;
  for (int kk = t; kk < K; kk += T) {
    const int k = kmin + kk;
    const float2 a = buf[padx(k)];
    const float2 b = buf[padx(L - k)];
    ou[kk] = make_float2((a.x + b.x) * h, (a.y + b.y) * h);
    oq[kk] = make_float2((a.y - b.y) * h, (b.x - a.x) * h);
  }
}

template <bool FP16, int L>
cudaError_t run_period_dft(const SegmentGeom& g, const void* S, const int* delays, const int* dms, int nb,
                           const float2* twl, int kmin, int K, int kpad, float2* out, cudaStream_t st) {
  using FS = FftShape<L>;
  constexpr int XT = 256 / FS::T;
  const int smem = XT * FS::STRIDE * 8;
  cudaError_t e = cudaFuncSetAttribute(k_period_dft<FP16, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long ntr = (long)nb * g.nbl * g.nchan;
  if (ntr <= 0) return cudaSuccess;
  const long blocks = (ntr + XT - 1) / XT;
  if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
  k_period_dft<FP16, L><<<(unsigned)blocks, XT * FS::T, smem, st>>>(g, S, delays, dms, nb, twl, kmin, K, kpad, out);
  return cudaGetLastError();
}

__device__ __forceinline__ void pmax_merge(float& m, int& i, float m2, int i2) {
  if (m2 > m || (m2 == m && i2 < i)) {
    m = m2;
    i = i2;
  }
}

// One warp per pair: the power maximum over the N row partials (lowest
// index on ties), the two images' variances from their Parseval sums (FP64),
// amplitude = sqrt(max P) / (2W), sigma = sqrt((var_U + var_Q) / 2),
// snr = amplitude / sigma; a candidate iff snr >= threshold.
__global__ void k_finalize_power(int npix, int ncol, const StatPartial* __restrict__ partials,
                                 const float* __restrict__ colsq, const float* __restrict__ mean0,
                                 const int4* __restrict__ pairs, int npairs, int pair_base, double W,
                                 double threshold, DevPeriodic* __restrict__ stats, DevPeriodic* __restrict__ cands,
                                 int* __restrict__ ncand, int cand_cap) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= npairs) return;
  const int4 pr = pairs[j];
  const StatPartial* pp = partials + (size_t)j * npix;
  float mx = -1.f;
  int mi = INT_MAX;
  for (int r = lane; r < npix; r += 32) pmax_merge(mx, mi, pp[r].max, pp[r].idx);
  double su = 0.0, sq = 0.0;
  for (int c = lane; c < ncol; c += 32) {
    su += (double)colsq[(size_t)pr.x * ncol + c];
    sq += (double)colsq[(size_t)pr.y * ncol + c];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    su += __shfl_xor_sync(0xffffffffu, su, off);
    sq += __shfl_xor_sync(0xffffffffu, sq, off);
    const float om = __shfl_xor_sync(0xffffffffu, mx, off);
    const int oi = __shfl_xor_sync(0xffffffffu, mi, off);
    pmax_merge(mx, mi, om, oi);
  }
  if (lane != 0) return;
  DevPeriodic o;
  o.d = pr.z;
  o.k = pr.w;
  o.x = 0;
  o.y = 0;
  o.amplitude = 0.f;
  o.sigma = 0.f;
  o.snr = 0.f;
  o.pad = 0;
  if (W > 0.0) {
    const double inv = 0.5 / W;
    const double mu = (double)mean0[pr.x] * inv, mq = (double)mean0[pr.y] * inv;
    double vu = su * inv * inv - mu * mu;
    double vq = sq * inv * inv - mq * mq;
    vu = vu > 0.0 ? vu : 0.0;
    vq = vq > 0.0 ? vq : 0.0;
    const double sigma = sqrt(0.5 * (vu + vq));
    const double amp = sqrt((double)mx) * inv;
    o.amplitude = (float)amp;
    o.sigma = (float)sigma;
    o.snr = sigma > 0.0 ? (float)(amp / sigma) : 0.f;
    o.y = mi / npix;
    o.x = mi - o.y * npix;
    if (sigma > 0.0 && amp / sigma >= threshold) {
      const int k = atomicAdd(ncand, 1);
      if (k < cand_cap) cands[k] = o;
    }
  }
  stats[pair_base + j] = o;
}

}  // namespace

cudaError_t launch_period_dft(const SegmentGeom& g, const void* S, const int* delays, const int* dms, int nb,
                              int L, const float2* twl, int kmin, int K, int kpad, float2* out, cudaStream_t st) {
  switch (L) {
#define RF_CASE(LL)                                                                                 \
  case LL:                                                                                          \
    return g.fp16 ? run_period_dft<true, LL>(g, S, delays, dms, nb, twl, kmin, K, kpad, out, st)   \
                  : run_period_dft<false, LL>(g, S, delays, dms, nb, twl, kmin, K, kpad, out, st);
    RF_CASE(16) RF_CASE(32) RF_CASE(64) RF_CASE(128) RF_CASE(256) RF_CASE(512) RF_CASE(1024) RF_CASE(2048)
    RF_CASE(4096) RF_CASE(8192)
#undef RF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_finalize_power(const SegmentGeom& g, const StatPartial* partials, const float* colsq,
                                  const float* mean0, const int4* pairs, int npairs, int pair_base, double W,
                                  double threshold, DevPeriodic* stats, DevPeriodic* cands, int* ncand, int cand_cap,
                                  cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  k_finalize_power<<<(npairs + 7) / 8, 256, 0, st>>>(g.npix, g.ncol, partials, colsq, mean0, pairs, npairs, pair_base,
                                                     W, threshold, stats, cands, ncand, cand_cap);
  return cudaGetLastError();
}

}  // namespace rf
