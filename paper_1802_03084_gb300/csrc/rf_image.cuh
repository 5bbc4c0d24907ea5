// rf_image.cuh -- imaging kernels of one (DM, dt, t') dirty image, Sec. 3.1:
// dedispersion + boxcar resampling + nearest-neighbour gridding + 2D inverse
// FFT + image statistics.
//
// The half-plane grid H[iv][iu] (iu = 0 .. iu_max) of an image is never
// materialised in global memory.  Pass A (k_grid_colfft) builds one column of
// H per transform directly in shared memory from the dedispersed, resampled
// visibilities and runs the length-N inverse FFT along v; the result
// T[iu][y] goes to a global (L2-resident) scratch.  Pass B (k_rowfft_stats)
// takes two image rows y, y+1 per transform: with Z[u] = T[u][y] + i T[u][y+1]
// on the Hermitian extension (Z[N-u] = conj T[u][y] + i conj T[u][y+1]),
// one complex inverse FFT gives row y in the real part and row y+1 in the
// imaginary part.  Pixel statistics (sum, sum of squares, max with lowest
// index) are reduced in the same kernel; the image itself is written only
// when a caller asks for it.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>

#include "rf_engine.h"
#include "rf_fft.cuh"

namespace rf {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Compile-time launch shape per image side N.
template <int N>
struct ImgCfg {
  static constexpr int T = N / 16;                               // threads per transform
  static constexpr int B = cmin(8, 512 / T);                     // images per group (pass A)
  static constexpr int C = cmax(1, cmin(8, 512 / (T * B)));      // columns per CTA (pass A)
  static constexpr int XA = B * C;                               // transforms per CTA (pass A)
  static constexpr int THREADS_A = T * XA;
  static constexpr int NW = THREADS_A / 32;                      // warps per CTA (pass A)
  static constexpr int WPC = cmax(1, NW / C);                    // warps per column (pass A)
  static constexpr int XB = cmin(512 / T, N / 2);                // row pairs per CTA (pass B)
  static constexpr int THREADS_B = T * XB;
  static constexpr int RB = 2 * XB;                              // rows per CTA (pass B)
  static constexpr int STRIDE = fft_stride<N>();
  static constexpr int SMEM_A = XA * STRIDE * 8;
  static constexpr int SMEM_B = XB * STRIDE * 8;
};

template <bool FP16>
__device__ __forceinline__ float2 load_sample(const void* __restrict__ S, size_t i);

template <>
__device__ __forceinline__ float2 load_sample<false>(const void* __restrict__ S, size_t i) {
  return __ldg(reinterpret_cast<const float2*>(S) + i);
}

template <>
__device__ __forceinline__ float2 load_sample<true>(const void* __restrict__ S, size_t i) {
  const __half2 h = __ldg(reinterpret_cast<const __half2*>(S) + i);
  return __half22float2(h);
}

// Pass A: for a group of B consecutive output integrations t0 .. t0+B-1 of
// trial (d, s) and C adjacent half-plane columns, build each column of the
// checkerboarded half-plane grid in shared memory and inverse-FFT it along v.
//   R[b,c](t') = sum_{j < dt} S[b,c][t' dt + j + delta[d][c]]    (dedisperse+resample)
//   H[iv][iu] += (-1)^(iu+iv) R   or   conj(R) for folded entries (gridding)
// Gridding: the entries of a column are sorted by cell and split (on the
// host) into WPC cell-aligned ranges, one per warp.  A warp takes 32 entries
// at a time, one per lane; each lane sums its B x dt samples, a segmented
// shuffle scan keyed on the cell row adds up the lanes of each cell, and the
// last lane of each cell adds the total into shared memory.  A cell belongs
// to one warp and its partial sums are added in a fixed order, so the grid
// is deterministic without atomics.
template <int N, bool FP16>
__global__ void __launch_bounds__(ImgCfg<N>::THREADS_A)
    k_grid_colfft(SegmentGeom g, DevTables tb, const void* __restrict__ S, const Group* __restrict__ groups,
                  int g_begin, int img_base, float2* __restrict__ Tbuf) {
  using K = ImgCfg<N>;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const Group gr = groups[g_begin + blockIdx.x];
  const int col0 = blockIdx.y * K::C;

  for (int i = tid; i < K::XA * K::STRIDE; i += K::THREADS_A) sm[i] = make_float2(0.f, 0.f);
  __syncthreads();

  const int dt = tb.dt_list[gr.s];
  const int* __restrict__ dl = tb.delays + (size_t)gr.d * g.nchan;
  const int tstart = gr.t0 * dt;
  for (int unit = warp; unit < K::C * K::WPC; unit += K::NW) {
    const int cl = unit / K::WPC;
    const int col = col0 + cl;
    if (col >= g.ncol) continue;  // warp-uniform
    const int* cwp = tb.col_warp_ptr + (size_t)col * (K::WPC + 1) + (unit - cl * K::WPC);
    const int ebeg = cwp[0];
    const int eend = cwp[1];
    float2* colbuf = sm + (size_t)cl * K::B * K::STRIDE;
    for (int base = ebeg; base < eend; base += 32) {
      const int e = base + lane;
      const bool valid = e < eend;
      float2 val[K::B];
#pragma unroll
      for (int k = 0; k < K::B; ++k) val[k] = make_float2(0.f, 0.f);
      int row = -1 - lane;  // distinct sentinel for lanes past the range
      if (valid) {
        const GridEntry en = tb.ent[e];
        row = en.row;
        const int c = en.cflags >> 2;
        const int tf = tstart + __ldg(dl + c);
        const size_t rowoff = (size_t)en.bc * g.nint_pad;
        const float sy = (en.cflags & ENT_CONJ) ? -1.f : 1.f;
        const float sg = (en.cflags & ENT_NEG) ? -1.f : 1.f;
#pragma unroll
        for (int k = 0; k < K::B; ++k) {
          if (k < gr.nimg) {
            float2 a = make_float2(0.f, 0.f);
            const int tk = tf + k * dt;
            for (int j = 0; j < dt; ++j) {
              const int ti = tk + j;
              if (ti < g.nint) a = cadd(a, load_sample<FP16>(S, rowoff + ti));
            }
            val[k] = make_float2(sg * a.x, sg * sy * a.y);
          }
        }
      }
      // inclusive segmented scan over lanes with equal row (rows are sorted)
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int rup = __shfl_up_sync(0xffffffffu, row, off);
        const bool take = lane >= off && rup == row;
#pragma unroll
        for (int k = 0; k < K::B; ++k) {
          const float vx = __shfl_up_sync(0xffffffffu, val[k].x, off);
          const float vy = __shfl_up_sync(0xffffffffu, val[k].y, off);
          if (take) {
            val[k].x += vx;
            val[k].y += vy;
          }
        }
      }
      const int rdown = __shfl_down_sync(0xffffffffu, row, 1);
      const bool tail = valid && (lane == 31 || e + 1 >= eend || rdown != row);
      if (tail) {
        float2* cp = colbuf + pad16(row);
#pragma unroll
        for (int k = 0; k < K::B; ++k) cp[k * K::STRIDE] = cadd(cp[k * K::STRIDE], val[k]);
      }
      __syncwarp();
    }
  }
  __syncthreads();

  const int xf = tid / K::T;
  const int t = tid - xf * K::T;
  float2 v[16];
  fft_inverse_to_regs<N>(v, sm + xf * K::STRIDE, tb.twiddle, t);
  const int col = col0 + xf / K::B;
  const int k = xf % K::B;
  if (col < g.ncol && k < gr.nimg) {
    const size_t slot = (size_t)(gr.img0 + k - img_base);
    float2* dst = Tbuf + (slot * g.ncol + col) * N;
    constexpr int LP = FftShape<N>::LAST_P;
#pragma unroll
    for (int m = 0; m < 16 / LP; ++m)
#pragma unroll
      for (int q = 0; q < LP; ++q) dst[fft_out_index<N>(t, m, q)] = v[m * LP + dft_perm<LP>(q)];
  }
}

__device__ __forceinline__ void max_merge(float& m, int& i, float m2, int i2) {
  if (m2 > m || (m2 == m && i2 < i)) {
    m = m2;
    i = i2;
  }
}

// Pass B: rows y0 .. y0 + RB - 1 of one image (slot = blockIdx.y); pairs of
// rows share one complex inverse FFT.  Writes one StatPartial per CTA.
template <int N>
__global__ void __launch_bounds__(ImgCfg<N>::THREADS_B)
    k_rowfft_stats(SegmentGeom g, DevTables tb, const float2* __restrict__ Tbuf, int img_base,
                   const double* __restrict__ weight, StatPartial* __restrict__ partials,
                   float* __restrict__ images) {
  using K = ImgCfg<N>;
  extern __shared__ float2 sm[];
  __shared__ double w_sum[32], w_sq[32];
  __shared__ float w_max[32];
  __shared__ int w_idx[32];
  const int tid = threadIdx.x;
  const int rb = blockIdx.x;
  const int slot = blockIdx.y;
  const int y0 = rb * K::RB;
  const int ncol = g.ncol;
  const float2* __restrict__ Ts = Tbuf + (size_t)slot * ncol * N;

  for (int i = tid; i < ncol * K::XB; i += K::THREADS_B) {
    const int p = i % K::XB;
    const int u = i / K::XB;
    const float4 ab = __ldg(reinterpret_cast<const float4*>(Ts + (size_t)u * N + y0 + 2 * p));
    float2* z = sm + p * K::STRIDE;
    if (u == 0) {
      z[0] = make_float2(ab.x, ab.z);
    } else {
      z[pad16(u)] = make_float2(ab.x - ab.w, ab.y + ab.z);       // a + i b
      z[pad16(N - u)] = make_float2(ab.x + ab.w, ab.z - ab.y);   // conj(a) + i conj(b)
    }
  }
  const int nz = N - 2 * ncol + 1;  // u = ncol .. N - ncol are empty
  for (int i = tid; i < nz * K::XB; i += K::THREADS_B) {
    const int p = i / nz;
    const int u = ncol + (i - p * nz);
    sm[p * K::STRIDE + pad16(u)] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  const int xf = tid / K::T;
  const int t = tid - xf * K::T;
  float2 v[16];
  fft_inverse_to_regs<N>(v, sm + xf * K::STRIDE, tb.twiddle, t);

  const int y = y0 + 2 * xf;
  float lmax = -FLT_MAX;
  int lidx = INT_MAX;
  float lsum = 0.f, lsq = 0.f;
  constexpr int LP = FftShape<N>::LAST_P;
  float scale = 0.f;
  if (images != nullptr) {
    const double W = weight[img_base + slot];
    scale = W > 0.0 ? (float)(0.5 / W) : 0.f;
  }
#pragma unroll
  for (int m = 0; m < 16 / LP; ++m) {
#pragma unroll
    for (int q = 0; q < LP; ++q) {
      const int o = fft_out_index<N>(t, m, q);
      const float2 z = v[m * LP + dft_perm<LP>(q)];
      max_merge(lmax, lidx, z.x, y * N + o);
      max_merge(lmax, lidx, z.y, (y + 1) * N + o);
      lsum += z.x + z.y;
      lsq = fmaf(z.x, z.x, lsq);
      lsq = fmaf(z.y, z.y, lsq);
      if (images != nullptr) {
        float* im = images + ((size_t)slot * N + y) * N;
        im[o] = z.x * scale;
        im[N + o] = z.y * scale;
      }
    }
  }
  // warp reduction (FP32 pairwise), then FP64 across warps; blocks smaller
  // than a warp (N = 16) reduce over their own lanes only.
  constexpr int WL = K::THREADS_B < 32 ? K::THREADS_B : 32;
  constexpr unsigned MASK = WL == 32 ? 0xffffffffu : ((1u << WL) - 1u);
#pragma unroll
  for (int off = WL / 2; off > 0; off >>= 1) {
    lsum += __shfl_xor_sync(MASK, lsum, off);
    lsq += __shfl_xor_sync(MASK, lsq, off);
    const float om = __shfl_xor_sync(MASK, lmax, off);
    const int oi = __shfl_xor_sync(MASK, lidx, off);
    max_merge(lmax, lidx, om, oi);
  }
  const int lane = tid & 31;
  const int wid = tid >> 5;
  if (lane == 0) {
    w_sum[wid] = (double)lsum;
    w_sq[wid] = (double)lsq;
    w_max[wid] = lmax;
    w_idx[wid] = lidx;
  }
  __syncthreads();
  if (tid == 0) {
    constexpr int NW = (K::THREADS_B + 31) / 32;
    double s = 0.0, q2 = 0.0;
    float mx = -FLT_MAX;
    int mi = INT_MAX;
    for (int w = 0; w < NW; ++w) {
      s += w_sum[w];
      q2 += w_sq[w];
      max_merge(mx, mi, w_max[w], w_idx[w]);
    }
    StatPartial sp;
    sp.sum = s;
    sp.sumsq = q2;
    sp.max = mx;
    sp.idx = mi;
    sp.pad[0] = sp.pad[1] = 0;
    partials[(size_t)slot * (N / K::RB) + rb] = sp;
  }
}

template <int N, bool FP16>
cudaError_t run_grid_colfft(const SegmentGeom& g, const DevTables& tb, const void* S, const Group* groups,
                            int g_begin, int ngroups, int img_base, float2* Tbuf, cudaStream_t st) {
  using K = ImgCfg<N>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_grid_colfft<N, FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM_A);
  if (attr != cudaSuccess) return attr;
  if (ngroups <= 0) return cudaSuccess;
  dim3 grid(ngroups, (g.ncol + K::C - 1) / K::C);
  k_grid_colfft<N, FP16><<<grid, K::THREADS_A, K::SMEM_A, st>>>(g, tb, S, groups, g_begin, img_base, Tbuf);
  return cudaGetLastError();
}

template <int N>
cudaError_t run_rowfft_stats(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, int nimg,
                             int img_base, const double* weight, StatPartial* partials, float* images,
                             cudaStream_t st) {
  using K = ImgCfg<N>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_rowfft_stats<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM_B);
  if (attr != cudaSuccess) return attr;
  if (nimg <= 0) return cudaSuccess;
  dim3 grid(N / K::RB, nimg);
  k_rowfft_stats<N><<<grid, K::THREADS_B, K::SMEM_B, st>>>(g, tb, Tbuf, img_base, weight, partials, images);
  return cudaGetLastError();
}

template <int N>
void fill_shape(ImageKernelShape* o) {
  using K = ImgCfg<N>;
  o->images_per_group = K::B;
  o->cols_per_cta = K::C;
  o->threads_a = K::THREADS_A;
  o->smem_a = K::SMEM_A;
  o->warps_per_col = K::WPC;
  o->rows_per_cta = K::RB;
  o->threads_b = K::THREADS_B;
  o->smem_b = K::SMEM_B;
}

#define RF_INSTANTIATE_IMAGE(N)                                                                              \
  template cudaError_t run_grid_colfft<N, false>(const SegmentGeom&, const DevTables&, const void*,          \
                                                 const Group*, int, int, int, float2*, cudaStream_t);       \
  template cudaError_t run_grid_colfft<N, true>(const SegmentGeom&, const DevTables&, const void*,           \
                                                const Group*, int, int, int, float2*, cudaStream_t);        \
  template cudaError_t run_rowfft_stats<N>(const SegmentGeom&, const DevTables&, const float2*, int, int,    \
                                           const double*, StatPartial*, float*, cudaStream_t);              \
  template void fill_shape<N>(ImageKernelShape*);

}  // namespace rf
