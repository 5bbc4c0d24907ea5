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

#include <algorithm>

#include "rf_engine.h"
#include "rf_fft.cuh"

namespace rf {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Compile-time launch shape per image side N.
template <int N>
struct ImgCfg {
  static constexpr int T = FftShape<N>::T;                       // threads per transform
  static constexpr int E = FftShape<N>::E;                       // values per thread
  // pass A: 256 threads, one column; a group is up to 32 consecutive t'
  // (one lane each while gridding); column FFTs in rounds of XA transforms
  static constexpr int THREADS_A = 256;
  static constexpr int NW = THREADS_A / 32;
  static constexpr int WPC = NW;                                 // warps gridding a column
  static constexpr int B = 32;                                   // images per group
  static constexpr int XA = cmin(THREADS_A / T, B);              // transforms per round
  static constexpr int CELL_PITCH = 33;                          // cell values per cell row (32 + pad)
  static constexpr int SMEM_A_FIXED = XA * fft_stride<N>() * 8;
  // pass B: XB row pairs (RB rows) per work item; the column-FFT tile of the
  // next item is prefetched while the current one is transformed
  static constexpr int XB = cmin(256 / T, N / 2);
  static constexpr int THREADS_B = T * XB;
  static constexpr int RB = 2 * XB;
  static constexpr int CH = XB;                                  // 16-byte chunks per tile row
  static constexpr int STRIDE = fft_stride<N>();
  static constexpr int SMEM_B_FIXED = XB * STRIDE * 8;
  static_assert(T <= 32 || (XA <= 15 && XB <= 15), "named barriers: at most 15 wide transforms per block");
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// Pass A: for a group of up to B = 32 consecutive output integrations
// t0 .. t0+31 of trial (d, s) and one half-plane column u, build the column
// of the checkerboarded half-plane grid and inverse-FFT it along v.
//   R[b,c](t') = sum_{j < dt} S[b,c][t' dt + j + delta[d][c]]    (dedisperse+resample)
//   H[iv][u] += (-1)^(u+iv) R   or   conj(R) for folded entries  (gridding)
// Gridding: lane k of every warp is image t0 + k, so one load instruction
// reads 32 consecutive time samples of one (b, c).  The column's entries are
// sorted by cell and split on the host into 8 cell-aligned ranges, one per
// warp; a warp walks its range entry by entry (metadata broadcast by
// shuffle, samples of 8 entries in flight), summing each cell in a register
// in a fixed order, and stores the cell's 32 values in a compact shared
// array.  Column FFTs: each transform zeroes its buffer, scatters one
// image's cells and runs the FFT; transforms synchronise only among their
// own threads.
template <int N, bool FP16>
__global__ void __launch_bounds__(ImgCfg<N>::THREADS_A)
    k_grid_colfft(SegmentGeom g, DevTables tb, const void* __restrict__ S, const Group* __restrict__ groups,
                  int g_begin, int img_base, float2* __restrict__ Tbuf) {
  using K = ImgCfg<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* fbuf = reinterpret_cast<float2*>(smraw);                              // [XA][STRIDE]
  float2* cellval = fbuf + K::XA * K::STRIDE;                                    // [max_cells][33]
  int* crow = reinterpret_cast<int*>(cellval + (size_t)g.max_cells * K::CELL_PITCH);  // [max_cells]
  int* sdel = crow + g.max_cells;                                                // [nchan]
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const Group gr = groups[g_begin + blockIdx.x];
  const int col = blockIdx.y;
  const int cell0 = tb.col_cell_ptr[col];
  const int ncells = tb.col_cell_ptr[col + 1] - cell0;
  for (int c = tid; c < ncells; c += K::THREADS_A) crow[c] = tb.cell_row[cell0 + c];
  {
    const int* __restrict__ dl = tb.delays + (size_t)gr.d * g.nchan;
    for (int c = tid; c < g.nchan; c += K::THREADS_A) sdel[c] = dl[c];
  }
  const int* cwp = tb.col_warp_ptr + (size_t)col * (K::WPC + 1) + warp;
  const int ebeg = cwp[0];
  const int eend = cwp[1];
  GridEntry nxt = {0, 0, 0, -1};
  if (ebeg + lane < eend) nxt = tb.ent[ebeg + lane];
  __syncthreads();

  // ---- gridding (lanes = images).  Image t' = t0 + lane reads sample
  // t' dt + delta of the dt-resampled series: phase delta mod dt, index
  // t' + delta div dt.
  {
    const int dt = tb.dt_list[gr.s];
    const int lp = tb.sdt_lp[gr.s];
    const unsigned char* __restrict__ Sd = reinterpret_cast<const unsigned char*>(tb.sdt_ptr[gr.s]);
    const size_t rowpitch = (size_t)dt * lp;
    const bool active = lane < gr.nimg;
    const int tq = gr.t0 + lane;
    const int lim = g.nint - tq * dt;  // the image has a sample iff delta < lim
    float2 acc = make_float2(0.f, 0.f);
    int cur = -1;
    for (int base = ebeg; base < eend; base += 32) {
      const GridEntry my = nxt;
      const bool mine = base + lane < eend;
      if (base + 32 + lane < eend) nxt = tb.ent[base + 32 + lane];
      const int mydel = mine ? sdel[my.cflags >> 2] : 0;
      const int mypart = (mydel % dt) * lp + mydel / dt;  // phase offset + index shift
      const int n = min(32, eend - base);
      for (int i0 = 0; i0 < n; i0 += 16) {
        float2 a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = (i0 + q) & 31;
          const int bc = __shfl_sync(0xffffffffu, my.bc, i);
          const int del = __shfl_sync(0xffffffffu, mydel, i);
          const int part = __shfl_sync(0xffffffffu, mypart, i);
          a[q] = make_float2(0.f, 0.f);
          if (active && i0 + q < n && del < lim) a[q] = load_sample<FP16>(Sd, (size_t)bc * rowpitch + part + tq);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = (i0 + q) & 31;
          const int cf = __shfl_sync(0xffffffffu, my.cflags, i);
          const int cell = __shfl_sync(0xffffffffu, my.cell, i);
          if (i0 + q < n) {
            if (cell != cur) {
              if (cur >= 0) cellval[cur * K::CELL_PITCH + lane] = acc;
              acc = make_float2(0.f, 0.f);
              cur = cell;
            }
            const float sy = (cf & ENT_CONJ) ? -1.f : 1.f;
            const float sg = (cf & ENT_NEG) ? -1.f : 1.f;
            acc.x += sg * a[q].x;
            acc.y += sg * sy * a[q].y;
          }
        }
      }
    }
    if (cur >= 0) cellval[cur * K::CELL_PITCH + lane] = acc;
  }
  __syncthreads();

  // ---- column FFTs, XA images per round
  const int xf = tid / K::T;
  const int t = tid - xf * K::T;
  if (xf < K::XA) {
    float2* buf = fbuf + xf * K::STRIDE;
    const int nrounds = (gr.nimg + K::XA - 1) / K::XA;
    for (int rd = 0; rd < nrounds; ++rd) {
      const int k = rd * K::XA + xf;
      for (int i = t; i < K::STRIDE; i += K::T) buf[i] = make_float2(0.f, 0.f);
      fft_sync<K::T>(xf);
      if (k < gr.nimg)
        for (int c = t; c < ncells; c += K::T) buf[padx(crow[c])] = cellval[c * K::CELL_PITCH + k];
      fft_sync<K::T>(xf);
      float2 v[K::E];
      fft_inverse_to_regs<N>(v, buf, tb.twiddle, t, xf);
      if (k < gr.nimg) {
        const size_t slot = (size_t)(gr.img0 + k - img_base);
        float2* dst = Tbuf + (slot * g.ncol + col) * N;
        constexpr int LP = FftShape<N>::LAST_P;
#pragma unroll
        for (int m = 0; m < K::E / LP; ++m)
#pragma unroll
          for (int q = 0; q < LP; ++q) dst[fft_out_index<N>(t, m, q)] = v[m * LP + dft_perm<LP>(q)];
      }
      fft_sync<K::T>(xf);
    }
  }
}

__device__ __forceinline__ void max_merge(float& m, int& i, float m2, int i2) {
  if (m2 > m || (m2 == m && i2 < i)) {
    m = m2;
    i = i2;
  }
}

// Pass B: work item = (image slot, block of RB rows); each pair of rows
// shares one complex inverse FFT.  Blocks loop over items; the column-FFT
// tile T[slot][u][y0 .. y0+RB) of the next item is copied to shared memory
// with cp.async (16-byte chunks, XOR-swizzled per row so the strided reads
// are free of bank conflicts) while the current item is transformed.  Each
// item writes one StatPartial: pixel sum and sum of squares over its RB rows
// (FP32: per thread, pairwise within warps, then across the block's warps;
// the items of an image are added in FP64 by the finalisation) and the max
// pixel with its lowest index.
template <int N>
__global__ void __launch_bounds__(ImgCfg<N>::THREADS_B, 2)
    k_rowfft_stats(SegmentGeom g, DevTables tb, const float2* __restrict__ Tbuf, int nimg, int img_base,
                   const double* __restrict__ weight, StatPartial* __restrict__ partials,
                   float* __restrict__ images) {
  using K = ImgCfg<N>;
  constexpr int NWB = (K::THREADS_B + 31) / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* fbuf = reinterpret_cast<float2*>(smraw);                  // [XB][STRIDE]
  float4* tile = reinterpret_cast<float4*>(fbuf + K::XB * K::STRIDE);  // [ncol][CH]
  __shared__ float w_sum[32], w_sq[32];
  __shared__ float w_max[32];
  __shared__ int s_idx;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int wid = tid >> 5;
  const int ncol = g.ncol;
  constexpr int nrb = N / K::RB;
  const int nitems = nimg * nrb;
  const int xf = tid / K::T;
  const int t = tid - xf * K::T;

  int item = blockIdx.x;
  if (item < nitems) {
    const int slot = item / nrb;
    const float2* src = Tbuf + (size_t)slot * ncol * N + (item - slot * nrb) * K::RB;
    for (int i = tid; i < ncol * K::CH; i += K::THREADS_B) {
      const int u = i / K::CH;
      const int c = i - u * K::CH;
      cp_async16(tile + u * K::CH + (c ^ (u & (K::CH - 1))), src + (size_t)u * N + 2 * c);
    }
    cp_async_commit();
  }
  for (; item < nitems; item += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    const int slot = item / nrb;
    const int y0 = (item - slot * nrb) * K::RB;
    // first-pass inputs Z[u], u = t + r T: a + i b for 0 < u < ncol, the
    // Hermitian mirror conj(a) + i conj(b) for N - u < ncol, real parts at
    // u = 0, zero elsewhere (columns beyond iu_max are empty)
    float2 v[K::E];
#pragma unroll
    for (int r = 0; r < K::E; ++r) {
      const int u = t + r * K::T;
      float2 z = make_float2(0.f, 0.f);
      if (u < ncol) {
        const float4 ab = tile[u * K::CH + (xf ^ (u & (K::CH - 1)))];
        z = (u == 0) ? make_float2(ab.x, ab.z) : make_float2(ab.x - ab.w, ab.y + ab.z);
      } else if (N - u < ncol) {
        const int uu = N - u;
        const float4 ab = tile[uu * K::CH + (xf ^ (uu & (K::CH - 1)))];
        z = make_float2(ab.x + ab.w, ab.z - ab.y);
      }
      v[r] = z;
    }
    __syncthreads();  // tile consumed: prefetch the next item
    const int next = item + gridDim.x;
    if (next < nitems) {
      const int ns = next / nrb;
      const float2* src = Tbuf + (size_t)ns * ncol * N + (next - ns * nrb) * K::RB;
      for (int i = tid; i < ncol * K::CH; i += K::THREADS_B) {
        const int u = i / K::CH;
        const int c = i - u * K::CH;
        cp_async16(tile + u * K::CH + (c ^ (u & (K::CH - 1))), src + (size_t)u * N + 2 * c);
      }
      cp_async_commit();
    }
    fft_inverse_from_regs<N>(v, fbuf + xf * K::STRIDE, tb.twiddle, t, xf);

    const int y = y0 + 2 * xf;
    float lmax = -FLT_MAX;
    float lsum = 0.f, lsq = 0.f;
    constexpr int LP = FftShape<N>::LAST_P;
    float scale = 0.f;
    if (images != nullptr) {
      const double W = weight[img_base + slot];
      scale = W > 0.0 ? (float)(0.5 / W) : 0.f;
    }
#pragma unroll
    for (int m = 0; m < K::E / LP; ++m) {
#pragma unroll
      for (int q = 0; q < LP; ++q) {
        const float2 z = v[m * LP + dft_perm<LP>(q)];
        lmax = fmaxf(lmax, fmaxf(z.x, z.y));
        lsum += z.x + z.y;
        lsq = fmaf(z.x, z.x, lsq);
        lsq = fmaf(z.y, z.y, lsq);
        if (images != nullptr) {
          const int o = fft_out_index<N>(t, m, q);
          float* im = images + ((size_t)slot * N + y) * N;
          im[o] = z.x * scale;
          im[N + o] = z.y * scale;
        }
      }
    }
    // FP32 warp sums and max, FP64 across warps; the index of the block
    // maximum is searched only by the threads that hold it.
    constexpr int WL = K::THREADS_B < 32 ? K::THREADS_B : 32;
    constexpr unsigned MASK = WL == 32 ? 0xffffffffu : ((1u << WL) - 1u);
    float wmax = lmax;
#pragma unroll
    for (int off = WL / 2; off > 0; off >>= 1) {
      lsum += __shfl_xor_sync(MASK, lsum, off);
      lsq += __shfl_xor_sync(MASK, lsq, off);
      wmax = fmaxf(wmax, __shfl_xor_sync(MASK, wmax, off));
    }
    if (lane == 0) {
      w_sum[wid] = lsum;
      w_sq[wid] = lsq;
      w_max[wid] = wmax;
    }
    if (tid == 0) s_idx = INT_MAX;
    __syncthreads();
    float bmax = w_max[0];
#pragma unroll
    for (int w = 1; w < NWB; ++w) bmax = fmaxf(bmax, w_max[w]);
    if (lmax == bmax) {
      int best = INT_MAX;
#pragma unroll
      for (int m = 0; m < K::E / LP; ++m) {
#pragma unroll
        for (int q = 0; q < LP; ++q) {
          const float2 z = v[m * LP + dft_perm<LP>(q)];
          const int o = fft_out_index<N>(t, m, q);
          if (z.x == bmax) best = min(best, y * N + o);
          if (z.y == bmax) best = min(best, (y + 1) * N + o);
        }
      }
      atomicMin(&s_idx, best);
    }
    __syncthreads();
    if (tid == 0) {
      float s = 0.f, q2 = 0.f;
      for (int w = 0; w < NWB; ++w) {
        s += w_sum[w];
        q2 += w_sq[w];
      }
      StatPartial sp;
      sp.sum = (double)s;
      sp.sumsq = (double)q2;
      sp.max = bmax;
      sp.idx = s_idx;
      sp.pad[0] = sp.pad[1] = 0;
      partials[(size_t)item] = sp;
    }
  }
}

inline int sm_count() {
  static int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

template <int N, bool FP16>
cudaError_t run_grid_colfft(const SegmentGeom& g, const DevTables& tb, const void* S, const Group* groups,
                            int g_begin, int ngroups, int img_base, float2* Tbuf, cudaStream_t st) {
  using K = ImgCfg<N>;
  const int smem = K::SMEM_A_FIXED + g.max_cells * (K::CELL_PITCH * 8 + 4) + g.nchan * 4;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_grid_colfft<N, FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_grid_colfft<N, FP16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (ngroups <= 0) return cudaSuccess;
  dim3 grid(ngroups, g.ncol);
  k_grid_colfft<N, FP16><<<grid, K::THREADS_A, smem, st>>>(g, tb, S, groups, g_begin, img_base, Tbuf);
  return cudaGetLastError();
}

template <int N>
cudaError_t run_rowfft_stats(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, int nimg,
                             int img_base, const double* weight, StatPartial* partials, float* images,
                             cudaStream_t st) {
  using K = ImgCfg<N>;
  const int smem = K::SMEM_B_FIXED + g.ncol * K::CH * 16;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_rowfft_stats<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rowfft_stats<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (nimg <= 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowfft_stats<N>, K::THREADS_B, smem);
  if (e != cudaSuccess) return e;
  const long nitems = (long)nimg * (N / K::RB);
  const long grid = std::min<long>(nitems, (long)std::max(per_sm, 1) * sm_count());
  k_rowfft_stats<N><<<(int)grid, K::THREADS_B, smem, st>>>(g, tb, Tbuf, nimg, img_base, weight, partials, images);
  return cudaGetLastError();
}

template <int N>
void fill_shape(ImageKernelShape* o) {
  using K = ImgCfg<N>;
  o->images_per_group = K::B;
  o->cols_per_cta = 1;
  o->threads_a = K::THREADS_A;
  o->smem_a = K::SMEM_A_FIXED;
  o->warps_per_col = K::WPC;
  o->rows_per_cta = K::RB;
  o->threads_b = K::THREADS_B;
  o->smem_b = K::SMEM_B_FIXED;
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
