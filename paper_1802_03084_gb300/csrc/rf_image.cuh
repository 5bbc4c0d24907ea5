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
#include <cstring>
#include <utility>

#include "rf_engine.h"
#include "rf_async.cuh"
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
  static constexpr int PART_IMAGES = N >= 2048 ? 16 : 32;        // images whose cells are staged at once
  static constexpr int SMEM_A_FIXED = XA * fft_stride<N>() * 8;
  // pass B (row pass): EB values per thread, TB threads per transform, XB row
  // pairs (RB rows) per work item; the column-FFT tile of the next item is
  // prefetched while the current one is transformed
  static constexpr int EB = N == 2048 ? RF_ROW_VALUES_2048 : E;
  static constexpr int TB = N / EB;
  static constexpr int XB = cmin((EB == 32 ? 256 : 512) / TB, N / 2);
  static constexpr int THREADS_B = TB * XB;
  static constexpr int RB = 2 * XB;
  static constexpr int PARTIALS = (N / 2) * (TB > 32 ? TB / 32 : 1);  // row-pass partials per image
  static constexpr int CH = XB;                                  // 16-byte chunks per tile row
  static constexpr int STRIDE = fft_stride<N>();
  // N = 2048 (32 values a thread): each row-pair transform is split by one
  // decimation-in-frequency step into two length-N/2 transforms, the even
  // and the odd pixels, one per warp of the transform (see row_zbuild)
  static constexpr int RSPLIT = (N == 2048 && EB == 32) ? 2 : 1;
  static constexpr int STRIDE_B = RSPLIT * fft_stride<N / RSPLIT>();  // float2 per row transform
  static constexpr int SMEM_B_FIXED = XB * STRIDE_B * 8;
  // N >= 1024: the row-pass tile arrives by tensor copies (TMA) whose
  // 16 CH-byte rows are swizzled by the hardware: chunk c of row u lands at
  // c ^ ((u >> SWZ_SH) & (CH - 1)) for 128-, 64- and 32-byte rows.  The same
  // pattern is used by the cp.async fallback and by every read of the tile.
  static constexpr bool TILE_TMA = N >= 1024;
  static constexpr int SWZ_SH = CH == 4 ? 1 : (CH == 2 ? 2 : 0);
  __device__ static __forceinline__ int swz(int u, int c) { return c ^ ((u >> SWZ_SH) & (CH - 1)); }
  static_assert((T <= 32 || XA <= 15) && (TB <= 32 || XB <= 15), "named barriers: at most 15 wide transforms per block");
  static_assert(FftShape<N>::P2 == fft_pass2_radix(N), "twiddle table layout and FFT passes disagree");
};

// Launch shape of the batched column pass (k_colfft) per image side N: each
// column is R = col_split(N) transforms of length L = N / R (TL threads of EL
// values each); a round runs XA columns' transforms (one image each) at once.
template <int N>
struct ColCfg {
  static constexpr int R = col_split(N);
  static constexpr int L = N / R;
  static constexpr int LOG2L = FftShape<L>::LOG2N;
  static constexpr int TL = FftShape<L>::T;
  static constexpr int EL = FftShape<L>::E;
  static constexpr int THREADS = 256;
  static constexpr int XA = cmin(THREADS / (R * TL), 32);       // images per round
  static constexpr int PI = N >= 2048 ? 16 : 32;                // images whose cells are staged at once
  static constexpr int STRIDE = fft_stride<L>();
  // FFT buffers [XA][R][STRIDE]; per cell of the busiest column: the staged
  // values (PI images), its row and (at most) one run with its R - 1 twiddles
  static constexpr int SMEM_FIXED = XA * R * STRIDE * 8;
  static constexpr int SMEM_PER_CELL = PI * 8 + 4 + 4 + (R - 1) * 8;
  static_assert(TL <= 32, "column sub-transforms fit one warp");
  static_assert(R <= 8, "at most eight sub-transforms per column");
  static_assert((XA * R * STRIDE * 8) % 16 == 0, "staged cells start 16-byte aligned");
};

// Image row of index i of the column-FFT output (see SegmentGeom::tsplit).
__device__ __forceinline__ int t_row(int i, int tsplit, int log2l) {
  return tsplit > 1 ? ((i & ((1 << log2l) - 1)) * tsplit + (i >> log2l)) : i;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }


// Column pass: the first-pass inputs of sub-transform p (of R) of staged
// image kl, through the sub-transform's own buffer.  Its lanes zero the
// buffer and scatter the column's runs into it: run j (cells at rows
// v1 + L v2 for one v1) puts, for R > 1 with the decimation-in-frequency
// step folded in,
//   Y_p[v1] = w_N^(v1 p) sum_{v2 < R} H[v1 + L v2] w_R^(v2 p)
// at row v1 (the run's cells in ascending v2, a fixed order; R = 1: the one
// cell's value).  Only the sub-transform's lanes synchronise.  runs[j] =
// (first cell << 4) | cells; cellv holds PI images per staged cell, 16-byte
// chunks swizzled by the cell.  Not live: the buffer stays zero.
// a times w_R^k, k < R <= 8: exact for the powers of i, the sqrt(1/2)
// constant for the odd eighths.
template <int R>
__device__ __forceinline__ float2 mul_wR(float2 a, int k) {
  const int e = k * (8 / R);  // eighths of a turn
  float2 b = a;
  if (e & 1) b = cmul(a, make_float2(RF_R2_2, RF_R2_2));  // w_8
  switch (e >> 1) {  // quarter turns
    case 1: return make_float2(-b.y, b.x);
    case 2: return make_float2(-b.x, -b.y);
    case 3: return make_float2(b.y, -b.x);
    default: return b;
  }
}

template <int N, int PI>
__device__ __forceinline__ void col_scatter(float2* buf, const int* __restrict__ runs, int nruns,
                                            const float2* __restrict__ cellv, const int* __restrict__ crow, int kl,
                                            bool live, const float2* __restrict__ rtw, int t, int p, int xsub) {
  using C = ColCfg<N>;
  constexpr int CPC = PI > 1 ? PI / 2 : 1;
  constexpr int L = C::L, R = C::R, TL = C::TL, STRIDE = C::STRIDE;
  if constexpr (STRIDE % 2 == 0) {  // 16 bytes at a time (every buffer then starts 16-byte aligned)
    float4* buf4 = reinterpret_cast<float4*>(buf);
    for (int i = t; i < STRIDE / 2; i += TL) buf4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    for (int i = t; i < STRIDE; i += TL) buf[i] = make_float2(0.f, 0.f);
  }
  fft_sync<TL>(xsub);
  if (live) {
    const int kc = kl >> 1, ko = kl & 1;
    for (int j = t; j < nruns; j += TL) {
      const int m = runs[j];
      const int c0 = m >> 4;
      const int v1 = crow[c0] & (L - 1);
      float2 a = cellv[c0 * PI + 2 * (kc ^ (c0 & (CPC - 1))) + ko];
      if constexpr (R > 1) {
        const int n = m & 15;
        if (p > 0) a = mul_wR<R>(a, ((crow[c0] >> C::LOG2L) * p) & (R - 1));
        for (int q = 1; q < n; ++q) {
          const int c = c0 + q;
          float2 h = cellv[c * PI + 2 * (kc ^ (c & (CPC - 1))) + ko];
          if (p > 0) h = mul_wR<R>(h, ((crow[c] >> C::LOG2L) * p) & (R - 1));
          a = cadd(a, h);
        }
        if (p > 0) a = cmul(a, rtw[j * (R - 1) + p - 1]);  // w_N^(v1 p), staged per run
      }
      buf[padx(v1)] = a;
    }
  }
  fft_sync<TL>(xsub);
}

// The length-L inverse FFT of the inputs col_scatter put in `buf`
// (sub-transform xsub of the block), written to dst[0 .. L) if dst.
template <int N>
__device__ __forceinline__ void col_fft_store(float2* buf, const float2* __restrict__ twc, int t, int xsub,
                                              float2* __restrict__ dst) {
  using C = ColCfg<N>;
  constexpr int L = C::L, TL = C::TL, EL = C::EL;
  float2 v[EL];
  fft_inverse_to_regs<L, true>(v, buf, twc, t, xsub);  // packed style (see rf_fft.cuh)
  if (dst != nullptr) {
    constexpr int LP = FftShape<L>::LAST_P;
#pragma unroll
    for (int m = 0; m < EL / LP; ++m)
#pragma unroll
      for (int q = 0; q < LP; ++q) dst[fft_out_index<L>(t, m, q)] = v[m * LP + dft_perm<LP>(q)];
  }
  fft_sync<TL>(xsub);  // the buffer is reused by the next transform
}

// Pass A2: the column FFTs of one group (up to 32 consecutive t' of a
// trial) and one half-plane column u.  The column's cell sums for the
// group's images (cellbuf row per cell, 32 images) are copied to shared
// memory with cp.async (16-byte chunks XOR-swizzled by cell), PI images at a
// time.  Each column is R = col_split(N) sub-transforms of length L = N/R.
// In rounds of XA images, each sub-transform zeroes its own buffer and
// scatters the column's runs into it (col_scatter), which for R > 1 folds in
// one decimation-in-frequency step: sub-transform p takes
//   Y_p[v1] = w_N^(v1 p) sum_{v2 < R} H[v1 + L v2] w_R^(v2 p),
// and its length-L inverse FFT is column output y = R k + p at k, stored at
// T[slot][u][p L + k] (see SegmentGeom::tsplit).  A sub-transform
// synchronises only its own lanes (one warp or part of one), so there is no
// third FFT pass and no barrier across warps for N >= 2048.
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_colfft(SegmentGeom g, DevTables tb, const Group* __restrict__ groups, int g_begin, int img_base,
             const float2* __restrict__ cellbuf, float2* __restrict__ Tbuf, float* __restrict__ colsq,
             float* __restrict__ mean0) {
  using C = ColCfg<N>;
  constexpr int PI = C::PI;          // images staged at a time
  constexpr int CPC = PI / 2;        // 16-byte chunks per cell row
  constexpr int L = C::L, R = C::R, TL = C::TL;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* fbuf = reinterpret_cast<float2*>(smraw);                       // [XA][R][STRIDE]
  float2* cellv = reinterpret_cast<float2*>(fbuf + C::XA * R * C::STRIDE);  // [max_cells][PI], swizzled
  float2* rtw = cellv + (size_t)g.max_cells * PI;                           // [max_cells][R - 1]
  int* crow = reinterpret_cast<int*>(rtw + (size_t)g.max_cells * (R - 1));  // [max_cells]
  int* runs = crow + g.max_cells;                                           // [max_cells]
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const Group gr = groups[g_begin + blockIdx.x];
  const int col = blockIdx.y;
  const int cell0 = tb.col_cell_ptr[col];
  const int ncells = tb.col_cell_ptr[col + 1] - cell0;
  const float2* __restrict__ src = cellbuf + ((size_t)blockIdx.x * g.ncells + cell0) * 32;
  // the column's cell rows and runs; visible after the first staging wait
  // and barrier below
  const int run0 = tb.col_run_ptr[col];
  const int nruns = tb.col_run_ptr[col + 1] - run0;
  for (int c = tid; c < ncells; c += C::THREADS) crow[c] = tb.cell_row[cell0 + c];
  for (int j = tid; j < nruns; j += C::THREADS) runs[j] = tb.col_runs[run0 + j];
  if constexpr (R > 1)
    for (int i = tid; i < nruns * (R - 1); i += C::THREADS) rtw[i] = tb.col_run_tw[(size_t)run0 * (R - 1) + i];
  const int xf = tid / (R * TL);          // image of the round
  const int p = (tid / TL) % R;           // sub-transform: output rows y = p mod R
  const int t = tid % TL;
  float2* buf = fbuf + (xf * R + p) * C::STRIDE;
  for (int kbase = 0; kbase < gr.nimg; kbase += PI) {
    if (kbase > 0) __syncthreads();  // the previous part's cells are consumed
    for (int i = tid; i < ncells * CPC; i += C::THREADS) {
      const int c = i / CPC;
      const int j = i - c * CPC;
      cp_async16(cellv + c * PI + 2 * (j ^ (c & (CPC - 1))), src + c * 32 + kbase + 2 * j);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();  // also orders the row map before its first use
    const int nk = min(PI, gr.nimg - kbase);

    // Parseval: the image's sum of squares is N^2 / (4 W^2) times the sum
    // of |G|^2 over the full Hermitian plane, which counts this column
    // twice unless u = 0; its mean is G(0, 0) / (2 W).  Each warp sums
    // |H|^2 of the column's cells for some of the images (FP32, fixed order).
    {
      const float wcol = col == 0 ? 1.f : 2.f;
      for (int kl = tid >> 5; kl < nk; kl += C::THREADS / 32) {
        float acc = 0.f;
        for (int c = lane; c < ncells; c += 32) {
          const float2 h = cellv[c * PI + 2 * ((kl >> 1) ^ (c & (CPC - 1))) + (kl & 1)];
          acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
          const size_t slot = (size_t)(gr.img0 + kbase + kl - img_base);
          colsq[slot * g.ncol + col] = wcol * acc;
          // row 0 sorts first in column 0; cell 0's first chunk is unswizzled
          if (col == 0) mean0[slot] = (ncells > 0 && crow[0] == 0) ? cellv[kl].x : 0.f;
        }
      }
    }

    if (xf < C::XA) {
      const int nrounds = (nk + C::XA - 1) / C::XA;
      for (int rd = 0; rd < nrounds; ++rd) {
        const int kl = rd * C::XA + xf;
        const bool live = kl < nk;
        float2* dst = live ? Tbuf + ((size_t)(gr.img0 + kbase + kl - img_base) * g.ncol + col) * N + p * L : nullptr;
        col_scatter<N, PI>(buf, runs, nruns, cellv, crow, kl, live, rtw, t, p, xf * R + p);
        col_fft_store<N>(buf, tb.twiddle_col, t, xf * R + p, dst);
      }
    }
  }
}

__device__ __forceinline__ void max_merge(float& m, int& i, float m2, int i2) {
  if (m2 > m || (m2 == m && i2 < i)) {
    m = m2;
    i = i2;
  }
}

// Row pass: the first-pass inputs of row pair xf of the item whose tile
// (T rows y0 .. y0 + RB of every imaged column u, swizzled 16-byte chunks)
// is in shared memory.
template <int N>
__device__ __forceinline__ void row_zbuild(float2 (&v)[ImgCfg<N>::EB], const float4* __restrict__ tile, int t,
                                           int xf, int ncol) {
  using K = ImgCfg<N>;
  constexpr int EB = K::EB, TB = K::TB;
  // first-pass inputs Z[u], u = t + r T: a + i b for 0 < u < ncol, the
  // Hermitian mirror conj(a) + i conj(b) for N - u < ncol, real parts at
  // u = 0, zero elsewhere (columns beyond iu_max are empty).  N/2 = (EB/2) TB,
  // so r < EB/2 can only be a direct column and r >= EB/2 only a mirror.
  if constexpr (K::RSPLIT == 2) {
    // split transform: pixel x = 2 k + s is output k of the length-H = N/2
    // inverse DFT of Y_s[u'] = (Z[u'] + (-1)^s Z[u' + H]) exp(+2 pi i u' s / N)
    // (one decimation-in-frequency step).  Warp s of the transform builds
    // Y_s at u' = j + 32 r (lane j, r < 32): Z[u'] is a direct column or
    // zero, Z[u' + H] the mirror of column H - u' or zero.  For s = 1 the
    // factor exp(+2 pi i r / 64) of u' is applied here and exp(+2 pi i j / N)
    // rides on the second-pass twiddles (see row_finish).
    constexpr int H = N / 2;
    static_assert(EB == 32 && TB == 64 && 32 % (K::CH << K::SWZ_SH) == 0, "split row transform layout");
    const int s = t >> 5, j = t & 31;
    const int rd_end = ncol > j ? (ncol - j + 31) / 32 : 0;  // j + 32 r < ncol
    const int xm = H - j - ncol;                              // H - j - 32 r < ncol  <=>  32 r > xm
    const int rm_beg = xm < 0 ? 0 : xm / 32 + 1;
    // the swizzle term of u = j + 32 r (H - j - 32 r) is that of j (H - j)
    const float4* pd = tile + j * K::CH + K::swz(j, xf);
    const float4* pm = tile + (size_t)(H - j) * K::CH + K::swz(H - j, xf);
    // with a = T[u'][y] = (ab.x, ab.y) and b = T[u'][y+1] = (ab.z, ab.w) of
    // the direct column u', and c, d the same of the mirror column H - u':
    //   Z[u'] +- Z[u' + H] = (P.x - Q.y, P.y + Q.x),
    //   P = a +- conj(c), Q = b +- conj(d)  (one packed FMA each)
    // except at u' = 0, where Z[0] takes the real parts (a.x, b.x)
    const float2 pm1 = make_float2(s == 0 ? 1.f : -1.f, s == 0 ? -1.f : 1.f);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      float4 ab = make_float4(0.f, 0.f, 0.f, 0.f), cd = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rd_end) ab = pd[r * 32 * K::CH];
      if (r >= rm_beg) cd = pm[-r * 32 * K::CH];
      const float2 P = f2_fma(make_float2(cd.x, cd.y), pm1, make_float2(ab.x, ab.y));
      const float2 Q = f2_fma(make_float2(cd.z, cd.w), pm1, make_float2(ab.z, ab.w));
      float2 d = make_float2(P.x - Q.y, P.y + Q.x);
      if (r == 0 && j == 0) {
        const float sg = s == 0 ? 1.f : -1.f;
        d = make_float2(fmaf(sg, cd.x + cd.w, ab.x), fmaf(sg, cd.z - cd.y, ab.z));
      }
      if (s != 0 && r > 0) d = r == 16 ? cmul_i(d) : cmul_c<false>(d, cos_r64(r), sin_r64(r));
      v[r] = d;
    }
  } else if constexpr (TB % (K::CH << K::SWZ_SH) == 0) {
    // the swizzle term of u = t + r T (or N - t - r T) is that of t (N - t)
    const int rd_end = ncol > t ? (ncol - t + TB - 1) / TB : 0;
    const int rm_beg = (N - ncol - t) / TB + 1;
    const float4* pd = tile + t * K::CH + K::swz(t, xf);
    const float4* pm = tile + (size_t)(N - t) * K::CH + K::swz(N - t, xf);
#pragma unroll
    for (int r = 0; r < EB / 2; ++r) {
      float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rd_end) ab = pd[r * TB * K::CH];
      v[r] = (r == 0 && t == 0) ? make_float2(ab.x, ab.z) : make_float2(ab.x - ab.w, ab.y + ab.z);
    }
#pragma unroll
    for (int r = EB / 2; r < EB; ++r) {
      float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r >= rm_beg) ab = pm[-r * TB * K::CH];
      v[r] = make_float2(ab.x + ab.w, ab.z - ab.y);
    }
  } else {
#pragma unroll
    for (int r = 0; r < EB; ++r) {
      const int u = t + r * TB;
      float2 z = make_float2(0.f, 0.f);
      if (u < ncol) {
        const float4 ab = tile[u * K::CH + K::swz(u, xf)];
        z = (u == 0) ? make_float2(ab.x, ab.z) : make_float2(ab.x - ab.w, ab.y + ab.z);
      } else if (N - u < ncol) {
        const int uu = N - u;
        const float4 ab = tile[uu * K::CH + K::swz(uu, xf)];
        z = make_float2(ab.x + ab.w, ab.z - ab.y);
      }
      v[r] = z;
    }
  }
}

// Row pass, after row_zbuild: the inverse FFT of the row pair (T rows
// i = y0 + 2 xf and i + 1, image rows t_row of them) in `buf`, the pair's
// max pixel with its lowest index (and under CLIP the kept-pixel sums), one
// StatPartial per warp of the transform, and the two image rows if `images`.
template <int N, bool CLIP>
__device__ __forceinline__ void row_finish(float2 (&v)[ImgCfg<N>::EB], float2* buf, const float2* __restrict__ tw,
                                           int t, int xf, int slot, int y0, int tsplit, int log2l,
                                           const double* __restrict__ weight, int img_base,
                                           float* __restrict__ images, StatPartial* __restrict__ partials,
                                           const float2* __restrict__ clip) {
  using K = ImgCfg<N>;
  constexpr int EB = K::EB, TB = K::TB;
  constexpr int H = N / K::RSPLIT;  // transform length per warp group
  // split transform (see row_zbuild): warp s runs the length-H transform of
  // Y_s in its own buffer; its second pass takes the pair table of
  // exp(+2 pi i k r / H) (s = 0, the table's section at N) or of
  // exp(+2 pi i r (2k + 1) / N) (s = 1, at N + H), so it is given the
  // table base tw + H + s H (the transform reads only its pair table)
  const int s = K::RSPLIT == 2 ? t >> 5 : 0;
  const int tt = K::RSPLIT == 2 ? t & 31 : t;
  if constexpr (K::RSPLIT == 2) {
    fft_inverse_from_regs<H, false, EB>(v, buf + s * fft_stride<H>(), tw + H + s * H, tt, xf);
  } else {
    fft_inverse_from_regs<N, false, EB>(v, buf, tw, t, xf);
  }
  // pixel of output register (m, q): output o of the transform, or of
  // sub-transform s as pixel 2 o + s
  auto pix = [&](int m, int q) {
    return K::RSPLIT == 2 ? 2 * fft_out_index<H, EB>(tt, m, q) + s : fft_out_index<N, EB>(t, m, q);
  };

  // per-row-pair statistics: the max pixel and its lowest index (the
  // noise comes from the grid by Parseval's identity, see k_colfft).  The
  // pair is T rows i, i + 1, image rows ya < yb (adjacent unless the
  // column pass split its transforms: then R apart)
  const int i = y0 + 2 * xf;
  const int ya = t_row(i, tsplit, log2l);
  const int yb = t_row(i + 1, tsplit, log2l);
  constexpr int LP = FftShape<H, EB>::LAST_P;
  constexpr int EM = EB / LP;
  if (images != nullptr) {
    const double W = weight[img_base + slot];
    const float scale = W > 0.0 ? (float)(0.5 / W) : 0.f;
    float* ima = images + ((size_t)slot * N + ya) * N;
    float* imb = images + ((size_t)slot * N + yb) * N;
#pragma unroll
    for (int m = 0; m < EM; ++m)
#pragma unroll
      for (int q = 0; q < LP; ++q) {
        const float2 z = v[m * LP + dft_perm<LP>(q)];
        const int o = pix(m, q);
        ima[o] = z.x * scale;
        imb[o] = z.y * scale;
      }
  }
  // max of row y (real parts) and of row y + 1 (imaginary parts), four
  // independent chains each
  float mxa[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
  float mya[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
#pragma unroll
  for (int e = 0; e < EB; e += 2) {
    mxa[(e >> 1) & 3] = fmax3f(mxa[(e >> 1) & 3], v[e].x, v[e + 1].x);
    mya[(e >> 1) & 3] = fmax3f(mya[(e >> 1) & 3], v[e].y, v[e + 1].y);
  }
  const float mx = fmaxf(fmaxf(mxa[0], mxa[1]), fmaxf(mxa[2], mxa[3]));
  const float my = fmaxf(fmaxf(mya[0], mya[1]), fmaxf(mya[2], mya[3]));
  const float lmax = fmaxf(mx, my);
  // reduce over the transform's T threads (a warp, a part of one, or
  // several warps joined through shared memory)
  constexpr int WL = TB < 32 ? TB : 32;
  constexpr unsigned MASK = 0xffffffffu;
  float wmax = lmax;
#pragma unroll
  for (int off = WL / 2; off > 0; off >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(MASK, wmax, off));
  // a lane holding the maximum finds its lowest index: row ya comes before
  // row yb, and within a row the lane's outputs ascend with (q, m)
  int best = INT_MAX;
  if (lmax == wmax) {
    if (mx == wmax) {
#pragma unroll
      for (int q = 0; q < LP; ++q)
#pragma unroll
        for (int m = 0; m < EM; ++m)
          if (v[m * LP + dft_perm<LP>(q)].x == wmax) {
            best = ya * N + pix(m, q);
            goto found;
          }
    } else {
#pragma unroll
      for (int q = 0; q < LP; ++q)
#pragma unroll
        for (int m = 0; m < EM; ++m)
          if (v[m * LP + dft_perm<LP>(q)].y == wmax) {
            best = yb * N + pix(m, q);
            goto found;
          }
    }
  found:;
  }
#pragma unroll
  for (int off = WL / 2; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(MASK, best, off));
  // clipped noise: sums of the kept pixels' deviations from mean0, rows y
  // and y + 1 in separate chains
  float s1 = 0.f, s2 = 0.f;
  int cn = 0;
  if constexpr (CLIP) {
    const float2 cw = clip[slot];
    float ax = 0.f, qx = 0.f, ay = 0.f, qy = 0.f;
    int nx = 0, ny = 0;
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const float dx = v[e].x - cw.x;
      const float dy = v[e].y - cw.x;
      if (fabsf(dx) <= cw.y) {
        ax += dx;
        qx = fmaf(dx, dx, qx);
        ++nx;
      }
      if (fabsf(dy) <= cw.y) {
        ay += dy;
        qy = fmaf(dy, dy, qy);
        ++ny;
      }
    }
    s1 = ax + ay;
    s2 = qx + qy;
    cn = nx + ny;
#pragma unroll
    for (int off = WL / 2; off > 0; off >>= 1) {
      s1 += __shfl_xor_sync(MASK, s1, off);
      s2 += __shfl_xor_sync(MASK, s2, off);
      cn += __shfl_xor_sync(MASK, cn, off);
    }
  }
  // one partial per warp of the transform (WPT of them when a transform
  // spans several warps; the finalisation combines them): no barrier
  if ((t & 31) == 0) {
    constexpr int WPT = TB > 32 ? TB / 32 : 1;
    StatPartial sp;
    sp.sum = s1;
    sp.sumsq = s2;
    sp.kept = cn;
    sp.max = wmax;
    sp.idx = best;
    sp.pad = 0;
    partials[(size_t)slot * K::PARTIALS + ((y0 >> 1) + xf) * WPT + (t >> 5)] = sp;  // by T row pair
  }
}

// Pass B: work item = (image slot, block of RB rows); each pair of rows
// shares one complex inverse FFT.  Blocks loop over items; the column-FFT
// tile T[slot][u][y0 .. y0+RB) of the next item is copied to shared memory
// with cp.async (16-byte chunks, XOR-swizzled per row so the strided reads
// are free of bank conflicts) while the current item is transformed.  Each
// warp of a row pair's transform writes one StatPartial (one per row pair
// when the transform fits a warp, T/32 of them when it spans several): the
// max pixel of its part of the two rows with its lowest index, and under
// CLIP the kept-pixel sums (FP32 per thread and across the warp's lanes; the
// finalisation combines an image's partials in FP64).
// With tma_boxes > 0 (N >= 1024 only) thread 0 fetches each item's tile with
// tma_boxes tensor copies of tma_rows u rows from `tmap` ([slot][u][2N
// floats]) and every thread waits on an mbarrier; a wait that gives up sets
// *err, waits once more (bounded) for the copy in flight, and the block
// returns.  Otherwise the threads copy it with cp.async.
// CLIP (the one-pass clipped noise): clip[slot] = {mean0, r} in raw pixel
// units, and each row pair also sums d = J - mean0 and d^2 over its pixels J
// with |d| <= r and counts them (FP32 per thread and across the transform's
// threads in a fixed order).
template <int N, bool CLIP>
__global__ void __launch_bounds__(ImgCfg<N>::THREADS_B, 2)
    k_rowfft_stats(SegmentGeom g, DevTables tb, const float2* __restrict__ Tbuf, int nimg, int img_base,
                   const double* __restrict__ weight, StatPartial* __restrict__ partials,
                   float* __restrict__ images, const __grid_constant__ CUtensorMap tmap, int tma_boxes,
                   int tma_rows, int* __restrict__ err, const float2* __restrict__ clip) {
  using K = ImgCfg<N>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* fbuf = reinterpret_cast<float2*>(smraw);  // [XB][STRIDE_B]
  unsigned char* tb0 = smraw + K::XB * K::STRIDE_B * 8;
  if constexpr (K::TILE_TMA) tb0 += (1024u - (smem_u32(tb0) & 1023u)) & 1023u;  // swizzle atom alignment
  float4* tile = reinterpret_cast<float4*>(tb0);    // [rows][CH]
  __shared__ __align__(8) unsigned long long tbar;
  __shared__ int s_done;  // warps done reading the tile in hand (warp-local transforms)
  const int tid = threadIdx.x;
  const int ncol = g.ncol;
  constexpr int nrb = N / K::RB;
  const int nitems = nimg * nrb;
  const int xf = tid / K::TB;
  const int t = tid - xf * K::TB;
  const int log2l = FftShape<N>::LOG2N - (g.tsplit > 1 ? __ffs(g.tsplit) - 1 : 0);
  const bool use_tma = K::TILE_TMA && tma_boxes > 0;
  // With tensor copies and transforms that synchronise only within a warp,
  // the warps of a block do not wait for one another: each waits for the
  // tile on its own, and the last warp to finish reading it issues the next
  // item's copy.  Otherwise two block barriers per item.
  constexpr bool WARP_LOCAL = K::TILE_TMA && (K::TB <= 32 || K::RSPLIT == 2);
  constexpr int NWB = K::THREADS_B / 32;
  unsigned phase = 0;
  if (use_tma) {
    if (tid == 0) {
      mbar_init(&tbar, 1);
      s_done = 0;
    }
    __syncthreads();
  }
  auto issue_tma = [&](int it) {  // by one thread
    const int sl = it / nrb;
    const int yb = (it - sl * nrb) * K::RB;
    mbar_expect_tx(&tbar, (unsigned)(tma_boxes * tma_rows * K::CH * 16));
    for (int b = 0; b < tma_boxes; ++b)
      tma_load_3d(tile + (size_t)b * tma_rows * K::CH, &tmap, 2 * yb, b * tma_rows, sl, &tbar);
  };
  auto fetch = [&](int it) {
    const int sl = it / nrb;
    const int yb = (it - sl * nrb) * K::RB;
    if (use_tma) {
      if (tid == 0) issue_tma(it);
    } else {
      const float2* src = Tbuf + (size_t)sl * ncol * N + yb;
      for (int i = tid; i < ncol * K::CH; i += K::THREADS_B) {
        const int u = i / K::CH;
        const int c = i - u * K::CH;
        cp_async16(tile + u * K::CH + K::swz(u, c), src + (size_t)u * N + 2 * c);
      }
      cp_async_commit();
    }
  };

  int item = blockIdx.x;
  if (item < nitems) fetch(item);
  for (; item < nitems; item += gridDim.x) {
    if (use_tma && WARP_LOCAL) {
      // a warp whose bounded wait gives up reports it, waits once more (so
      // that a late copy does not land after the block has left) and leaves;
      // no later copy is issued without its arrival below, so the other
      // warps' waits run out in turn
      if (!__all_sync(0xffffffffu, mbar_wait(&tbar, phase))) {
        if ((tid & 31) == 0) atomicExch(err, 1);
        mbar_wait(&tbar, phase);
        return;
      }
      phase ^= 1u;
    } else if (use_tma) {
      const bool ok = mbar_wait(&tbar, phase);
      if (__syncthreads_or(!ok)) {
        // the item's tile copy has not completed: give it one more bounded
        // wait, so that it does not land in shared memory after the block
        // has left, then report the timeout and leave
        if (tid == 0) {
          atomicExch(err, 1);
          mbar_wait(&tbar, phase);
        }
        __syncthreads();
        return;
      }
      phase ^= 1u;
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    const int slot = item / nrb;
    const int y0 = (item - slot * nrb) * K::RB;
    float2 v[K::EB];
    row_zbuild<N>(v, tile, t, xf, ncol);
    if (use_tma && WARP_LOCAL) {
      // tile consumed by this warp; the last of the block's warps resets the
      // count and issues the next item's copy (no warp waits for the tile
      // of item + 2 grid strides before every warp has read item + 1's)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if ((tid & 31) == 0) {
        __threadfence_block();
        if (atomicAdd(&s_done, 1) == NWB - 1) {
          s_done = 0;
          __threadfence_block();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if (item + (int)gridDim.x < nitems) issue_tma(item + gridDim.x);
        }
      }
    } else {
      __syncthreads();  // tile consumed: prefetch the next item
      if (item + (int)gridDim.x < nitems) fetch(item + gridDim.x);
    }
    row_finish<N, CLIP>(v, fbuf + xf * K::STRIDE_B, tb.twiddle, t, xf, slot, y0, g.tsplit, log2l,
                        images != nullptr ? weight : nullptr, img_base, images, partials, clip);
  }
}

// ------------------------------------------------------- fused imaging pass
// Launch shape of the fused column + row pass (N = 1024 .. 4096): one block
// shape serves both roles; a chunk is CI = ColCfg<N>::XA images, one column
// round.
template <int N>
struct FusedCfg {
  using K = ImgCfg<N>;
  using C = ColCfg<N>;
  static constexpr int CI = C::XA;                    // images per chunk
  static constexpr int NRB = N / K::RB;               // row items per image
  static constexpr int FB = cmax(K::XB * K::STRIDE_B, C::XA * C::R * C::STRIDE);  // float2 of FFT buffers
  static constexpr int THREADS = K::THREADS_B;
  static_assert(K::THREADS_B == C::THREADS, "one block shape for both roles");
  static_assert(K::TILE_TMA && CI >= 2, "fused pass: N = 1024 .. 4096");
};

// The fused imaging pass of one wave: the column FFTs and the row FFTs with
// statistics in one persistent launch, the column-FFT output staying in an
// L2-resident ring of `ring` chunk slots instead of a wave-sized buffer in
// HBM.  Blocks take work items in order from one counter (two ahead of the
// item in hand, so the counter's latency is hidden).  Step s holds the ncol
// column items of chunk s (u = 0 .. ncol-1: stage the column's row map,
// rows and cells for the chunk's images, Parseval sums, one round of column
// transforms, store into ring slot s mod ring), then the row items of chunk
// s - 1 (image, block of RB rows: tensor-copy tile, row FFTs, statistics,
// as in k_rowfft_stats).  A row item waits until every warp of its chunk's
// ncol column items has stored; a warp of a column item of chunk s >= ring
// waits, before it stores, until the row items of chunk s - ring have read
// the slot.  Every wait is on items taken from the counter earlier, and a
// block finishes its item before it starts the next one it took, so the
// smallest unfinished item always has its inputs: the order cannot
// deadlock.  Each wait is bounded; one that gives up sets *err (the other
// blocks then stop at their next wait or item) and the block leaves after
// its copies in flight have landed.  The staging area (a row item's tile, or
// a column item's map, rows and cells) is filled for the next item as soon
// as the current one has read it.
// counters: [0] work counter, [1 + c] warps of chunk c's column items that
// stored, [1 + nchunks + c] row items that read chunk c's slot; zero at launch.
template <int N>
__global__ void __launch_bounds__(FusedCfg<N>::THREADS, 2)
    k_image_fused(SegmentGeom g, DevTables tb, const Group* __restrict__ groups, int g_begin,
                  const FusedChunk* __restrict__ chunks, int nchunks, int img_base,
                  const float2* __restrict__ cellbuf, float2* __restrict__ Tring, int ring,
                  float* __restrict__ colsq, float* __restrict__ mean0, StatPartial* __restrict__ partials,
                  const __grid_constant__ CUtensorMap tmap, int tma_boxes, int tma_rows, int* __restrict__ counters,
                  int* __restrict__ err) {
  using K = ImgCfg<N>;
  using C = ColCfg<N>;
  using F = FusedCfg<N>;
  constexpr int CI = F::CI;
  constexpr int CPC = CI / 2;       // 16-byte chunks per staged cell row
  constexpr int NRB = F::NRB;
  constexpr int WPB = F::THREADS / 32;
  constexpr int L = C::L, R = C::R, TL = C::TL;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* fbuf = reinterpret_cast<float2*>(smraw);
  unsigned char* st0 = smraw + F::FB * 8;
  st0 += (1024u - (smem_u32(st0) & 1023u)) & 1023u;  // swizzle atom alignment of the tile
  float4* tile = reinterpret_cast<float4*>(st0);                           // row role: [rows][CH]
  float2* cellv = reinterpret_cast<float2*>(st0);                          // column role: [max_cells][CI]
  float2* rtw = cellv + (size_t)g.max_cells * CI;                           // [max_cells][R - 1]
  int* crow = reinterpret_cast<int*>(rtw + (size_t)g.max_cells * (R - 1));  // [max_cells]
  int* runs = crow + g.max_cells;                                           // [max_cells]
  __shared__ __align__(8) unsigned long long tbar;
  __shared__ int s_q;     // the item after next
  __shared__ int s_fail;  // a wait gave up, or another block reported one
  __shared__ int s_pf;    // the next item's tile copy was issued
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int ncol = g.ncol;
  const int ips = ncol + CI * NRB;  // items per step
  const long total = (long)(nchunks + 1) * ips;
  int* const work = counters;
  int* const colcnt = counters + 1;
  int* const rowcnt = counters + 1 + nchunks;
  const int log2l = FftShape<N>::LOG2N - (g.tsplit > 1 ? __ffs(g.tsplit) - 1 : 0);
  const unsigned tile_bytes = (unsigned)(tma_boxes * tma_rows * K::CH * 16);
  // roles' thread layouts
  const int xfb = tid / K::TB, tb_ = tid - xfb * K::TB;                // row role
  const int xfa = tid / (R * TL), pa = (tid / TL) % R, ta = tid % TL;  // column role

  // An item's place in the order: kind 0 none, 1 column (chunk c, column a),
  // 2 row (chunk c, image a, block b), with its chunk and the wave slot of the
  // chunk's first image.  The chunk and group loads are issued one item ahead.
  struct Item {
    int kind, c, a, b, slot0;
    FusedChunk ch;
  };
  auto locate = [&](long qq) -> Item {  // arithmetic, then the chunk's loads
    Item it{0, 0, 0, 0, 0, {0, 0, 0, 0}};
    if (qq >= total) return it;
    const int st = (int)(qq / ips), o = (int)(qq - (long)st * ips);
    if (o < ncol) {
      it.c = st;
      it.a = o;
      it.kind = st < nchunks ? 1 : 0;
    } else {
      it.c = st - 1;
      const int j = o - ncol;
      it.a = j / NRB;
      it.b = j - it.a * NRB;
      it.kind = (it.c >= 0 && it.c < nchunks) ? 2 : 0;
    }
    if (it.kind != 0) {
      it.ch = chunks[it.c];
      it.slot0 = groups[it.ch.g].img0 + it.ch.kbase - img_base;
    }
    return it;
  };
  // the kind once the chunk is known: a row item past the chunk's images is none
  auto kind_of = [&](const Item& it) { return (it.kind == 2 && it.a >= it.ch.nk) ? 0 : it.kind; };
  auto ring_slot = [&](int c, int jj) { return (c % ring) * CI + jj; };
  auto issue_tile = [&](int c, int jj, int rb) {  // thread 0
    fence_proxy_async_global();
    mbar_expect_tx(&tbar, tile_bytes);
    for (int bx = 0; bx < tma_boxes; ++bx)
      tma_load_3d(tile + (size_t)bx * tma_rows * K::CH, &tmap, 2 * rb * K::RB, bx * tma_rows, ring_slot(c, jj),
                  &tbar);
  };
  auto issue_stage = [&](const FusedChunk& ch, int u) {  // all threads: the column's rows, runs and cells
    const int cell0 = tb.col_cell_ptr[u];
    const int nc = tb.col_cell_ptr[u + 1] - cell0;
    const int run0 = tb.col_run_ptr[u];
    const int nr = tb.col_run_ptr[u + 1] - run0;
    for (int cc = tid; cc < nc; cc += F::THREADS) cp_async4(crow + cc, tb.cell_row + cell0 + cc);
    for (int j = tid; j < nr; j += F::THREADS) cp_async4(runs + j, tb.col_runs + run0 + j);
    if constexpr (R > 1)
      for (int i = tid; i < nr * (R - 1); i += F::THREADS) cp_async8(rtw + i, tb.col_run_tw + (size_t)run0 * (R - 1) + i);
    const float2* src = cellbuf + ((size_t)(ch.g - g_begin) * g.ncells + cell0) * 32 + ch.kbase;
    for (int i = tid; i < nc * CPC; i += F::THREADS) {
      const int cc = i / CPC;
      const int j = i - cc * CPC;
      cp_async16(cellv + cc * CI + 2 * (j ^ (cc & (CPC - 1))), src + cc * 32 + 2 * j);
    }
    cp_async_commit();
  };
  // fill the staging area for item qn after the current item has read it:
  // a column item's stage (all threads), or a row item's tile if its chunk is
  // complete (thread 0; *pf tells)
  auto prefetch = [&](const Item& nx, bool& stage_ready, int& pf) {
    const int k2 = kind_of(nx);
    stage_ready = false;
    if (k2 == 2) {
      if (tid == 0 && ld_acquire_gpu(colcnt + nx.c) >= ncol * WPB) {
        issue_tile(nx.c, nx.a, nx.b);
        pf = 1;
      }
    } else if (k2 == 1) {
      issue_stage(nx.ch, nx.a);
      stage_ready = true;
    }
  };

  if (tid == 0) {
    mbar_init(&tbar, 1);
    s_fail = 0;
    s_pf = 0;
    s_q = atomicAdd(work, 1);
  }
  __syncthreads();
  long q = s_q;
  __syncthreads();
  if (tid == 0) s_q = atomicAdd(work, 1);
  __syncthreads();
  long qn = s_q;
  unsigned phase = 0;
  bool tile_ready = false;   // a tile copy for item q is in flight
  bool stage_ready = false;  // item q's column stage is in flight (cp.async)
  Item cur = locate(q);

  while (q < total) {
    int qf = 0;
    if (tid == 0) qf = atomicAdd(work, 1);  // the item after next, used at the item's end
    const Item nxt = locate(qn);             // its loads complete during this item
    int pf = 0;                              // thread 0: a tile copy for item qn was issued
    bool next_stage = false;
    const int kind = kind_of(cur);
    const int c = cur.c, a = cur.a, b = cur.b;
    if (kind == 2) {
      // ------------------------------------------------------------ row item
      if (!tile_ready) {
        bool bad = false;
        if (tid == 0) {
          if (wait_count(colcnt + c, ncol * WPB, err)) issue_tile(c, a, b);
          else bad = true;
        }
        if (__syncthreads_or(bad)) {
          if (tid == 0) atomicExch(err, 1);
          cp_async_wait_all();
          __syncthreads();
          return;
        }
      }
      const bool ok = mbar_wait(&tbar, phase);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(err, 1);
          mbar_wait(&tbar, phase);  // once more, so the copy does not land after the block has left
        }
        cp_async_wait_all();
        __syncthreads();
        return;
      }
      phase ^= 1u;
      if (tid == 0) {  // the tile's reads of the ring slot are complete
        fence_proxy_async_global();
        __threadfence();
        atomicAdd(rowcnt + c, 1);
      }
      float2 v[K::EB];
      row_zbuild<N>(v, tile, tb_, xfb, ncol);
      __syncthreads();  // the staging area is read
      prefetch(nxt, next_stage, pf);
      const int slot = cur.slot0 + a;
      row_finish<N, false>(v, fbuf + xfb * K::STRIDE_B, tb.twiddle, tb_, xfb, slot, b * K::RB, g.tsplit, log2l,
                           nullptr, img_base, nullptr, partials, nullptr);
    } else if (kind == 1) {
      // --------------------------------------------------------- column item
      const FusedChunk ch = cur.ch;
      const int u = a;
      const int ncells = tb.col_cell_ptr[u + 1] - tb.col_cell_ptr[u];
      const int nruns = tb.col_run_ptr[u + 1] - tb.col_run_ptr[u];
      if (!stage_ready) issue_stage(ch, u);
      cp_async_wait_all();
      __syncthreads();
      const int wslot0 = cur.slot0;
      // Parseval sums of the column, one warp per image
      if (warp < ch.nk) {
        const int kl = warp;
        float acc = 0.f;
        for (int cc = lane; cc < ncells; cc += 32) {
          const float2 h = cellv[cc * CI + 2 * ((kl >> 1) ^ (cc & (CPC - 1))) + (kl & 1)];
          acc = fmaf(h.x, h.x, fmaf(h.y, h.y, acc));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
          colsq[(size_t)(wslot0 + kl) * ncol + u] = (u == 0 ? 1.f : 2.f) * acc;
          if (u == 0) mean0[wslot0 + kl] = (ncells > 0 && crow[0] == 0) ? cellv[kl].x : 0.f;
        }
      }
      float2* buf = fbuf + (xfa * R + pa) * C::STRIDE;
      col_scatter<N, CI>(buf, runs, nruns, cellv, crow, xfa, xfa < ch.nk, rtw, ta, pa, xfa * R + pa);
      __syncthreads();  // the staging area is read
      prefetch(nxt, next_stage, pf);
      // this warp's slot rows are free once the row items of chunk c - ring have read them
      bool ok = true;
      if (c >= ring) {
        if (lane == 0) ok = wait_count(rowcnt + (c - ring), chunks[c - ring].nk * NRB, err);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok && lane == 0) atomicExch(err, 1);
      }
      float2* dst = (ok && xfa < ch.nk) ? Tring + ((size_t)ring_slot(c, xfa) * ncol + u) * N + pa * L : nullptr;
      col_fft_store<N>(buf, tb.twiddle_col, ta, xfa * R + pa, dst);
      if (ok) {
        // the warp's stores, then one cumulative fence and the count (the
        // row items read the slot through the async proxy)
        __syncwarp();
        if (lane == 0) {
          fence_proxy_async_global();
          __threadfence();
          atomicAdd(colcnt + c, 1);
        }
      }
    } else {
      // an empty place of the order (a missing image of a short chunk, the
      // first and last steps): nothing was staged for it
      __syncthreads();
      prefetch(nxt, next_stage, pf);
    }
    // end of the item: publish the item after next and the prefetch; stop
    // if any block has given up
    if (tid == 0) {
      s_q = qf;
      s_pf = pf;
      s_fail = ld_acquire_gpu(err) != 0;
    }
    __syncthreads();
    tile_ready = s_pf != 0;
    stage_ready = next_stage;
    q = qn;
    qn = s_q;
    cur = nxt;
    if (s_fail) {
      if (tid == 0 && tile_ready) mbar_wait(&tbar, phase);
      cp_async_wait_all();
      __syncthreads();
      return;
    }
  }
  cp_async_wait_all();
}

// The most dynamic shared memory a block of `kern` can have: the device's
// opt-in per-block limit (227 KB on sm_103a) less the kernel's static shared
// memory.  Kernels whose request depends on the plan set their attribute to
// this bound, not to the request: the attribute belongs to the kernel, and
// plans searched at once on other host threads (the serving runtime) would
// otherwise lower it under each other's launches.  0 if it cannot be read.
template <class Kernel>
int max_dynamic_smem(Kernel kern) {
  cudaFuncAttributes fa;
  int dev = 0, optin = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return optin - (int)fa.sharedSizeBytes;
}

// Launch `kern`, with the scheduling priority of `pl` where it sets one (a
// launch attribute, so that a captured graph keeps it on the kernel node).
template <class... P, class... A>
cudaError_t launch_with(void (*kern)(P...), dim3 grid, dim3 block, int smem, cudaStream_t st,
                        const PassLaunch* pl, A&&... args) {
  if (pl == nullptr || !pl->set_priority) {
    kern<<<grid, block, smem, st>>>(std::forward<A>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = pl->priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Dynamic shared memory of a column-pass block that keeps a second column
// block off an SM (two such blocks and their reserved shares exceed the
// SM's shared memory) while one row-pass block of `row_smem` bytes still
// fits beside it.  `smem` if that cannot be had (or is already so).
inline int one_per_sm_smem(int smem, int row_smem, int smem_max) {
  int dev = 0, sm_smem = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return smem;
  }
  const int floor = sm_smem / 2 - reserved + 16;
  if (smem >= floor || floor > smem_max || floor + row_smem + 2 * reserved > sm_smem) return smem;
  return floor;
}



// Periodicity row pass (Sec. 3.1 footnote).  A pair is the two quadrature
// images (U and Q) of one (DM trial, fluctuation frequency); work item =
// (pair, block of XB rows), and each transform takes one row y with
// Z[u] = T_U[u][y] + i T_Q[u][y] (Hermitian-extended as in the search's row
// pass), so its output holds row y of I_U in the real parts and of I_Q in
// the imaginary parts.  Per row it writes the maximum of I_U^2 + I_Q^2 (raw
// pixel units) and its lowest index.  pairs[j] = {U slot, Q slot, -, -}.
// The tile is [ncol][CH] 16-byte chunks {U[u][y], Q[u][y]} copied with
// cp.async, or, where every transform fits one warp and tma_boxes > 0
// (N = 1024), two tiles [rows][XB] of U and of Q rows, each filled by
// tma_boxes tensor copies of tma_rows u rows from `tmap` ([slot][u][2N
// floats], boxes of XB complex values, 64-byte rows swizzled by the hardware:
// chunk c of row u at c ^ ((u >> 1) & 3)).  Then, as in the search's row
// pass, no block barrier is left: each warp waits for the tiles on an
// mbarrier (bounded; a warp that gives up sets *err, waits once more and
// leaves) and the last warp to read them issues the next item's copies.
template <int N>
__global__ void __launch_bounds__(ImgCfg<N>::THREADS_B, 2)
    k_rowfft_power(SegmentGeom g, DevTables tb, const float2* __restrict__ Tbuf, const int4* __restrict__ pairs,
                   int npairs, StatPartial* __restrict__ partials, const __grid_constant__ CUtensorMap tmap,
                   int tma_boxes, int tma_rows, int* __restrict__ err) {
  using K = ImgCfg<N>;
  constexpr int EB = K::EB, TB = K::TB;
  constexpr bool PTMA = K::TILE_TMA && TB <= 32;  // warp-local transforms (N = 1024)
  static_assert(!PTMA || (K::XB == 8 && EB == 32), "power tiles: 64-byte rows of 8 complex values");
  constexpr int NWB = K::THREADS_B / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* fbuf = reinterpret_cast<float2*>(smraw);                       // [XB][STRIDE_B]
  float4* tile = reinterpret_cast<float4*>(fbuf + K::XB * K::STRIDE_B);  // [ncol][CH]
  // tensor-copy tiles of U and Q rows, [rows][4 chunks]: U 1024-byte
  // aligned, Q 512 bytes after it (the 64-byte swizzle repeats every 8 rows)
  unsigned char* tu0 = smraw + K::XB * K::STRIDE_B * 8;
  tu0 += (1024u - (smem_u32(tu0) & 1023u)) & 1023u;
  const unsigned tsz = ((unsigned)(tma_boxes * tma_rows * K::XB * 8) + 511u) & ~511u;
  float2* tileU = reinterpret_cast<float2*>(tu0);
  float2* tileQ = reinterpret_cast<float2*>(tu0 + tsz);
  __shared__ float w_max[32];
  __shared__ int w_idx[32];
  __shared__ __align__(8) unsigned long long tbar;
  __shared__ int s_done;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int wid = tid >> 5;
  const int ncol = g.ncol;
  constexpr int nrb = N / K::XB;  // row blocks per pair
  const int nitems = npairs * nrb;
  const int xf = tid / TB;
  const int t = tid - xf * TB;
  const int log2l = FftShape<N>::LOG2N - (g.tsplit > 1 ? __ffs(g.tsplit) - 1 : 0);

  const bool use_tma = PTMA && tma_boxes > 0;
  unsigned phase = 0;
  if (use_tma) {
    if (tid == 0) {
      mbar_init(&tbar, 1);
      s_done = 0;
    }
    __syncthreads();
  }
  auto issue_tma = [&](int it) {  // by one thread
    const int pj = it / nrb;
    const int yb = (it - pj * nrb) * K::XB;
    const int4 pr = pairs[pj];
    mbar_expect_tx(&tbar, (unsigned)(2 * tma_boxes * tma_rows * K::XB * 8));
    for (int b = 0; b < tma_boxes; ++b) {
      tma_load_3d(tileU + (size_t)b * tma_rows * K::XB, &tmap, 2 * yb, b * tma_rows, pr.x, &tbar);
      tma_load_3d(tileQ + (size_t)b * tma_rows * K::XB, &tmap, 2 * yb, b * tma_rows, pr.y, &tbar);
    }
  };
  auto prefetch = [&](int it) {
    if (use_tma) {
      if (tid == 0) issue_tma(it);
      return;
    }
    const int pj = it / nrb;
    const int yb = (it - pj * nrb) * K::XB;
    const int4 pr = pairs[pj];
    const float2* su = Tbuf + (size_t)pr.x * ncol * N + yb;
    const float2* sq = Tbuf + (size_t)pr.y * ncol * N + yb;
    for (int i = tid; i < ncol * K::CH; i += K::THREADS_B) {
      const int u = i / K::CH;
      const int c = i - u * K::CH;
      float2* d = reinterpret_cast<float2*>(tile + u * K::CH + (c ^ (u & (K::CH - 1))));
      cp_async8(d, su + (size_t)u * N + c);
      cp_async8(d + 1, sq + (size_t)u * N + c);
    }
    cp_async_commit();
  };

  int item = blockIdx.x;
  if (item < nitems) prefetch(item);
  for (; item < nitems; item += gridDim.x) {
    if (use_tma) {
      if (!__all_sync(0xffffffffu, mbar_wait(&tbar, phase))) {
        if (lane == 0) atomicExch(err, 1);
        mbar_wait(&tbar, phase);
        return;
      }
      phase ^= 1u;
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    const int pj = item / nrb;
    const int iy = (item - pj * nrb) * K::XB + xf;   // T row; image row y below
    const int y = t_row(iy, g.tsplit, log2l);
    float2 v[EB];
    if (PTMA && use_tma) {
      // the U and Q tiles: complex value xf of u row u is half (xf & 1) of
      // chunk (xf >> 1) ^ ((u >> 1) & 3); for u = t + 32 r (N - t - 32 r)
      // the swizzle term is that of t (N - t)
      const int rd_end = ncol > t ? (ncol - t + TB - 1) / TB : 0;
      const int rm_beg = (N - ncol - t) / TB + 1;
      auto at = [&](int u) { return (u * 4 + ((xf >> 1) ^ ((u >> 1) & 3))) * 2 + (xf & 1); };
      const float2* pdu = tileU + at(t);
      const float2* pdq = tileQ + at(t);
      const float2* pmu = tileU + at(N - t);
      const float2* pmq = tileQ + at(N - t);
      constexpr int RS = TB * 4 * 2;  // float2 per 32 u rows
#pragma unroll
      for (int r = 0; r < EB / 2; ++r) {
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (r < rd_end) {
          a = pdu[r * RS];
          b = pdq[r * RS];
        }
        v[r] = (r == 0 && t == 0) ? make_float2(a.x, b.x) : make_float2(a.x - b.y, a.y + b.x);
      }
#pragma unroll
      for (int r = EB / 2; r < EB; ++r) {
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (r >= rm_beg) {
          a = pmu[-r * RS];
          b = pmq[-r * RS];
        }
        v[r] = make_float2(a.x + b.y, b.x - a.y);
      }
    } else if constexpr (TB % K::CH == 0) {
      // as in the search's row pass: u = t + r T (or N - t - r T) has the
      // swizzle term of t (N - t), and the loads are predicated, not branched
      const int rd_end = ncol > t ? (ncol - t + TB - 1) / TB : 0;
      const int rm_beg = (N - ncol - t) / TB + 1;
      const float4* pd = tile + t * K::CH + (xf ^ (t & (K::CH - 1)));
      const float4* pm = tile + (size_t)(N - t) * K::CH + (xf ^ ((N - t) & (K::CH - 1)));
#pragma unroll
      for (int r = 0; r < EB / 2; ++r) {
        float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rd_end) ab = pd[r * TB * K::CH];
        v[r] = (r == 0 && t == 0) ? make_float2(ab.x, ab.z) : make_float2(ab.x - ab.w, ab.y + ab.z);
      }
#pragma unroll
      for (int r = EB / 2; r < EB; ++r) {
        float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r >= rm_beg) ab = pm[-r * TB * K::CH];
        v[r] = make_float2(ab.x + ab.w, ab.z - ab.y);
      }
    } else {
#pragma unroll
      for (int r = 0; r < EB; ++r) {
        const int u = t + r * TB;
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
    }
    if (use_tma) {
      // tiles read by this warp; the last of the block's warps issues the
      // next item's copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&s_done, 1) == NWB - 1) {
          s_done = 0;
          __threadfence_block();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if (item + (int)gridDim.x < nitems) issue_tma(item + gridDim.x);
        }
      }
    } else {
      __syncthreads();  // tile consumed: prefetch the next item
      if (item + (int)gridDim.x < nitems) prefetch(item + gridDim.x);
    }
    fft_inverse_from_regs<N, false, EB>(v, fbuf + xf * K::STRIDE_B, tb.twiddle, t, xf);

    constexpr int LP = FftShape<N, EB>::LAST_P;
    constexpr int EM = EB / LP;
    float pa[4] = {-1.f, -1.f, -1.f, -1.f};
#pragma unroll
    for (int e = 0; e < EB; ++e) pa[e & 3] = fmaxf(pa[e & 3], fmaf(v[e].x, v[e].x, v[e].y * v[e].y));
    const float lmax = fmaxf(fmaxf(pa[0], pa[1]), fmaxf(pa[2], pa[3]));
    constexpr int WL = TB < 32 ? TB : 32;
    constexpr unsigned MASK = 0xffffffffu;
    float wmax = lmax;
#pragma unroll
    for (int off = WL / 2; off > 0; off >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(MASK, wmax, off));
    int best = INT_MAX;
    if (lmax == wmax) {
#pragma unroll
      for (int q = 0; q < LP; ++q)
#pragma unroll
        for (int m = 0; m < EM; ++m) {
          const float2 z = v[m * LP + dft_perm<LP>(q)];
          if (fmaf(z.x, z.x, z.y * z.y) == wmax) {
            best = y * N + fft_out_index<N, EB>(t, m, q);
            goto found;
          }
        }
    found:;
    }
#pragma unroll
    for (int off = WL / 2; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(MASK, best, off));
    float mx = wmax;
    int mi = best;
    if (TB > 32) {
      constexpr int WPT = TB / 32;
      const int wi = t >> 5;
      if (lane == 0) {
        w_max[wid] = wmax;
        w_idx[wid] = best;
      }
      fft_sync<TB>(xf);
      if (t == 0) {
        const int w0 = wid - wi;
        mx = -1.f;
        mi = INT_MAX;
        for (int w = 0; w < WPT; ++w) max_merge(mx, mi, w_max[w0 + w], w_idx[w0 + w]);
      }
      fft_sync<TB>(xf);
    }
    if (t == 0) {
      StatPartial sp;
      sp.sum = 0.0;
      sp.sumsq = 0.0;
      sp.max = mx;
      sp.idx = mi;
      sp.kept = 0;
      sp.pad = 0;
      partials[(size_t)pj * N + iy] = sp;
    }
  }
}

template <int N>
cudaError_t run_rowfft_power(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, const int4* pairs,
                             int npairs, StatPartial* partials, const TileMap* tm, int* err, cudaStream_t st) {
  using K = ImgCfg<N>;
  // tensor-copy tiles where every transform fits one warp (see k_rowfft_power)
  const bool tma = K::TILE_TMA && K::TB <= 32 && tm != nullptr && tm->nbox > 0 && err != nullptr;
  const int tsz = tma ? (tm->nbox * tm->rows * K::XB * 8 + 511) / 512 * 512 : 0;
  const int smem = tma ? K::SMEM_B_FIXED + 1024 + 2 * tsz : K::SMEM_B_FIXED + g.ncol * K::CH * 16;
  const int smem_max = max_dynamic_smem(k_rowfft_power<N>);
  if (smem > smem_max) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_rowfft_power<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rowfft_power<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (npairs <= 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowfft_power<N>, K::THREADS_B, smem);
  if (e != cudaSuccess) return e;
  const long nitems = (long)npairs * (N / K::XB);
  const long grid = std::min<long>(nitems, (long)std::max(per_sm, 1) * sm_count());
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  k_rowfft_power<N><<<(int)grid, K::THREADS_B, smem, st>>>(g, tb, Tbuf, pairs, npairs, partials,
                                                           tma ? tm->map : none, tma ? tm->nbox : 0,
                                                           tma ? tm->rows : 0, err);
  return cudaGetLastError();
}


template <int N>
int rowfft_tile_rows(int ncol);

template <int N>
cudaError_t run_colfft(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin, int ngroups,
                       int img_base, const float2* cellbuf, float2* Tbuf, float* colsq, float* mean0,
                       cudaStream_t st, const PassLaunch* pl) {
  using C = ColCfg<N>;
  using K = ImgCfg<N>;
  int smem = C::SMEM_FIXED + g.max_cells * C::SMEM_PER_CELL;
  const int smem_max = max_dynamic_smem(k_colfft<N>);
  if (smem > smem_max) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_colfft<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_colfft<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (ngroups <= 0) return cudaSuccess;
  if (pl != nullptr && pl->one_per_sm)
    smem = one_per_sm_smem(smem, K::SMEM_B_FIXED + (K::TILE_TMA ? 1024 : 0) + rowfft_tile_rows<N>(g.ncol) * K::CH * 16,
                           smem_max);
  dim3 grid(ngroups, g.ncol);
  return launch_with(k_colfft<N>, grid, dim3(C::THREADS), smem, st, pl, g, tb, groups, g_begin, img_base, cellbuf,
                     Tbuf, colsq, mean0);
}

// Rows of the row-pass tile: ncol, or the boxes' total under tensor copies.
template <int N>
int rowfft_tile_rows(int ncol) {
  if (!ImgCfg<N>::TILE_TMA) return ncol;
  int nbox, rows;
  tile_boxes(ncol, &nbox, &rows);
  return nbox * rows;
}

template <int N, bool CLIP>
cudaError_t run_rowfft_stats_k(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, int nimg,
                               int img_base, const double* weight, StatPartial* partials, float* images,
                               const TileMap* tm, int* err, cudaStream_t st, const float2* clip,
                               const PassLaunch* pl) {
  using K = ImgCfg<N>;
  const int smem = K::SMEM_B_FIXED + (K::TILE_TMA ? 1024 : 0) + rowfft_tile_rows<N>(g.ncol) * K::CH * 16;
  auto kern = k_rowfft_stats<N, CLIP>;
  const int smem_max = max_dynamic_smem(kern);
  if (smem > smem_max) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (nimg <= 0) return cudaSuccess;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::THREADS_B, smem);
  if (e != cudaSuccess) return e;
  const long nitems = (long)nimg * (N / K::RB);
  long grid = std::min<long>(nitems, (long)std::max(per_sm, 1) * sm_count());
  // short-lived blocks of items_per_block items (the kernel strides by the grid)
  if (pl != nullptr && pl->items_per_block > 0)
    grid = std::max(grid, std::min<long>((nitems + pl->items_per_block - 1) / pl->items_per_block, INT_MAX));
  const bool tma = K::TILE_TMA && tm != nullptr && tm->nbox > 0 && err != nullptr;
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  return launch_with(kern, dim3((unsigned)grid), dim3(K::THREADS_B), smem, st, pl, g, tb, Tbuf, nimg, img_base,
                     weight, partials, images, tma ? tm->map : none, tma ? tm->nbox : 0, tma ? tm->rows : 0, err,
                     clip);
}

template <int N>
cudaError_t run_rowfft_stats(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, int nimg,
                             int img_base, const double* weight, StatPartial* partials, float* images,
                             const TileMap* tm, int* err, cudaStream_t st, const float2* clip,
                             const PassLaunch* pl) {
  if (clip != nullptr)
    return run_rowfft_stats_k<N, true>(g, tb, Tbuf, nimg, img_base, weight, partials, images, tm, err, st, clip,
                                       pl);
  return run_rowfft_stats_k<N, false>(g, tb, Tbuf, nimg, img_base, weight, partials, images, tm, err, st, nullptr,
                                      pl);
}

template <int N>
cudaError_t run_image_fused(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                            const FusedChunk* chunks, int nchunks, int img_base, const float2* cellbuf,
                            float2* Tring, int ring, const TileMap& tm, float* colsq, float* mean0,
                            StatPartial* partials, int* counters, int* err, cudaStream_t st) {
  using K = ImgCfg<N>;
  using C = ColCfg<N>;
  using F = FusedCfg<N>;
  if (nchunks <= 0) return cudaSuccess;
  if (tm.nbox <= 0 || ring < 2) return cudaErrorInvalidValue;
  const int tile = rowfft_tile_rows<N>(g.ncol) * K::CH * 16;
  const int cols = g.max_cells * (F::CI * 8 + 8 + (C::R - 1) * 8);
  const int smem = F::FB * 8 + 1024 + std::max(tile, cols);
  auto kern = k_image_fused<N>;
  const int smem_max = max_dynamic_smem(kern);
  if (smem > smem_max) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counters, 0, (size_t)(1 + 2 * nchunks) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, F::THREADS, smem);
  if (e != cudaSuccess) return e;
  const long items = (long)(nchunks + 1) * (g.ncol + F::CI * F::NRB);
  const long grid = std::min<long>(items, (long)std::max(per_sm, 1) * sm_count());
  kern<<<(int)grid, F::THREADS, smem, st>>>(g, tb, groups, g_begin, chunks, nchunks, img_base, cellbuf, Tring, ring,
                                           colsq, mean0, partials, tm.map, tm.nbox, tm.rows, counters, err);
  return cudaGetLastError();
}

template <int N>
void fill_shape(ImageKernelShape* o) {
  using K = ImgCfg<N>;
  o->images_per_group = K::B;
  o->cols_per_cta = 1;
  o->threads_a = ColCfg<N>::THREADS;
  o->smem_a = ColCfg<N>::SMEM_FIXED;
  o->warps_per_col = 0;
  o->rows_per_cta = K::RB;
  o->partials_per_image = K::PARTIALS;
  o->threads_b = K::THREADS_B;
  o->smem_b = K::SMEM_B_FIXED;
  o->smem_a_per_cell = ColCfg<N>::SMEM_PER_CELL;
  o->smem_b_per_row = K::CH * 16;
  o->tile_tma = K::TILE_TMA;
}

#define RF_INSTANTIATE_IMAGE(N)                                                                              \
  template cudaError_t run_colfft<N>(const SegmentGeom&, const DevTables&, const Group*, int, int, int,      \
                                     const float2*, float2*, float*, float*, cudaStream_t,                  \
                                     const PassLaunch*);                                                    \
  template cudaError_t run_rowfft_stats<N>(const SegmentGeom&, const DevTables&, const float2*, int, int,    \
                                           const double*, StatPartial*, float*, const TileMap*, int*,       \
                                           cudaStream_t, const float2*, const PassLaunch*);                 \
  template void fill_shape<N>(ImageKernelShape*);                                                           \
  template cudaError_t run_rowfft_power<N>(const SegmentGeom&, const DevTables&, const float2*, const int4*, \
                                           int, StatPartial*, const TileMap*, int*, cudaStream_t);

#define RF_INSTANTIATE_FUSED(N)                                                                              \
  template cudaError_t run_image_fused<N>(const SegmentGeom&, const DevTables&, const Group*, int,            \
                                          const FusedChunk*, int, int, const float2*, float2*, int,         \
                                          const TileMap&, float*, float*, StatPartial*, int*, int*, cudaStream_t);

}  // namespace rf
