// rf_fft.cuh -- shared-memory Stockham FFT building blocks for the imaging
// kernels (the 2D inverse FFT of the dirty image, Sec. 3.1 / Sec. 3.2: "the 2d
// FFT for imaging" is the most demanding stage).
//
// A length-N transform (N a power of two, 16..8192) is done by T = N/16
// threads.  Each pass is a radix-P Stockham autosort step: thread t loads the
// P inputs j + r*(N/P) of each of its 16/P butterflies j, applies the twiddles
// exp(+2 pi i k r / (Ns P)) with k = j mod Ns, does a radix-P inverse DFT in
// registers and stores output q at (j / Ns) Ns P + k + q Ns.  All passes are
// radix 16 except the last, whose radix is N / 16^floor(log16 N) when N is not
// a power of 16.  Data stay in one padded shared-memory buffer per transform;
// a barrier separates the loads and stores of a pass, so the transform is in
// place.  The sign is +1 (inverse DFT, no 1/N scaling).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rf {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }  // i * a
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// exp(2 pi i k / 16) for the constant twiddles inside the radix-8/16 kernels.
#define RF_C16_1 0.92387953251128675613f
#define RF_S16_1 0.38268343236508977173f
#define RF_R2_2 0.70710678118654752440f

// Padded shared-memory index: one spare slot every 16 complex values keeps the
// strided stores of the first pass free of bank conflicts.
__host__ __device__ __forceinline__ constexpr int pad16(int i) { return i + (i >> 4); }

// Per-transform shared-memory stride (in float2).  The extra 2 makes buffers
// of consecutive transforms start on different bank pairs.
template <int N>
__host__ __device__ constexpr int fft_stride() { return N + N / 16 + 2; }

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

// In-register inverse radix-4 on v[0], v[S], v[2S], v[3S] (natural order out).
template <int S>
__device__ __forceinline__ void dft4(float2* v) {
  float2 t0 = cadd(v[0], v[2 * S]);
  float2 t1 = csub(v[0], v[2 * S]);
  float2 t2 = cadd(v[S], v[3 * S]);
  float2 t3 = cmul_i(csub(v[S], v[3 * S]));
  v[0] = cadd(t0, t2);
  v[S] = cadd(t1, t3);
  v[2 * S] = csub(t0, t2);
  v[3 * S] = csub(t1, t3);
}

// Radix-P inverse DFT of v[0..P) in registers.  The result X[q] sits in
// v[dft_perm<P>(q)].
template <int P>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<1>(float2*) {}

template <>
__device__ __forceinline__ void dft<2>(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft<4>(float2* v) { dft4<1>(v); }

// 8 = 2 x 4: r = 4 r1 + r2, q = q1 + 2 q2.  Radix-2 over r1 for each r2,
// twiddle w8^(r2 q1), radix-4 over r2; X[q1 + 2 q2] lands in v[4 q1 + q2].
template <>
__device__ __forceinline__ void dft<8>(float2* v) {
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) {
    float2 a = v[r2], b = v[r2 + 4];
    v[r2] = cadd(a, b);
    v[r2 + 4] = csub(a, b);
  }
  v[5] = cmul(v[5], make_float2(RF_R2_2, RF_R2_2));
  v[6] = cmul_i(v[6]);
  v[7] = cmul(v[7], make_float2(-RF_R2_2, RF_R2_2));
  dft4<1>(v);
  dft4<1>(v + 4);
}

// 16 = 4 x 4: r = 4 r1 + r2, q = q1 + 4 q2.  Radix-4 over r1 for each r2
// (stride 4), twiddle w16^(r2 q1), radix-4 over r2; X[q1 + 4 q2] lands in
// v[4 q1 + q2].
template <>
__device__ __forceinline__ void dft<16>(float2* v) {
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4<4>(v + r2);
  // v[r2 + 4 q1] *= w16^(r2 q1)
  v[5] = cmul(v[5], make_float2(RF_C16_1, RF_S16_1));   // w^1
  v[9] = cmul(v[9], make_float2(RF_R2_2, RF_R2_2));     // w^2
  v[13] = cmul(v[13], make_float2(RF_S16_1, RF_C16_1)); // w^3
  v[6] = cmul(v[6], make_float2(RF_R2_2, RF_R2_2));     // w^2
  v[10] = cmul_i(v[10]);                                // w^4
  v[14] = cmul(v[14], make_float2(-RF_R2_2, RF_R2_2));  // w^6
  v[7] = cmul(v[7], make_float2(RF_S16_1, RF_C16_1));   // w^3
  v[11] = cmul(v[11], make_float2(-RF_R2_2, RF_R2_2));  // w^6
  v[15] = cmul(v[15], make_float2(-RF_C16_1, -RF_S16_1)); // w^9
  // Y[r2][q1] sits at v[r2 + 4 q1], so for fixed q1 the second radix-4 runs
  // over the contiguous v[4 q1 .. 4 q1 + 3].
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) dft4<1>(v + 4 * q1);
}

template <int P>
__host__ __device__ constexpr int dft_perm(int q) {
  return P == 16 ? 4 * (q & 3) + (q >> 2) : (P == 8 ? 4 * (q & 1) + (q >> 1) : q);
}

// Compile-time pass layout of a length-N transform.
template <int N>
struct FftShape {
  static_assert(N >= 16 && (N & (N - 1)) == 0, "N must be a power of two >= 16");
  static constexpr int T = N / 16;                     // threads per transform
  static constexpr int LOG2N = ilog2c(N);
  static constexpr int NFULL = LOG2N / 4;              // radix-16 passes
  static constexpr int RL = 1 << (LOG2N % 4);          // last radix (1 = none)
  static constexpr int NPASS = NFULL + (RL > 1 ? 1 : 0);
  static constexpr int LAST_P = RL > 1 ? RL : 16;
  static constexpr int LAST_NS = N / LAST_P;           // stride of the last pass
};

// Load phase of one pass: v[m P + r] = s[j + r N/P], j = t + m T.
template <int N, int P>
__device__ __forceinline__ void pass_load(float2 (&v)[16], const float2* s, int t) {
  constexpr int T = N / 16;
  constexpr int J = N / P;
#pragma unroll
  for (int m = 0; m < 16 / P; ++m) {
    const int j = t + m * T;
#pragma unroll
    for (int r = 0; r < P; ++r) v[m * P + r] = s[pad16(j + r * J)];
  }
}

// Twiddle + radix-P DFT of each butterfly held by the thread.
template <int N, int P>
__device__ __forceinline__ void pass_compute(float2 (&v)[16], const float2* __restrict__ tw, int t, int Ns) {
  constexpr int T = N / 16;
#pragma unroll
  for (int m = 0; m < 16 / P; ++m) {
    const int j = t + m * T;
    if (Ns > 1) {
      const int k = j & (Ns - 1);
      const int step = k * (N / (Ns * P));
#pragma unroll
      for (int r = 1; r < P; ++r) v[m * P + r] = cmul(v[m * P + r], __ldg(tw + step * r));
    }
    dft<P>(v + m * P);
  }
}

// Store phase of a non-final pass.
template <int N, int P>
__device__ __forceinline__ void pass_store(const float2 (&v)[16], float2* s, int t, int Ns) {
  constexpr int T = N / 16;
#pragma unroll
  for (int m = 0; m < 16 / P; ++m) {
    const int j = t + m * T;
    const int k = j & (Ns - 1);
    const int base = (j - k) * P + k;
#pragma unroll
    for (int q = 0; q < P; ++q) s[pad16(base + q * Ns)] = v[m * P + dft_perm<P>(q)];
  }
}

// Runs every pass but the last on the buffer `s` (in place), then loads and
// computes the last pass into registers.  On return the thread holds the
// outputs X[o] for o = t + m T + q (N / LAST_P) in v[m LAST_P + dft_perm(q)]
// (m < 16/LAST_P, q < LAST_P).  Every thread of the block must call this
// (it contains __syncthreads); `s` must be filled before the call and
// visible to all threads (a barrier before the call).
template <int N>
__device__ __forceinline__ void fft_inverse_to_regs(float2 (&v)[16], float2* s, const float2* __restrict__ tw, int t) {
  using S = FftShape<N>;
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < S::NPASS - 1; ++p) {
    pass_load<N, 16>(v, s, t);
    __syncthreads();
    pass_compute<N, 16>(v, tw, t, Ns);
    pass_store<N, 16>(v, s, t, Ns);
    __syncthreads();
    Ns *= 16;
  }
  pass_load<N, S::LAST_P>(v, s, t);
  pass_compute<N, S::LAST_P>(v, tw, t, Ns);
}

// Output index of register (m, q) after fft_inverse_to_regs.
template <int N>
__device__ __forceinline__ int fft_out_index(int t, int m, int q) {
  using S = FftShape<N>;
  return t + m * S::T + q * (N / S::LAST_P);
}

}  // namespace rf
