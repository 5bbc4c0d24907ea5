// rf_fft.cuh -- shared-memory Stockham FFT building blocks for the imaging
// kernels (the 2D inverse FFT of the dirty image, Sec. 3.1 / Sec. 3.2: the
// 2D FFT is the most demanding stage of the search).
//
// A length-N transform (N a power of two, 16..8192) is done by T = N/E
// threads that each hold E = 32 complex values (E = 16 for N = 16; a kernel
// may ask for E = 16 at any N, whose passes then all take their twiddles by
// products of table entries, see twiddle_mul).  Each
// pass is a radix-P Stockham autosort step: thread t loads the P inputs
// j + r (N/P) of each of its E/P butterflies j, multiplies them by
// exp(+2 pi i k r / (Ns P)) with k = j mod Ns, does a radix-P inverse DFT in
// registers and stores output q at (j / Ns) Ns P + k + q Ns.  All passes are
// radix E except the last, whose radix is N / E^floor(log_E N) when N is not
// a power of E.  For N = 1024 that is two radix-32 passes.  The data stay in
// one padded shared-memory buffer per transform (a spare slot every 32
// values keeps the strided first-pass stores free of bank conflicts); a
// barrier separates the loads and stores of a pass so the transform is in
// place.  Transforms of at most 32 threads synchronise with __syncwarp, wider
// ones with a named barrier of their own.  Sign +1 (inverse DFT), no 1/N.
//
// Twiddles: the second pass (Ns = E) reads its P - 1 twiddles per butterfly
// from a table of exactly those values that follows the N table entries
// (FP64-computed, rounded to FP32).  A third pass (N >= 2048, radix 2..8)
// builds the powers w^(s r) from the table values w^s, w^2s, w^4s by one
// complex product each, at most four roundings from the table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rf {

// Complex add and subtract as one packed FP32-pair instruction each
// (add/sub.rn.f32x2: both components rounded to nearest, as two scalar ops).
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
}
// Packed FP32-pair multiply and fused multiply-add (rounded to nearest).
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a times the constant twiddle (c, s) as two packed instructions:
// (a.x, a.x) (c, s) + (a.y, a.y) (-s, c).
__device__ __forceinline__ float2 cmul_const(float2 a, float c, float s) {
  return f2_fma(make_float2(a.y, a.y), make_float2(-s, c), f2_mul(make_float2(a.x, a.x), make_float2(c, s)));
}
// t + i u and t - i u as one packed FMA each on the swapped pair (u.y, u.x).
__device__ __forceinline__ float2 c_add_iu(float2 t, float2 u) {
  return f2_fma(make_float2(u.y, u.x), make_float2(-1.f, 1.f), t);
}
__device__ __forceinline__ float2 c_sub_iu(float2 t, float2 u) {
  return f2_fma(make_float2(u.y, u.x), make_float2(1.f, -1.f), t);
}
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }  // i * a

// cos and sin of 2 pi k / 32, k = 1..7 (the others follow by symmetry).
#define RF_C32_1 0.98078528040323044913f
#define RF_S32_1 0.19509032201612826785f
#define RF_C32_2 0.92387953251128675613f
#define RF_S32_2 0.38268343236508977173f
#define RF_C32_3 0.83146961230254523708f
#define RF_S32_3 0.55557023301960222474f
#define RF_R2_2 0.70710678118654752440f

// cos(pi k / 32), k = 0 .. 16.
__host__ __device__ constexpr float cos_pi32(int k) {
  return k == 0 ? 1.f : k == 1 ? 0.99518472667219688624f : k == 2 ? 0.98078528040323044913f
       : k == 3 ? 0.95694033573220886494f : k == 4 ? 0.92387953251128675613f : k == 5 ? 0.88192126434835502971f
       : k == 6 ? 0.83146961230254523708f : k == 7 ? 0.77301045336273696081f : k == 8 ? 0.70710678118654752440f
       : k == 9 ? 0.63439328416364549822f : k == 10 ? 0.55557023301960222474f : k == 11 ? 0.47139673682599764856f
       : k == 12 ? 0.38268343236508977173f : k == 13 ? 0.29028467725446236764f : k == 14 ? 0.19509032201612826785f
       : k == 15 ? 0.09801714032956060199f : 0.f;
}
// exp(+2 pi i r / 64) = exp(+i pi r / 32), r = 0 .. 31.
__host__ __device__ constexpr float cos_r64(int r) { return r <= 16 ? cos_pi32(r) : -cos_pi32(32 - r); }
__host__ __device__ constexpr float sin_r64(int r) { return cos_pi32(r < 16 ? 16 - r : r - 16); }

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

// Padded shared-memory index: one spare slot every 32 complex values.
__host__ __device__ __forceinline__ constexpr int padx(int i) { return i + (i >> 5); }

// Two styles of the same arithmetic, picked per kernel at compile time
// (PK): with PK the products by constant twiddles are packed FP32-pair
// instructions, cmul_const, and the radix-4 outputs t1 +- i u take one packed
// FMA each on the swapped pair (u.y, u.x); without it both are scalar.  The
// packed style issues fewer instructions but needs more registers: it is
// faster in the column pass and slower in the row pass.
template <bool PK>
__device__ __forceinline__ float2 cmul_c(float2 a, float c, float s) {
  if constexpr (PK) return cmul_const(a, c, s);
  else return cmul(a, make_float2(c, s));
}

// In-register inverse radix-4 on v[0], v[S], v[2S], v[3S] (natural order out).
template <int S, bool PK>
__device__ __forceinline__ void dft4(float2* v) {
  const float2 t0 = cadd(v[0], v[2 * S]);
  const float2 t1 = csub(v[0], v[2 * S]);
  const float2 t2 = cadd(v[S], v[3 * S]);
  const float2 u = csub(v[S], v[3 * S]);
  v[0] = cadd(t0, t2);
  v[2 * S] = csub(t0, t2);
  if constexpr (PK) {
    v[S] = c_add_iu(t1, u);
    v[3 * S] = c_sub_iu(t1, u);
  } else {
    v[S] = make_float2(t1.x - u.y, t1.y + u.x);
    v[3 * S] = make_float2(t1.x + u.y, t1.y - u.x);
  }
}

// Radix-P inverse DFT of v[0..P) in registers; X[q] ends in v[dft_perm<P>(q)].
template <int P, bool PK>
struct DftK;

template <bool PK>
struct DftK<1, PK> {
  __device__ static __forceinline__ void run(float2*) {}
};

template <bool PK>
struct DftK<2, PK> {
  __device__ static __forceinline__ void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool PK>
struct DftK<4, PK> {
  __device__ static __forceinline__ void run(float2* v) { dft4<1, PK>(v); }
};

// 8 = 2 x 4: r = 4 r1 + r2, q = q1 + 2 q2.  Radix-2 over r1 for each r2,
// twiddle w8^(r2 q1), radix-4 over r2; X[q1 + 2 q2] lands in v[4 q1 + q2].
template <bool PK>
struct DftK<8, PK> {
  __device__ static __forceinline__ void run(float2* v) {
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) {
      const float2 a = v[r2], b = v[r2 + 4];
      v[r2] = cadd(a, b);
      v[r2 + 4] = csub(a, b);
    }
    v[5] = cmul_c<PK>(v[5], RF_R2_2, RF_R2_2);
    v[6] = cmul_i(v[6]);
    v[7] = cmul_c<PK>(v[7], -RF_R2_2, RF_R2_2);
    dft4<1, PK>(v);
    dft4<1, PK>(v + 4);
  }
};

// 16 = 4 x 4: r = 4 r1 + r2, q = q1 + 4 q2.  Radix-4 over r1 for each r2
// (stride 4) leaves Y[r2][q1] at v[r2 + 4 q1]; twiddle w16^(r2 q1); radix-4
// over r2, i.e. over the contiguous v[4 q1 .. 4 q1 + 3]; X[q1 + 4 q2] lands
// in v[4 q1 + q2].
template <bool PK>
struct DftK<16, PK> {
  __device__ static __forceinline__ void run(float2* v) {
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) dft4<4, PK>(v + r2);
    v[5] = cmul_c<PK>(v[5], RF_C32_2, RF_S32_2);      // w16^1
    v[9] = cmul_c<PK>(v[9], RF_R2_2, RF_R2_2);        // w16^2
    v[13] = cmul_c<PK>(v[13], RF_S32_2, RF_C32_2);    // w16^3
    v[6] = cmul_c<PK>(v[6], RF_R2_2, RF_R2_2);        // w16^2
    v[10] = cmul_i(v[10]);                            // w16^4
    v[14] = cmul_c<PK>(v[14], -RF_R2_2, RF_R2_2);     // w16^6
    v[7] = cmul_c<PK>(v[7], RF_S32_2, RF_C32_2);      // w16^3
    v[11] = cmul_c<PK>(v[11], -RF_R2_2, RF_R2_2);     // w16^6
    v[15] = cmul_c<PK>(v[15], -RF_C32_2, -RF_S32_2);  // w16^9
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) dft4<1, PK>(v + 4 * q1);
  }
};

// 32 = 2 x 16: r = 16 r1 + r2, q = q1 + 2 q2.  Radix-2 over r1 for each r2
// leaves Y[r2][q1] at v[r2 + 16 q1]; twiddle w32^(r2 q1); radix-16 over the
// contiguous halves; X[q1 + 2 q2] lands in v[16 q1 + dft_perm<16>(q2)].
template <bool PK>
struct DftK<32, PK> {
  __device__ static __forceinline__ void run(float2* v) {
#pragma unroll
    for (int r2 = 0; r2 < 16; ++r2) {
      const float2 a = v[r2], b = v[r2 + 16];
      v[r2] = cadd(a, b);
      v[r2 + 16] = csub(a, b);
    }
    // w32^r for r = 1..15
    v[17] = cmul_c<PK>(v[17], RF_C32_1, RF_S32_1);
    v[18] = cmul_c<PK>(v[18], RF_C32_2, RF_S32_2);
    v[19] = cmul_c<PK>(v[19], RF_C32_3, RF_S32_3);
    v[20] = cmul_c<PK>(v[20], RF_R2_2, RF_R2_2);
    v[21] = cmul_c<PK>(v[21], RF_S32_3, RF_C32_3);
    v[22] = cmul_c<PK>(v[22], RF_S32_2, RF_C32_2);
    v[23] = cmul_c<PK>(v[23], RF_S32_1, RF_C32_1);
    v[24] = cmul_i(v[24]);
    v[25] = cmul_c<PK>(v[25], -RF_S32_1, RF_C32_1);
    v[26] = cmul_c<PK>(v[26], -RF_S32_2, RF_C32_2);
    v[27] = cmul_c<PK>(v[27], -RF_S32_3, RF_C32_3);
    v[28] = cmul_c<PK>(v[28], -RF_R2_2, RF_R2_2);
    v[29] = cmul_c<PK>(v[29], -RF_C32_3, RF_S32_3);
    v[30] = cmul_c<PK>(v[30], -RF_C32_2, RF_S32_2);
    v[31] = cmul_c<PK>(v[31], -RF_C32_1, RF_S32_1);
    DftK<16, PK>::run(v);
    DftK<16, PK>::run(v + 16);
  }
};

template <int P, bool PK = false>
__device__ __forceinline__ void dft(float2* v) {
  DftK<P, PK>::run(v);
}

template <int P>
__host__ __device__ constexpr int dft_perm(int q) {
  return P == 32 ? 16 * (q & 1) + (4 * ((q >> 1) & 3) + (q >> 3))
                 : (P == 16 ? 4 * (q & 3) + (q >> 2) : (P == 8 ? 4 * (q & 1) + (q >> 1) : q));
}

// Compile-time pass layout of a length-N transform with EV complex values
// per thread (32 by default; 16 below N = 32).
template <int N, int EV = (N >= 32 ? 32 : 16)>
struct FftShape {
  static_assert(N >= 16 && N <= 8192 && (N & (N - 1)) == 0, "N must be a power of two in [16, 8192]");
  static_assert(EV == 16 || EV == 32, "16 or 32 values per thread");
  static constexpr int E = EV;                          // complex values per thread
  static constexpr int T = N / E;                       // threads per transform
  static constexpr int LOG2N = ilog2c(N);
  static constexpr int LOG2E = ilog2c(E);
  static constexpr int NFULL = LOG2N / LOG2E;           // radix-E passes
  static constexpr int RL = 1 << (LOG2N % LOG2E);       // last radix (1 = none)
  static constexpr int NPASS = NFULL + (RL > 1 ? 1 : 0);
  static constexpr int LAST_P = RL > 1 ? RL : E;
  static constexpr int P2 = NPASS == 1 ? 0 : (NPASS == 2 ? LAST_P : E);  // radix of the second pass
  static constexpr int STRIDE = N + N / 32 + 2;         // float2 per transform buffer
  static_assert(NPASS <= 3, "at most three passes");
};

template <int N>
__host__ __device__ constexpr int fft_stride() { return FftShape<N>::STRIDE; }

// Barrier among the T threads of transform `xf` of a block.
template <int T>
__device__ __forceinline__ void fft_sync(int xf) {
  if (T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + xf), "r"(T) : "memory");
  }
}

// Twiddles w^(s r), r = 1 .. P-1, from the table entries w^(s 2^i): one
// complex product per non-power-of-two r (at most four roundings from the
// table); fewer loads and registers than reading every power.
template <int N, int P>
__device__ __forceinline__ void twiddle_mul(float2* v, const float2* __restrict__ tw, int s) {
  float2 W[P];
#pragma unroll
  for (int p2 = 1; p2 < P; p2 <<= 1) W[p2] = __ldg(tw + s * p2);
#pragma unroll
  for (int r = 3; r < P; ++r) {
    const int lb = r & -r;
    if (r != lb) W[r] = cmul(W[r - lb], W[lb]);
  }
#pragma unroll
  for (int r = 1; r < P; ++r) v[r] = cmul(v[r], W[r]);
}

// Load phase of one pass: v[m P + r] = s[j + r N/P], j = t + m T.  When
// m T and r N/P are multiples of 32 (N >= 1024), padx(t + m T + r N/P) =
// padx(t) + padx(m T) + padx(r N/P): one index per thread, the rest constant.
template <int N, int P, int EV = FftShape<N>::E>
__device__ __forceinline__ void pass_load(float2 (&v)[EV], const float2* s, int t) {
  constexpr int E = FftShape<N, EV>::E;
  constexpr int T = FftShape<N, EV>::T;
  constexpr int J = N / P;
  if constexpr (T % 32 == 0 && J % 32 == 0) {
    const float2* st = s + padx(t);
#pragma unroll
    for (int m = 0; m < E / P; ++m)
#pragma unroll
      for (int r = 0; r < P; ++r) v[m * P + r] = st[padx(m * T) + padx(r * J)];
  } else {
#pragma unroll
    for (int m = 0; m < E / P; ++m) {
      const int j = t + m * T;
#pragma unroll
      for (int r = 0; r < P; ++r) v[m * P + r] = s[padx(j + r * J)];
    }
  }
}

// Twiddle + radix-P DFT of each butterfly held by the thread.
template <int N, int P, bool PK = false, int EV = FftShape<N>::E>
__device__ __forceinline__ void pass_compute(float2 (&v)[EV], const float2* __restrict__ tw, int t, int Ns) {
  constexpr int E = FftShape<N, EV>::E;
  constexpr int T = FftShape<N, EV>::T;
#pragma unroll
  for (int m = 0; m < E / P; ++m) {
    const int j = t + m * T;
    if (Ns > 1) {
      const int k = j & (Ns - 1);
      twiddle_mul<N, P>(v + m * P, tw, k * (N / (Ns * P)));
    }
    dft<P, PK>(v + m * P);
  }
}

// Twiddle + radix-P DFT of the second pass (Ns = E = 32): butterfly j takes
// exp(+2 pi i k r / (32 P)), k = j mod 32, from the pair table
// tw2[(r / 2) 64 + 2 k + (r mod 2)]: one 16-byte load per pair of r,
// consecutive across the transform's threads.
template <int N, int P, bool PK = false>
__device__ __forceinline__ void pass2_compute(float2 (&v)[FftShape<N>::E], const float2* __restrict__ tw2, int t) {
  constexpr int E = FftShape<N>::E;
  constexpr int T = FftShape<N>::T;
  static_assert(E == 32 && P % 2 == 0, "pair table of a radix-32 second pass");
#pragma unroll
  for (int m = 0; m < E / P; ++m) {
    const int k = (t + m * T) & (E - 1);
    const float4* w4 = reinterpret_cast<const float4*>(tw2) + k;
#pragma unroll
    for (int rp = 0; rp < P / 2; ++rp) {
      const float4 w = __ldg(w4 + rp * E);
      if (rp > 0) v[m * P + 2 * rp] = cmul(v[m * P + 2 * rp], make_float2(w.x, w.y));
      v[m * P + 2 * rp + 1] = cmul(v[m * P + 2 * rp + 1], make_float2(w.z, w.w));
    }
    dft<P, PK>(v + m * P);
  }
}

// Store phase of a non-final pass.  Output q of butterfly j goes to
// base + q Ns.  When q Ns is a multiple of 32, or Ns = 1 and base is (P = 32),
// padx(base + q Ns) = padx(base) + padx(q Ns) with the second term constant.
template <int N, int P, int EV = FftShape<N>::E>
__device__ __forceinline__ void pass_store(const float2 (&v)[EV], float2* s, int t, int Ns) {
  constexpr int E = FftShape<N, EV>::E;
  constexpr int T = FftShape<N, EV>::T;
#pragma unroll
  for (int m = 0; m < E / P; ++m) {
    const int j = t + m * T;
    const int k = j & (Ns - 1);
    const int base = (j - k) * P + k;
    if (Ns % 32 == 0 || (Ns == 1 && P % 32 == 0)) {
      float2* sb = s + padx(base);
#pragma unroll
      for (int q = 0; q < P; ++q) sb[padx(q * Ns)] = v[m * P + dft_perm<P>(q)];
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) s[padx(base + q * Ns)] = v[m * P + dft_perm<P>(q)];
    }
  }
}

// max(a, b, c) in one instruction (a NaN operand is ignored, as by fmaxf).
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Runs the passes after the first-pass load.  On entry v holds the first
// pass's inputs (v[r] = x[t + r T]); `tw` is the transform's twiddle table
// (fft_twiddle_len(N) entries: the N powers of w, then the second pass's
// table); on return the thread holds the outputs
// X[o] for o = t + m T + q (N / LAST_P) in v[m LAST_P + dft_perm(q)].
template <int N, bool PK = false, int EV = FftShape<N>::E>
__device__ __forceinline__ void fft_inverse_from_regs(float2 (&v)[EV], float2* s, const float2* __restrict__ tw,
                                                      int t, int xf) {
  using S = FftShape<N, EV>;
  if constexpr (S::NPASS == 1) {
    pass_compute<N, S::LAST_P, PK>(v, tw, t, 1);
  } else if constexpr (S::E != 32) {
    // 16 values a thread: every pass's twiddles from the length-N table
    // (products of w^(s 2^i), see twiddle_mul)
    pass_compute<N, S::E, PK, EV>(v, tw, t, 1);
    pass_store<N, S::E, EV>(v, s, t, 1);
    fft_sync<S::T>(xf);
    if constexpr (S::NPASS == 2) {
      pass_load<N, S::LAST_P, EV>(v, s, t);
      pass_compute<N, S::LAST_P, PK, EV>(v, tw, t, S::E);
    } else {
      pass_load<N, S::E, EV>(v, s, t);
      fft_sync<S::T>(xf);
      pass_compute<N, S::E, PK, EV>(v, tw, t, S::E);
      pass_store<N, S::E, EV>(v, s, t, S::E);
      fft_sync<S::T>(xf);
      pass_load<N, S::LAST_P, EV>(v, s, t);
      pass_compute<N, S::LAST_P, PK, EV>(v, tw, t, S::E * S::E);
    }
  } else {
    pass_compute<N, S::E, PK>(v, tw, t, 1);
    pass_store<N, S::E>(v, s, t, 1);
    fft_sync<S::T>(xf);
    pass_load<N, S::P2>(v, s, t);
    if constexpr (S::NPASS == 2) {
      pass2_compute<N, S::P2, PK>(v, tw + N, t);
    } else {
      fft_sync<S::T>(xf);
      pass2_compute<N, S::E, PK>(v, tw + N, t);
      pass_store<N, S::E>(v, s, t, S::E);
      fft_sync<S::T>(xf);
      pass_load<N, S::LAST_P>(v, s, t);
      pass_compute<N, S::LAST_P, PK>(v, tw, t, S::E * S::E);
    }
  }
}

// The same with the first-pass inputs read from the padded buffer `s`
// (filled and made visible to the transform's threads by the caller).
template <int N, bool PK = false, int EV = FftShape<N>::E>
__device__ __forceinline__ void fft_inverse_to_regs(float2 (&v)[EV], float2* s, const float2* __restrict__ tw,
                                                    int t, int xf) {
  using S = FftShape<N, EV>;
  constexpr int P0 = S::NPASS == 1 ? S::LAST_P : S::E;
  pass_load<N, P0, EV>(v, s, t);
  if (S::NPASS > 1) fft_sync<S::T>(xf);  // in place: all loads before the first store
  fft_inverse_from_regs<N, PK, EV>(v, s, tw, t, xf);
}

// Output index of register (m, q) after the last pass.
template <int N, int EV = FftShape<N>::E>
__device__ __forceinline__ int fft_out_index(int t, int m, int q) {
  using S = FftShape<N, EV>;
  return t + m * S::T + q * (N / S::LAST_P);
}

}  // namespace rf
