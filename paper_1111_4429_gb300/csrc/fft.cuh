// In-register mixed-radix FFT of one line per thread (radices 2, 3, 4, 5),
// the 1D transforms of the matrix elements' FFT form (the unnumbered
// equation after Eq. eqn_matrix_elem).
//
// The line length N is a compile-time constant, so every loop below unrolls
// completely and every array index is static: the line lives in registers.
// Algorithm: Stockham autosort, decimation in frequency.  A stage of radix r
// on a sub-length n (stride s, m = n/r) reads a_j = x[q + s(p + j m)],
// forms the r-point DFT b_k = sum_j a_j e^{S 2 pi i j k / r}, multiplies by
// the twiddle e^{S 2 pi i p k / n} and writes y[q + s(r p + k)]; the next
// stage runs on n/r with stride s r.  After the last stage the output is in
// natural order.  S = +1 computes sum_j x_j e^{+2 pi i j k/N} (unnormalized),
// the sign both transforms of the matrix-element path use.
//
// Twiddles e^{2 pi i t/N} come from a table of cos/sin values filled by the
// host in extended precision (upload_twiddles); inside a stage the table
// index is a compile-time constant, so the loads are constant-bank operands.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace bgw {

template <typename T> struct cpx_t;
template <> struct cpx_t<double> { using type = double2; };
template <> struct cpx_t<float> { using type = float2; };
template <typename T> using cpx = typename cpx_t<T>::type;

template <typename T> __device__ __forceinline__ cpx<T> mk(T x, T y) { cpx<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ cpx<T> add(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cpx<T> sub(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cpx<T> mul(cpx<T> a, cpx<T> b) {
  return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
template <typename T> __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
template <typename T> __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// i^S * a  for S = +-1
template <typename T, int S> __device__ __forceinline__ cpx<T> mul_i(cpx<T> a) {
  return S > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// Supported line lengths and their offsets in the twiddle table.
// Lengths 6, 9 and 15 serve only as the quarter-length sub-transforms of
// 24, 36 and 60 (fft_quarters).
__host__ __device__ constexpr int twiddle_offset(int n) {
  return n == 8 ? 0 : n == 10 ? 8 : n == 12 ? 18 : n == 16 ? 30 : n == 20 ? 46 : n == 24 ? 66
       : n == 30 ? 90 : n == 32 ? 120 : n == 36 ? 152 : n == 40 ? 188 : n == 48 ? 228
       : n == 50 ? 276 : n == 60 ? 326 : n == 64 ? 386 : n == 9 ? 450 : n == 15 ? 459 : n == 6 ? 474 : -1;
}
constexpr int kTwiddleTotal = 480;
constexpr int kSupportedN[] = {8, 10, 12, 16, 20, 24, 30, 32, 36, 40, 48, 50, 60, 64};

// First radix of a sub-length: 4 while it divides, then 2, 3, 5.
__host__ __device__ constexpr int first_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : 5;
}

// Mathematical constants of the radix-3 and radix-5 butterflies:
// sin(2pi/3) = sqrt(3)/2; cos(2pi/5) = (sqrt5-1)/4; cos(4pi/5) = -(sqrt5+1)/4;
// sin(2pi/5) = sqrt(10+2 sqrt5)/4; sin(4pi/5) = sqrt(10-2 sqrt5)/4.
#define BGW_S3 0.86602540378443864676
#define BGW_C51 0.30901699437494742410
#define BGW_C52 (-0.80901699437494742410)
#define BGW_S51 0.95105651629515357212
#define BGW_S52 0.58778525229247312917

template <typename T, int R, int S>
__device__ __forceinline__ void dft_small(const cpx<T> (&a)[R], cpx<T> (&b)[R]) {
  if constexpr (R == 2) {
    b[0] = add<T>(a[0], a[1]);
    b[1] = sub<T>(a[0], a[1]);
  } else if constexpr (R == 4) {
    cpx<T> s02 = add<T>(a[0], a[2]), d02 = sub<T>(a[0], a[2]);
    cpx<T> s13 = add<T>(a[1], a[3]), d13 = mul_i<T, S>(sub<T>(a[1], a[3]));
    b[0] = add<T>(s02, s13);
    b[2] = sub<T>(s02, s13);
    b[1] = add<T>(d02, d13);
    b[3] = sub<T>(d02, d13);
  } else if constexpr (R == 3) {
    const T c = T(-0.5), s = T(S) * T(BGW_S3);
    cpx<T> sum = add<T>(a[1], a[2]);
    cpx<T> dif = sub<T>(a[1], a[2]);
    b[0] = add<T>(a[0], sum);
    cpx<T> t = mk<T>(fma(c, sum.x, a[0].x), fma(c, sum.y, a[0].y));
    cpx<T> u = mul_i<T, 1>(scale<T>(dif, s));  // i s (a1 - a2)
    b[1] = add<T>(t, u);
    b[2] = sub<T>(t, u);
  } else {  // R == 5
    const T c1 = T(BGW_C51), c2 = T(BGW_C52);
    const T s1 = T(S) * T(BGW_S51), s2 = T(S) * T(BGW_S52);
    cpx<T> p14 = add<T>(a[1], a[4]), m14 = sub<T>(a[1], a[4]);
    cpx<T> p23 = add<T>(a[2], a[3]), m23 = sub<T>(a[2], a[3]);
    b[0] = add<T>(a[0], add<T>(p14, p23));
    cpx<T> t1 = mk<T>(fma(c1, p14.x, fma(c2, p23.x, a[0].x)), fma(c1, p14.y, fma(c2, p23.y, a[0].y)));
    cpx<T> t2 = mk<T>(fma(c2, p14.x, fma(c1, p23.x, a[0].x)), fma(c2, p14.y, fma(c1, p23.y, a[0].y)));
    cpx<T> u1 = mk<T>(fma(s1, m14.x, s2 * m23.x), fma(s1, m14.y, s2 * m23.y));
    cpx<T> u2 = mk<T>(fma(s2, m14.x, -s1 * m23.x), fma(s2, m14.y, -s1 * m23.y));
    u1 = mul_i<T, 1>(u1);
    u2 = mul_i<T, 1>(u2);
    b[1] = add<T>(t1, u1);
    b[4] = sub<T>(t1, u1);
    b[2] = add<T>(t2, u2);
    b[3] = sub<T>(t2, u2);
  }
}

// Twiddle tables: entry twiddle_offset(N) + t holds (cos, sin)(2 pi t / N).
// Each translation unit that includes this header owns its copy and fills it
// with upload_twiddles() once per device before launching its kernels.
static __constant__ double2 c_twiddle64[kTwiddleTotal];
static __constant__ float2 c_twiddle32[kTwiddleTotal];

template <typename T> __device__ __forceinline__ cpx<T> twiddle_entry(int i);
template <> __device__ __forceinline__ double2 twiddle_entry<double>(int i) { return c_twiddle64[i]; }
template <> __device__ __forceinline__ float2 twiddle_entry<float>(int i) { return c_twiddle32[i]; }

// e^{S 2 pi i t / N}
template <typename T, int N, int S>
__device__ __forceinline__ cpx<T> twiddle(int t) {
  static_assert(twiddle_offset(N) >= 0, "no twiddle table for this length");
  cpx<T> w = twiddle_entry<T>(twiddle_offset(N) + t);
  return mk<T>(w.x, T(S) * w.y);
}

template <typename T, int N, int n, int st, int S>
__device__ __forceinline__ void fft_stage(cpx<T> (&x)[N], cpx<T> (&y)[N]) {
  constexpr int r = first_radix(n);
  constexpr int m = n / r;
#pragma unroll
  for (int p = 0; p < m; ++p) {
#pragma unroll
    for (int q = 0; q < st; ++q) {
      cpx<T> a[r], b[r];
#pragma unroll
      for (int j = 0; j < r; ++j) a[j] = x[q + st * (p + j * m)];
      dft_small<T, r, S>(a, b);
      y[q + st * (r * p)] = b[0];
#pragma unroll
      for (int k = 1; k < r; ++k) {
        if constexpr (m == 1) {   // a single stage: no twiddles
          y[q + st * (r * p + k)] = b[k];
        } else if (p == 0) {
          y[q + st * (r * p + k)] = b[k];
        } else {
          y[q + st * (r * p + k)] = mul<T>(b[k], twiddle<T, N, S>((p * k * (N / n)) % N));
        }
      }
    }
  }
  if constexpr (m > 1) fft_stage<T, N, m, st * r, S>(y, x);
}

// Number of stages for sub-length n.
__host__ __device__ constexpr int fft_num_stages(int n) { return n <= 1 ? 0 : 1 + fft_num_stages(n / first_radix(n)); }

// In-place (in registers) FFT of one line: a_k <- sum_j a_j e^{S 2 pi i j k/N}.
template <typename T, int N, int S>
__device__ __forceinline__ void fft_line(cpx<T> (&a)[N]) {
  cpx<T> tmp[N];
  fft_stage<T, N, N, 1, S>(a, tmp);
  if constexpr (fft_num_stages(N) % 2 == 1) {
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = tmp[i];
  }
}

// The two outer quarters of a length-N transform (N = 4M), for lines whose
// kept outputs all lie in k < M or k >= 3M (a band |k| < M around zero):
//   lo[k2] = X[k2],  hi[k2] = X[k2 + 3M],  k2 = 0 .. M-1,
// with X[k] = sum_n x_n e^{+2 pi i n k / N} and x_n = load(n).  Decimation
// in time by 4: with n = n1 + 4 n2 and k = k2 + M k1,
//   X[k2 + M k1] = sum_{n1} e^{2 pi i n1 k1 / 4} e^{2 pi i n1 k2 / N} Y_{n1}[k2],
// Y_{n1} the length-M transform of x_{n1 + 4 n2}; k1 = 0 and 3 only, so the
// factors e^{2 pi i n1 k1 / 4} are 1 and (-i)^{n1}.  One sub-transform is
// live at a time: about 2.5 N registers instead of the 4 N of a full line,
// and half of the final radix-4 combinations are never formed.
template <typename T, int N, typename Load>
__device__ __forceinline__ void fft_quarters(Load load, cpx<T> (&lo)[N / 4], cpx<T> (&hi)[N / 4]) {
  constexpr int M = N / 4;
  static_assert(N % 4 == 0, "fft_quarters needs N divisible by 4");
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    cpx<T> y[M];
#pragma unroll
    for (int n2 = 0; n2 < M; ++n2) y[n2] = load(n1 + 4 * n2);
    fft_line<T, M, 1>(y);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) {
      const cpx<T> t = (n1 == 0 || k2 == 0) ? y[k2] : mul<T>(y[k2], twiddle<T, N, 1>(n1 * k2));
      const cpx<T> u = n1 == 0 ? t : n1 == 1 ? mk<T>(t.y, -t.x) : n1 == 2 ? mk<T>(-t.x, -t.y) : mk<T>(-t.y, t.x);
      if (n1 == 0) {
        lo[k2] = t;
        hi[k2] = u;
      } else {
        lo[k2] = add<T>(lo[k2], t);
        hi[k2] = add<T>(hi[k2], u);
      }
    }
  }
}

// Fill this translation unit's twiddle tables on the current device.  The
// values are computed on the host in long double and rounded once.
static inline cudaError_t upload_twiddles() {
  static const int ns[] = {8, 10, 12, 16, 20, 24, 30, 32, 36, 40, 48, 50, 60, 64, 9, 15, 6};
  double2 h64[kTwiddleTotal];
  float2 h32[kTwiddleTotal];
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int n : ns) {
    for (int t = 0; t < n; ++t) {
      long double ang = two_pi * (long double)t / (long double)n;
      double c = (double)cosl(ang), s = (double)sinl(ang);
      // exact values at the quarter turns
      if (4 * t == n) { c = 0.0; s = 1.0; }
      if (2 * t == n) { c = -1.0; s = 0.0; }
      if (4 * t == 3 * n) { c = 0.0; s = -1.0; }
      if (t == 0) { c = 1.0; s = 0.0; }
      h64[twiddle_offset(n) + t] = make_double2(c, s);
      h32[twiddle_offset(n) + t] = make_float2((float)c, (float)s);
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_twiddle64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_twiddle32, h32, sizeof(h32));
}

}  // namespace bgw
