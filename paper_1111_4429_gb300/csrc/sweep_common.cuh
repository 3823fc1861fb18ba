// Sweep of one diagonal block in shared memory (the diagonal step of both
// sweeps in epsinv.cu, which invert eps~ of Eq. epsilon).
//
// D (Hermitian positive definite, kb <= 32) is held as its lower triangle
// L[i][j], i >= j.  Pivot s: every lower element outside row/column s loses
// col_i conj(col_j) / d (col = column s of the full matrix, d = L[s][s]), the
// pivot column is divided by d and the pivot becomes -1/d.  After kb pivots
// L holds -D^-1.  The 528 lower elements are packed into 17 full warps: the
// FP64 pipe of the SM this runs on is the limit, and idle lanes of a warp
// still occupy it.
#pragma once
#include "runtime.h"

namespace bgw {

constexpr int kSwNB = 32;
constexpr int kDiagThreads = (kSwNB * (kSwNB + 1) / 2 + 31) / 32 * 32;  // 544

struct DiagSmem {
  double2 L[kSwNB][kSwNB + 1];
  double2 col[kSwNB];    // column s of the current matrix
  double2 ncolr[kSwNB];  // -conj(col) / d
  double rpiv;
};

// Lower element handled by thread t (triangular order); low = t owns one.
__device__ __forceinline__ void diag_thread_element(int t, int kb, int& i, int& j, bool& low) {
  i = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  j = t - i * (i + 1) / 2;
  low = t < kSwNB * (kSwNB + 1) / 2 && i < kb;
}

// Called by all kDiagThreads threads after L (lower) is loaded; ends with a
// __syncthreads().  A non-positive or non-finite pivot sets *status.
__device__ __forceinline__ void diag_sweep_smem(DiagSmem& sm, int kb, int t, int i, int j, bool low,
                                                int* status) {
  for (int s = 0; s < kb; ++s) {
    __syncthreads();
    if (t < kb) {
      const int r = t;
      double2 cv;
      if (r > s) {
        cv = sm.L[r][s];
      } else if (r < s) {
        const double2 x = sm.L[s][r];
        cv = make_double2(x.x, -x.y);
      } else {
        cv = sm.L[s][s];
      }
      sm.col[r] = cv;
      const double d = sm.L[s][s].x;
      double rr;
      if (!(d > 0.0) || !isfinite(d)) {
        if (r == 0) atomicExch(status, (int)kDevZeroPivot);
        rr = 0.0;
      } else {
        rr = 1.0 / d;
      }
      sm.ncolr[r] = make_double2(-cv.x * rr, cv.y * rr);
      if (r == s) sm.rpiv = rr;
    }
    __syncthreads();
    if (low) {
      if (i != s && j != s) {
        const double2 a = sm.col[i], c = sm.ncolr[j];
        double2 v = sm.L[i][j];
        v.x = fma(a.x, c.x, fma(-a.y, c.y, v.x));
        v.y = fma(a.x, c.y, fma(a.y, c.x, v.y));
        sm.L[i][j] = v;
      } else if (i == s && j == s) {
        sm.L[s][s] = make_double2(-sm.rpiv, 0.0);
      } else if (j == s) {  // i > s: A_is / d
        const double2 a = sm.col[i];
        sm.L[i][s] = make_double2(a.x * sm.rpiv, a.y * sm.rpiv);
      } else {              // i == s, j < s: A_sj / d = conj(col_j) / d
        const double2 c = sm.ncolr[j];
        sm.L[s][j] = make_double2(-c.x, -c.y);
      }
    }
  }
  __syncthreads();
}

// The same sweep with NT threads (NT < 528): each thread owns the lower
// elements t, t + NT, ...  Called by all NT threads after L (lower) is
// loaded; ends with a __syncthreads().
template <int NT>
__device__ __forceinline__ void diag_sweep_smem_n(DiagSmem& sm, int kb, int t, int* status) {
  constexpr int NE = (kSwNB * (kSwNB + 1) / 2 + NT - 1) / NT;
  int ei[NE], ej[NE];
  bool el[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) diag_thread_element(t + q * NT, kb, ei[q], ej[q], el[q]);
  for (int s = 0; s < kb; ++s) {
    __syncthreads();
    if (t < kb) {
      const int r = t;
      double2 cv;
      if (r > s) {
        cv = sm.L[r][s];
      } else if (r < s) {
        const double2 x = sm.L[s][r];
        cv = make_double2(x.x, -x.y);
      } else {
        cv = sm.L[s][s];
      }
      sm.col[r] = cv;
      const double d = sm.L[s][s].x;
      double rr;
      if (!(d > 0.0) || !isfinite(d)) {
        if (r == 0) atomicExch(status, (int)kDevZeroPivot);
        rr = 0.0;
      } else {
        rr = 1.0 / d;
      }
      sm.ncolr[r] = make_double2(-cv.x * rr, cv.y * rr);
      if (r == s) sm.rpiv = rr;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      if (!el[q]) continue;
      const int i = ei[q], j = ej[q];
      if (i != s && j != s) {
        const double2 a = sm.col[i], c = sm.ncolr[j];
        double2 v = sm.L[i][j];
        v.x = fma(a.x, c.x, fma(-a.y, c.y, v.x));
        v.y = fma(a.x, c.y, fma(a.y, c.x, v.y));
        sm.L[i][j] = v;
      } else if (i == s && j == s) {
        sm.L[s][s] = make_double2(-sm.rpiv, 0.0);
      } else if (j == s) {
        const double2 a = sm.col[i];
        sm.L[i][s] = make_double2(a.x * sm.rpiv, a.y * sm.rpiv);
      } else {
        const double2 c = sm.ncolr[j];
        sm.L[s][j] = make_double2(-c.x, -c.y);
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The same sweep in double-FP32 arithmetic (a value is hi + lo, two floats,
// about 2^-46 relative per operation) for updates whose target precision is
// far coarser than FP64 (the five-slice tensor-core update, near 2^-34).
// GB300's FP32 pipe issues 64 times the FP64 pipe's operations, so the
// double-FP32 sweep, about 12 FP32 operations per FP64 multiply-add, leaves
// the FP64 pipe, the sweep's limit, out of the step.  The error-free
// transformations are Knuth's two-sum, the fast two-sum for |a| >= |b| and
// the FMA product error.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 ff_fast(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_from(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double ff_to(float2 a) { return (double)a.x + (double)a.y; }

// (h + l) 2^ex as one double for the level sums of the update, built in the
// integer pipe without branches (the SM's FP64 pipe is the epilogue's
// bottleneck, and straight-line code lets the compiler interleave a thread's
// sixteen conversions).  h and l are finite and, where nonzero, far inside
// FP32's normal range (sums of level values, integers times 2^-8L, and their
// rounding errors: |h + l| >= 2^-90 or 0); |ex| < 900.  A two-sum first
// makes the pair non-overlapping: s = fl(h + l), |t| <= ulp(s) / 2, and
// |t| <= ulp(s) / 4 when s is a power of two and t lowers it.  The bits of
// s 2^ex as a double are s's own fields re-biased; t, counted in units of
// that double's last place (half that unit where t takes s below a power of
// two) and rounded, is added to the bit pattern as an integer: s + t stays
// inside the binade of s otherwise, and the pattern is monotonic in the
// magnitude.  The result is within half a unit in the last place of the
// exact (h + l) 2^ex plus the rounding of t to that unit.
__device__ __forceinline__ double ff2d_pair(float s, float t, int ex) {
  const unsigned us = __float_as_uint(s), ut = __float_as_uint(t);
  const unsigned k = (us << 1) != 0u ? (unsigned)(896 + ex) << 20 : 0u;
  const unsigned hi = (us & 0x80000000u) | (((us & 0x7FFFFFFFu) >> 3) + k);
  const unsigned lo = us << 29;
  const bool lowers = (int)(us ^ ut) < 0;   // t's sign differs from s's
  const int ge = (int)((us >> 23) & 0xFFu) - (int)((ut >> 23) & 0xFFu) - ((lowers && (us << 9) == 0u) ? 1 : 0);
  const unsigned mt = (ut & 0x7FFFFFu) | 0x800000u;
  const unsigned d = ge <= 29 ? mt << (29 - ge) : (((mt >> min(ge - 30, 31)) + 1u) >> 1);
  const long long b =
      (long long)(((unsigned long long)hi << 32) | lo) + (lowers ? -(long long)d : (long long)d);
  return __longlong_as_double(b);
}
// The rare FP64 forms, out of line: a short slow path inline would be
// predicated and its FP64 instructions issued on every call.
static __device__ __noinline__ double ff_to_slow(float hi, float lo) { return (double)hi + (double)lo; }
static __device__ __noinline__ float2 ff_from_slow(double x) { return ff_from(x); }

// hi + lo as a double for any finite pair: the integer form above where the
// sum lies in [2^-66, 2^123), else the FP64 pipe.
__device__ __forceinline__ double ff_to_any(float hi, float lo) {
  const float2 st = ff_two_sum(hi, lo);
  const unsigned es = (__float_as_uint(st.x) >> 23) & 0xFFu;
  if (es >= 61u && es <= 250u) return ff2d_pair(st.x, st.y, 0);
  return ff_to_slow(hi, lo);
}

// (hi + lo) 2^ex as a double for any finite pair and |ex| < 600: the integer
// form where the two-summed pair lies in [2^-66, 2^123), else the FP64 pipe.
static __device__ __noinline__ double ff_to_scaled_slow(float hi, float lo, int ex) {
  return ldexp((double)hi + (double)lo, ex);
}
__device__ __forceinline__ double ff_to_scaled_any(float hi, float lo, int ex) {
  const float2 st = ff_two_sum(hi, lo);
  const unsigned es = (__float_as_uint(st.x) >> 23) & 0xFFu;
  if (es >= 61u && es <= 250u) return ff2d_pair(st.x, st.y, ex);
  return ff_to_scaled_slow(hi, lo, ex);
}

// ff_from(x) (hi = x rounded to FP32, lo = the remainder rounded) from x's
// fields in the integer pipe for 2^-74 <= |x| < 2^126 (FP64 pipe otherwise):
// hi is x's 53-bit mantissa rounded to 24 bits (half to even, the carry runs
// into the exponent), lo the integer remainder d (|d| <= 2^28) converted and
// scaled by x's last place, exactly as the FP64 form rounds it.
__device__ __forceinline__ float2 ff_from_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FFull);
  if (E < 949 || E > 1149) return ff_from_slow(x);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned q = (unsigned)(m >> 29);
  const unsigned r = (unsigned)(m & 0x1FFFFFFFull);
  const unsigned up = (r > 0x10000000u || (r == 0x10000000u && (q & 1u))) ? 1u : 0u;
  q += up;
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sgn | (((unsigned)(E - 897) << 23) + q));
  const float lo = __int2float_rn((int)r - (int)(up << 29)) * __uint_as_float((unsigned)(E - 948) << 23);
  return make_float2(hi, sgn ? -lo : lo);
}

// -x by the sign bit (no FP64 instruction)
__device__ __forceinline__ double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a b
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return ff_fast(p, e);
}
// 1 / d for d > 0: the FP32 reciprocal and one Newton step in double FP32
__device__ __forceinline__ float2 ff_rcp(float2 d) {
  const float r0 = __frcp_rn(d.x);
  const float2 t = ff_mul(d, make_float2(r0, 0.f));                     // d r0 = 1 - err
  const float2 e = ff_two_sum(1.f, -t.x);
  const float err = __fsub_rn(__fadd_rn(e.x, e.y), t.y);               // 1 - d r0 (small)
  return ff_fast(r0, __fmul_rn(r0, err));
}

// v + a1 b1 + a2 b2 with both products as exact pairs and the high words
// two-summed; the result is left unnormalized (hi, lo): lo gathers the
// error terms, so hi + lo carries the sum to about 2^-43 of the largest
// term, and consumers that need a leading word close to the value (the
// pivot's reciprocal) renormalize it first.
__device__ __forceinline__ float2 ff_dot2(float2 v, float2 a1, float2 b1, float2 a2, float2 b2) {
  const float p1 = __fmul_rn(a1.x, b1.x);
  float e1 = __fmaf_rn(a1.x, b1.x, -p1);
  e1 = __fmaf_rn(a1.x, b1.y, e1);
  e1 = __fmaf_rn(a1.y, b1.x, e1);
  const float p2 = __fmul_rn(a2.x, b2.x);
  float e2 = __fmaf_rn(a2.x, b2.x, -p2);
  e2 = __fmaf_rn(a2.x, b2.y, e2);
  e2 = __fmaf_rn(a2.y, b2.x, e2);
  const float2 s1 = ff_two_sum(v.x, p1);
  const float2 s2 = ff_two_sum(s1.x, p2);
  return make_float2(s2.x, __fadd_rn(__fadd_rn(v.y, __fadd_rn(e1, e2)), __fadd_rn(s1.y, s2.y)));
}

// Double-FP32 form of diag_sweep_smem_n with one barrier per pivot: the
// matrix ping-pongs between sm.L (as float4: re hi, re lo, im hi, im lo) and
// the scratch buffer (32 x 33 float4, 16.9 KiB of shared memory the caller
// does not need meanwhile).  Pivot s reads buffer s & 1 and writes every
// lower element into the other; each thread forms the column entries it
// needs itself, and the thread that writes the next pivot element forms its
// reciprocal, so no step has a serial phase.  Converts sm.L from and back to
// double2, so callers read and write sm.L as double2 before and after.
// Called by all NT threads after L (lower) is loaded; ends with a
// __syncthreads().  A non-positive or non-finite pivot sets *status.
template <int NT>
__device__ __forceinline__ void diag_sweep_ff_n(DiagSmem& sm, float4* scratch, int kb, int t, int* status,
                                                float4* dff = nullptr) {
  constexpr int NE = (kSwNB * (kSwNB + 1) / 2 + NT - 1) / NT;
  typedef float4 Row[kSwNB + 1];
  Row* const B0 = reinterpret_cast<Row*>(sm.L);
  Row* const B1 = reinterpret_cast<Row*>(scratch);
  float2* rps = reinterpret_cast<float2*>(sm.col);   // reciprocal of the pivot of step s in rps[s & 1]
  int ei[NE], ej[NE];
  bool el[NE];
  __syncthreads();   // the caller's loads of L are visible before the conversion
  auto rcp_checked = [&](float2 d) {
    d = ff_two_sum(d.x, d.y);   // leading word first (the pair may be unnormalized)
    if (!(d.x > 0.f) || !isfinite(d.x)) {
      atomicExch(status, (int)kDevZeroPivot);
      return make_float2(0.f, 0.f);
    }
    return ff_rcp(d);
  };
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    diag_thread_element(t + q * NT, kb, ei[q], ej[q], el[q]);
    if (el[q]) {
      const double2 x = sm.L[ei[q]][ej[q]];
      const float2 re = ff_from_int(x.x), im = ff_from_int(x.y);
      B0[ei[q]][ej[q]] = make_float4(re.x, re.y, im.x, im.y);
      if (ei[q] == 0 && ej[q] == 0) rps[0] = rcp_checked(re);
    }
  }
  for (int s = 0; s < kb; ++s) {
    __syncthreads();
    Row* const R = (s & 1) ? B1 : B0;   // selects, not an indexed array (kept out of local memory)
    Row* const W = (s & 1) ? B0 : B1;
    const float2 rp = rps[s & 1];
    // column s of the full (Hermitian) matrix at index x: R[x][s] below the
    // pivot, conj(R[s][x]) above it
    auto col = [&](int x) {
      const bool up = x < s;
      const float4 v = up ? R[s][x] : R[x][s];
      const float g = up ? -1.f : 1.f;
      return make_float4(v.x, v.y, g * v.z, g * v.w);
    };
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      if (!el[q]) continue;
      const int i = ei[q], j = ej[q];
      float4 out;
      if (i != s && j != s) {
        const float4 a4 = col(i), c4 = col(j), v4 = R[i][j];
        // ncolr_j = -conj(col_j) / d
        const float2 cr = ff_mul(ff_neg(make_float2(c4.x, c4.y)), rp), ci = ff_mul(make_float2(c4.z, c4.w), rp);
        const float2 ar = make_float2(a4.x, a4.y), ai = make_float2(a4.z, a4.w);
        const float2 vr = ff_dot2(make_float2(v4.x, v4.y), ar, cr, ff_neg(ai), ci);   // + a_r c_r - a_i c_i
        const float2 vi = ff_dot2(make_float2(v4.z, v4.w), ar, ci, ai, cr);           // + a_r c_i + a_i c_r
        out = make_float4(vr.x, vr.y, vi.x, vi.y);
        if (i == s + 1 && j == s + 1) rps[(s + 1) & 1] = rcp_checked(vr);
      } else if (i == s && j == s) {
        out = make_float4(-rp.x, -rp.y, 0.f, 0.f);
      } else if (j == s) {  // i > s: A_is / d
        const float4 a4 = R[i][s];
        const float2 xr = ff_mul(make_float2(a4.x, a4.y), rp), xi = ff_mul(make_float2(a4.z, a4.w), rp);
        out = make_float4(xr.x, xr.y, xi.x, xi.y);
      } else {              // i == s, j < s: conj(col_j) / d
        const float4 c4 = R[s][j];   // col_j = conj(R[s][j]); conj(col_j) = R[s][j]
        const float2 xr = ff_mul(make_float2(c4.x, c4.y), rp), xi = ff_mul(make_float2(c4.z, c4.w), rp);
        out = make_float4(xr.x, xr.y, xi.x, xi.y);
      }
      W[i][j] = out;
    }
  }
  __syncthreads();
  Row* const F = (kb & 1) ? B1 : B0;
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    if (!el[q]) continue;
    const float4 x = F[ei[q]][ej[q]];
    sm.L[ei[q]][ej[q]] = make_double2(ff_to_any(x.x, x.y), ff_to_any(x.z, x.w));
    if (dff) {
      // -D^-1 as normalized double-FP32 pairs, both triangles (ld kSwNB):
      // the next panel product reads them without FP64 conversions
      const float2 re = ff_two_sum(x.x, x.y), im = ff_two_sum(x.z, x.w);
      const int i = ei[q], j = ej[q];
      dff[i * kSwNB + j] = make_float4(-re.x, -re.y, -im.x, -im.y);
      if (i != j) dff[j * kSwNB + i] = make_float4(-re.x, -re.y, im.x, im.y);
    }
  }
  __syncthreads();
}

}  // namespace bgw
