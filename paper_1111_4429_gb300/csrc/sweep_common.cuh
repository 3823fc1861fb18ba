// Sweep of one diagonal block in shared memory (the diagonal step of both
// sweeps in epsinv.cu).
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

}  // namespace bgw
