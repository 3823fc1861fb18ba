// Symmetrized dielectric matrix and its inverse (paper, Eqs. epsilon and
// untruncated_bare_coulomb with the symmetric Coulomb form), FP64 throughout:
//   sv_G       = sqrt(4 pi) / |(q + G) B|             (= v(q+G)^{1/2})
//   eps~[G][G'] = delta_GG' - sv_G chi[G][G'] sv_G'
//   epsinv      = eps~^-1 by a Hermitian blocked sweep (bgw_epsinv) or by
//                 blocked Gauss-Jordan elimination (the allocation-free
//                 entry point).
//
// Gauss-Jordan step on the column block k (width kb, rows/cols K = k0..k0+kb):
//   D^-1 of the diagonal block (one CTA, elimination in shared memory)
//   R[r][j] = (D^-1 A_K,:)[r][j] for j outside K,  R[r][K] = D^-1
//   C[i][s] = A[i][k0+s]                (copy of the column panel)
//   A[i][j] <- R[i-k0][j]                                         i in K
//   A[i][j] <- (j in K ? 0 : A[i][j]) - sum_s C[i][s] R[s][j]     otherwise
// After the last block A holds eps~^-1.  No pivoting: eps~ = I - v^1/2 chi
// v^1/2 is Hermitian positive definite (chi <= 0), for which elimination
// without pivoting is backward stable; a zero or non-finite pivot is
// recorded in the device status word.
#include <cuda.h>

#include <cmath>
#include <memory>
#include <vector>

#include "runtime.h"
#include "sweep_common.cuh"

namespace bgw {

namespace {
constexpr int NB = 32;   // Gauss-Jordan block width
constexpr int TU = 64;   // update tile edge
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
}  // namespace

// Cell, q and Coulomb model as one by-value kernel argument.
struct CoulombArgs {
  double b[9];  // bvec rows
  double q[3];
  double cut;   // r_c or z_c
  int model;    // BGW_COULOMB_*
};

CoulombArgs coulomb_args(const bgw_cell* cell) {
  CoulombArgs a;
  for (int i = 0; i < 9; ++i) a.b[i] = (&cell->bvec[0][0])[i];
  for (int i = 0; i < 3; ++i) a.q[i] = cell->q_frac[i];
  a.cut = cell->coulomb_cut;
  a.model = cell->coulomb;
  return a;
}

// sqrt(v(k)), k = (q + G) B (Section "Coulomb Interaction"; bulk form Eq.
// untruncated_bare_coulomb).  The truncated brackets 1 - cos(k r_c) and
// 1 - exp(-k_xy z_c) cos(k_z z_c) are taken as 2 sin^2(k r_c / 2) and
// -expm1(-k_xy z_c) + exp(-k_xy z_c) 2 sin^2(k_z z_c / 2): sums of
// non-negative terms, exact rewrites that keep full relative precision at
// small k.  The host has rejected k = 0 except for the sphere.
__device__ __forceinline__ double coulomb_sqrt_at(const CoulombArgs& a, const int32_t* g) {
  const double f0 = g[0] + a.q[0], f1 = g[1] + a.q[1], f2 = g[2] + a.q[2];
  const double kx = f0 * a.b[0] + f1 * a.b[3] + f2 * a.b[6];
  const double ky = f0 * a.b[1] + f1 * a.b[4] + f2 * a.b[7];
  const double kz = f0 * a.b[2] + f1 * a.b[5] + f2 * a.b[8];
  const double k2 = kx * kx + ky * ky + kz * kz;
  constexpr double kFourPi = 4.0 * 3.14159265358979323846;
  if (a.model == BGW_COULOMB_SPHERE) {
    if (k2 == 0.0) return sqrt(2.0 * 3.14159265358979323846) * a.cut;  // (2 pi r_c^2)^{1/2}
    const double s = sin(0.5 * a.cut * sqrt(k2));
    return sqrt(kFourPi * 2.0 / k2) * fabs(s);
  }
  if (a.model == BGW_COULOMB_SLAB) {
    const double x = sqrt(kx * kx + ky * ky) * a.cut;
    const double s = sin(0.5 * kz * a.cut);
    return sqrt(kFourPi / k2 * (-expm1(-x) + exp(-x) * 2.0 * s * s));
  }
  return sqrt(kFourPi / k2);
}

__global__ void coulomb_sqrt_kernel(const int32_t* __restrict__ geps, int ng, CoulombArgs a,
                                    double* __restrict__ sv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ng) return;
  sv[i] = coulomb_sqrt_at(a, geps + 3 * i);
}

// W[i][j] = sv_i epsinv[i][j] sv_j for up to kWBatch matrices per launch
// (grid.y = matrix).  Each matrix is streamed flat: a thread takes four
// elements a block-width apart, issues the four 16-byte loads before any
// store, and finds (i, j) with one 32-bit division each (ng <= 65535, so
// ng^2 < 2^32).
constexpr int kWBatch = 8;
constexpr int kWThreads = 256, kWUnroll = 4;
struct WBatch {
  const double2* in[kWBatch];
  double2* out[kWBatch];
  const double* sv[kWBatch];
  int ng[kWBatch];
};

__global__ void __launch_bounds__(kWThreads) screened_w_kernel(WBatch b) {
  const int m = blockIdx.y;
  const unsigned ng = (unsigned)b.ng[m];
  const unsigned n2 = ng * ng;
  const double* sv = b.sv[m];
  const double2* in = b.in[m];
  double2* out = b.out[m];
  const unsigned long long step = (unsigned long long)gridDim.x * kWThreads * kWUnroll;
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * kWThreads * kWUnroll + threadIdx.x; e0 < n2;
       e0 += step) {
    double2 x[kWUnroll];
    double s[kWUnroll];
#pragma unroll
    for (int u = 0; u < kWUnroll; ++u) {
      const unsigned long long e = e0 + u * kWThreads;
      if (e < n2) {
        x[u] = in[e];
        const unsigned i = (unsigned)e / ng;   // e < n2 < 2^32
        s[u] = sv[i] * sv[(unsigned)e - i * ng];
      }
    }
#pragma unroll
    for (int u = 0; u < kWUnroll; ++u) {
      const unsigned long long e = e0 + u * kWThreads;
      if (e < n2) out[e] = make_double2(s[u] * x[u].x, s[u] * x[u].y);
    }
  }
}

__global__ void eps_form_kernel(const double2* __restrict__ chi, const double* __restrict__ sv, int ng,
                                double2* __restrict__ work, double2* __restrict__ eps) {
  const size_t n2 = (size_t)ng * ng;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ng), j = (int)(e - (size_t)i * ng);
    const double s = sv[i] * sv[j];
    const double2 x = chi[e];
    double2 r = make_double2(-s * x.x, -s * x.y);
    if (i == j) r.x += 1.0;
    work[e] = r;
    if (eps) eps[e] = r;
  }
}

// Inverse of the diagonal block A[k0:k0+kb, k0:k0+kb] -> Dinv[kb][kb] (ld NB).
// The reciprocal of each pivot is formed once (thread 0) and shared: on this
// part every FP64 operation of one SM counts.
__global__ void __launch_bounds__(NB * NB) gj_diag_kernel(const double2* __restrict__ A, int ng, int k0,
                                                          int kb, double2* __restrict__ Dinv,
                                                          int* __restrict__ status) {
  __shared__ double2 D[NB][NB + 1];
  __shared__ double2 pinv;
  const int i = threadIdx.y, j = threadIdx.x;
  const bool in = i < kb && j < kb;
  D[i][j] = in ? A[(size_t)(k0 + i) * ng + k0 + j] : make_double2(i == j ? 1.0 : 0.0, 0.0);
  for (int s = 0; s < kb; ++s) {
    __syncthreads();
    if (i == 0 && j == 0) {
      const double2 piv = D[s][s];
      const double m2 = piv.x * piv.x + piv.y * piv.y;
      if (!(m2 > 0.0) || !isfinite(m2)) {
        atomicExch(status, (int)kDevZeroPivot);
        pinv = make_double2(0.0, 0.0);
      } else {
        const double r = 1.0 / m2;
        pinv = make_double2(piv.x * r, -piv.y * r);  // 1/piv
      }
    }
    __syncthreads();
    const double2 p = pinv;
    const double2 f = D[i][s];
    const double2 rs = D[s][j];
    __syncthreads();
    const double2 rsn = (j == s) ? p : cmul(rs, p);
    if (i == s) {
      D[i][j] = rsn;
    } else {
      double2 v = (j == s) ? make_double2(0.0, 0.0) : D[i][j];
      const double2 t = cmul(f, rsn);
      D[i][j] = make_double2(v.x - t.x, v.y - t.y);
    }
  }
  __syncthreads();
  if (in) Dinv[i * NB + j] = D[i][j];
}

// R[r][j] (ld ng) for all columns j; C[i][s] (ld NB) copy of the column panel.
// grid (ceil(ng/64), 1 + ceil(ng/256)): blockIdx.y == 0 computes R for 64
// columns, blockIdx.y >= 1 copies 256 rows of the column panel.
__global__ void __launch_bounds__(256) gj_panels_kernel(const double2* __restrict__ A, int ng, int k0, int kb,
                                                        const double2* __restrict__ Dinv,
                                                        double2* __restrict__ R, double2* __restrict__ C) {
  const int tid = threadIdx.x;
  if (blockIdx.y > 0) {
    const int i = (blockIdx.y - 1) * 256 + tid;
    if (blockIdx.x != 0 || i >= ng) return;
    for (int s = 0; s < kb; ++s) C[(size_t)i * NB + s] = A[(size_t)i * ng + k0 + s];
    return;
  }
  __shared__ double2 Ds[NB][NB];
  __shared__ double2 As[NB][64];
  const int j0 = blockIdx.x * 64;
  for (int e = tid; e < NB * NB; e += 256) Ds[e / NB][e % NB] = Dinv[e];
  for (int e = tid; e < NB * 64; e += 256) {
    const int s = e / 64, jj = e % 64;
    As[s][jj] = (s < kb && j0 + jj < ng) ? A[(size_t)(k0 + s) * ng + j0 + jj] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < NB * 64; e += 256) {
    const int r = e / 64, jj = e % 64, j = j0 + jj;
    if (r >= kb || j >= ng) continue;
    double2 v;
    if (j >= k0 && j < k0 + kb) {
      v = Ds[r][j - k0];
    } else {
      v = make_double2(0.0, 0.0);
      for (int s = 0; s < kb; ++s) {
        const double2 t = cmul(Ds[r][s], As[s][jj]);
        v.x += t.x;
        v.y += t.y;
      }
    }
    R[(size_t)r * ng + j] = v;
  }
}

// Rank-kb update of the whole matrix.  grid (ceil(ng/64), ceil(ng/64)).
__global__ void __launch_bounds__(256) gj_update_kernel(double2* __restrict__ A, int ng, int k0, int kb,
                                                        const double2* __restrict__ R,
                                                        const double2* __restrict__ C) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 (*Cs)[NB + 1] = reinterpret_cast<double2 (*)[NB + 1]>(smem_raw);
  double2 (*Rs)[TU] = reinterpret_cast<double2 (*)[TU]>(smem_raw + sizeof(double2) * TU * (NB + 1));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * TU, j0 = blockIdx.x * TU;
  for (int e = tid; e < TU * NB; e += 256) {
    const int ii = e / NB, s = e % NB;
    Cs[ii][s] = (i0 + ii < ng && s < kb) ? C[(size_t)(i0 + ii) * NB + s] : make_double2(0.0, 0.0);
  }
  for (int e = tid; e < NB * TU; e += 256) {
    const int s = e / TU, jj = e % TU;
    Rs[s][jj] = (s < kb && j0 + jj < ng) ? R[(size_t)s * ng + j0 + jj] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int s = 0; s < kb; ++s) {
    double2 cv[4], rv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) cv[a] = Cs[ty + 16 * a][s];
#pragma unroll
    for (int b = 0; b < 4; ++b) rv[b] = Rs[s][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b].x = fma(cv[a].x, rv[b].x, acc[a][b].x);
        acc[a][b].x = fma(-cv[a].y, rv[b].y, acc[a][b].x);
        acc[a][b].y = fma(cv[a].x, rv[b].y, acc[a][b].y);
        acc[a][b].y = fma(cv[a].y, rv[b].x, acc[a][b].y);
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= ng) continue;
    const bool irow = i >= k0 && i < k0 + kb;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j >= ng) continue;
      double2* dst = A + (size_t)i * ng + j;
      if (irow) {
        *dst = R[(size_t)(i - k0) * ng + j];
      } else {
        const bool jcol = j >= k0 && j < k0 + kb;
        double2 v = jcol ? make_double2(0.0, 0.0) : *dst;
        *dst = make_double2(v.x - acc[a][b].x, v.y - acc[a][b].y);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Hermitian blocked sweep (the inverse used by bgw_epsinv).
//
// eps~ is Hermitian positive definite, so only its lower triangle is kept
// and updated.  Sweeping the block K (rows/cols k0..k0+kb) with D = A_KK and
// R the other indices maps
//   A_KK -> -D^-1,  A_RK -> A_RK D^-1,  A_KR -> D^-1 A_KR,
//   A_RR -> A_RR - A_RK D^-1 A_KR,
// which keeps the matrix Hermitian; after every block has been swept the
// matrix holds -eps~^-1.  With C = A_RK (read from the stored lower triangle:
// the column panel below K, the conjugated row panel left of K) and
// P = C D^-1 the trailing update of a lower element is
//   A_ij -= sum_s P_is conj(C_js),
// half the work of a full Gauss-Jordan step.
// Matrices swept together: one launch per step serves every matrix
// (blockIdx.y / blockIdx.x selects the matrix), so the single-CTA diagonal
// step of one matrix runs beside those of the others.
constexpr int kSweepBatch = 128;
struct SweepMat {
  double2* A;     // the matrix (lower triangle swept in place)
  double2* C;     // [ng][NB] column panel of the current block
  double2* P;     // [ng][NB] C D^-1
  double2* Dinv;  // [NB][NB]
  int ng;
};
struct SweepBatch {
  int n;
  SweepMat m[kSweepBatch];
};

// Diagonal block of one sweep step (sweep_common.cuh): Dinv gets D^-1 (both
// triangles) and A_KK gets -D^-1 (lower).
__global__ void __launch_bounds__(kDiagThreads) sw_diag_kernel(const __grid_constant__ SweepBatch b, int k0,
                                                               int* __restrict__ status) {
  __shared__ DiagSmem sm;
  const SweepMat& M = b.m[blockIdx.x];
  const int ng = M.ng;
  if (k0 >= ng) return;
  const int kb = min(NB, ng - k0);
  double2* A = M.A;
  const int t = threadIdx.x;
  int i, j;
  bool low;
  diag_thread_element(t, kb, i, j, low);
  if (low) sm.L[i][j] = A[(size_t)(k0 + i) * ng + k0 + j];
  diag_sweep_smem(sm, kb, t, i, j, low, status);
  for (int e2 = threadIdx.x; e2 < NB * NB; e2 += blockDim.x) {
    const int r = e2 / NB, c = e2 % NB;
    if (r >= kb || c >= kb) continue;
    const double2 v = (r >= c) ? sm.L[r][c] : make_double2(sm.L[c][r].x, -sm.L[c][r].y);
    M.Dinv[r * NB + c] = make_double2(-v.x, -v.y);
    if (r >= c) A[(size_t)(k0 + r) * ng + k0 + c] = v;
  }
}

// One warp per row i outside K (lane = column s of the panel):
//   C_i = A_iK (stored lower part), P_i = C_i D^-1, then A_iK <- P_i.
// grid (ceil(max ng / 8), nmat), block 256.
__global__ void __launch_bounds__(256) sw_panel_kernel(const __grid_constant__ SweepBatch b, int k0) {
  __shared__ double2 Ds[NB][NB];
  __shared__ double2 Cs[8][NB];
  const SweepMat& M = b.m[blockIdx.y];
  const int ng = M.ng;
  if (k0 >= ng || blockIdx.x * 8 >= ng) return;
  const int kb = min(NB, ng - k0);
  double2* A = M.A;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < NB * NB; e += 256) Ds[e / NB][e % NB] = M.Dinv[e];
  const int i = blockIdx.x * 8 + warp;
  const bool row_ok = i < ng && (i < k0 || i >= k0 + kb);
  double2 cv = make_double2(0.0, 0.0);
  if (row_ok && lane < kb) {
    if (i >= k0 + kb) {
      cv = A[(size_t)i * ng + k0 + lane];
    } else {
      const double2 t = A[(size_t)(k0 + lane) * ng + i];
      cv = make_double2(t.x, -t.y);
    }
  }
  Cs[warp][lane] = cv;
  __syncthreads();
  if (!row_ok) return;
  double2 pv = make_double2(0.0, 0.0);
  for (int t = 0; t < kb; ++t) {
    const double2 a = Cs[warp][t], d = Ds[t][lane];
    pv.x = fma(a.x, d.x, fma(-a.y, d.y, pv.x));
    pv.y = fma(a.x, d.y, fma(a.y, d.x, pv.y));
  }
  if (lane < kb) {
    M.C[(size_t)i * NB + lane] = cv;
    M.P[(size_t)i * NB + lane] = pv;
    if (i >= k0 + kb)
      A[(size_t)i * ng + k0 + lane] = pv;
    else
      A[(size_t)(k0 + lane) * ng + i] = make_double2(pv.x, -pv.y);
  }
}

// Lower 64x64 tiles: A_ij -= sum_s P_is conj(C_js) for i >= j outside K.
// grid (tiles of the largest matrix, nmat), block 256, dynamic smem.
__global__ void __launch_bounds__(256) sw_update_kernel(const __grid_constant__ SweepBatch b, int k0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 (*Ps)[NB + 1] = reinterpret_cast<double2 (*)[NB + 1]>(smem_raw);
  double2 (*Cs)[NB + 1] = reinterpret_cast<double2 (*)[NB + 1]>(smem_raw + sizeof(double2) * TU * (NB + 1));
  const SweepMat& M = b.m[blockIdx.y];
  const int ng = M.ng;
  if (k0 >= ng) return;
  const int kb = min(NB, ng - k0);
  const int nt = (ng + TU - 1) / TU;
  const long long t = blockIdx.x;
  if (t >= (long long)nt * (nt + 1) / 2) return;
  int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
  while ((long long)I * (I + 1) / 2 > t) --I;
  const int J = (int)(t - (long long)I * (I + 1) / 2);
  const int i0 = I * TU, j0 = J * TU;
  // tiles whose rows or columns all lie inside K have nothing to update
  if (i0 >= k0 && min(i0 + TU, ng) <= k0 + kb) return;
  if (j0 >= k0 && min(j0 + TU, ng) <= k0 + kb) return;
  double2* A = M.A;
  const double2* P = M.P;
  const double2* C = M.C;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < TU * NB; e += 256) {
    const int r = e / NB, s = e % NB;
    const bool sk = s < kb;
    Ps[r][s] = (sk && i0 + r < ng) ? P[(size_t)(i0 + r) * NB + s] : make_double2(0.0, 0.0);
    const double2 cc = (sk && j0 + r < ng) ? C[(size_t)(j0 + r) * NB + s] : make_double2(0.0, 0.0);
    Cs[r][s] = make_double2(cc.x, -cc.y);  // conj(C_js)
  }
  __syncthreads();
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = make_double2(0.0, 0.0);
  for (int s = 0; s < kb; ++s) {
    double2 pv[4], cv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) pv[a] = Ps[ty + 16 * a][s];
#pragma unroll
    for (int c = 0; c < 4; ++c) cv[c] = Cs[tx + 16 * c][s];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[a][c].x = fma(pv[a].x, cv[c].x, acc[a][c].x);
        acc[a][c].x = fma(-pv[a].y, cv[c].y, acc[a][c].x);
        acc[a][c].y = fma(pv[a].x, cv[c].y, acc[a][c].y);
        acc[a][c].y = fma(pv[a].y, cv[c].x, acc[a][c].y);
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= ng || (i >= k0 && i < k0 + kb)) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j > i || (j >= k0 && j < k0 + kb)) continue;
      double2* dst = A + (size_t)i * ng + j;
      const double2 v = *dst;
      *dst = make_double2(v.x - acc[a][c].x, v.y - acc[a][c].y);
    }
  }
}

// The swept lower triangle holds -eps~^-1: negate and mirror into both
// triangles.  One thread per lower element; grid (blocks, nmat).
__global__ void sw_finish_kernel(const __grid_constant__ SweepBatch b) {
  const SweepMat& M = b.m[blockIdx.y];
  const int ng = M.ng;
  double2* A = M.A;
  const long long nlow = (long long)ng * (ng + 1) / 2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nlow;
       e += (long long)gridDim.x * blockDim.x) {
    // row of the packed index: an FP32 estimate (the FP64 pipe is slow on
    // this part) corrected by integer steps; signs flipped on the bits
    int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((long long)(i + 1) * (i + 2) / 2 <= e) ++i;
    while ((long long)i * (i + 1) / 2 > e) --i;
    const int j = (int)(e - (long long)i * (i + 1) / 2);
    const double2 v = A[(size_t)i * ng + j];
    const double nx = neg_bits(v.x);
    if (i == j) {
      A[(size_t)i * ng + j] = make_double2(nx, 0.0);
    } else {
      A[(size_t)i * ng + j] = make_double2(nx, neg_bits(v.y));
      A[(size_t)j * ng + i] = make_double2(nx, v.y);
    }
  }
}

// eps~ formation for every matrix of the batch, then the batched sweep.
int epsinv_batch_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells,
                     const int32_t* const* d_geps, const void* const* chi, void* const* eps, void* const* epsinv,
                     cudaStream_t st, bool tc_update, bool real_values) {
  const int group = tc_update ? 96 : kSweepBatch;
  for (int m0 = 0; m0 < nmat; m0 += group) {
    const int nb = std::min(group, nmat - m0);
    size_t pan = 0;
    int ngmax = 0;
    for (int m = m0; m < m0 + nb; ++m) {
      pan += (size_t)ng[m] * NB;
      ngmax = std::max(ngmax, ng[m]);
    }
    Scratch sv, dinv, R, Cp;
    sv.pool = dinv.pool = R.pool = Cp.pool = &c->pool;
    int rc;
    if ((rc = c->pool.alloc((size_t)ngmax * sizeof(double), &sv.ptr)) != BGW_OK ||
        (rc = c->pool.alloc((size_t)nb * NB * NB * sizeof(double2), &dinv.ptr)) != BGW_OK ||
        (rc = c->pool.alloc(pan * sizeof(double2), &R.ptr)) != BGW_OK ||
        (rc = c->pool.alloc(pan * sizeof(double2), &Cp.ptr)) != BGW_OK)
      return fail(c, rc, "bgw_epsinv: scratch allocation failed");
    SweepBatch sb;
    sb.n = nb;
    size_t off = 0;
    for (int k = 0; k < nb; ++k) {
      const int m = m0 + k;
      double2* A = static_cast<double2*>(epsinv[m]);
      {
        TimedScope ts(c, kTEpsForm, st);
        coulomb_sqrt_kernel<<<(ng[m] + 255) / 256, 256, 0, st>>>(d_geps[m], ng[m], coulomb_args(cells[m]),
                                                                 sv.as<double>());
        const size_t n2 = (size_t)ng[m] * ng[m];
        const unsigned eb = (unsigned)std::min<size_t>((n2 + 255) / 256, 152 * 16);
        eps_form_kernel<<<eb, 256, 0, st>>>(static_cast<const double2*>(chi[m]), sv.as<double>(), ng[m], A,
                                            static_cast<double2*>(eps ? eps[m] : nullptr));
        BGW_CUDA(c, cudaGetLastError());
        c->launches += 2;
      }
      sb.m[k].A = A;
      sb.m[k].C = Cp.as<double2>() + off;
      sb.m[k].P = R.as<double2>() + off;
      sb.m[k].Dinv = dinv.as<double2>() + (size_t)k * NB * NB;
      sb.m[k].ng = ng[m];
      off += (size_t)ng[m] * NB;
    }
    TimedScope ts_inv(c, kTInverse, st);
    const int nt = (ngmax + TU - 1) / TU;
    const long long ntl = (long long)nt * (nt + 1) / 2;
    const size_t upd_smem = sizeof(double2) * 2 * TU * (NB + 1);
    BGW_CUDA(c, cudaFuncSetAttribute(sw_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem));
    std::unique_ptr<OzPlan, void (*)(OzPlan*)> oz(nullptr, oz_plan_delete);
    if (tc_update) {
      oz.reset(oz_plan_new());
      std::vector<int> ngs(nb);
      std::vector<double2*> As(nb);
      std::vector<const double2*> Cs(nb), Ps(nb);
      std::vector<double2*> Ds(nb);
      for (int k = 0; k < nb; ++k) {
        ngs[k] = sb.m[k].ng;
        As[k] = sb.m[k].A;
        Cs[k] = sb.m[k].C;
        Ps[k] = sb.m[k].P;
        Ds[k] = sb.m[k].Dinv;
      }
      if ((rc = oz_prepare(c, nb, ngs.data(), As.data(), Cs.data(), Ps.data(), Ds.data(), oz.get(), false,
                           real_values, c->run_slices, c->run_ff_chain)) != BGW_OK)
        return rc;
      oz_set_bulk_items(oz.get(), c->update_items);   // the option's width, else the SM-count rule
    }
    if (!tc_update) {
      for (int k0 = 0; k0 < ngmax; k0 += NB) {
        sw_diag_kernel<<<nb, kDiagThreads, 0, st>>>(sb, k0, c->d_status);
        sw_panel_kernel<<<dim3((ngmax + 7) / 8, nb), 256, 0, st>>>(sb, k0);
        sw_update_kernel<<<dim3((unsigned)ntl, nb), 256, upd_smem, st>>>(sb, k0);
        BGW_CUDA(c, cudaGetLastError());
        c->launches += 3;
      }
    } else {
      // Look-ahead: the chain that the next step waits for (panel, slices, then
      // the update of the tiles touching the next block, whose CTA holding the
      // next diagonal block also sweeps it)
      // runs on a high-priority side stream, while the main stream updates the
      // other tiles of the current step.  Dependencies:
      //   step k's chain waits for the main-stream update of step k-2 (same
      //     slice buffer; tiles of block k may still be pending there);
      //   step k's next-block update waits for the main-stream update of k-1;
      //   step k's main-stream update waits for step k's slices.
      if (!c->side) {
        int lo = 0, hi = 0;
        BGW_CUDA(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
        BGW_CUDA(c, cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi));
        for (auto& e : c->la_ev) BGW_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      }
      cudaStream_t s2 = c->side;
      cudaEvent_t ev_fork = c->la_ev[0], ev_slice = c->la_ev[1];
      cudaEvent_t ev_rest[2] = {c->la_ev[2], c->la_ev[3]};
      BGW_CUDA(c, cudaEventRecord(ev_fork, st));
      BGW_CUDA(c, cudaStreamWaitEvent(s2, ev_fork, 0));
      int k = 0;
      for (int k0 = 0; k0 < ngmax; k0 += NB, ++k) {
        const int buf = k & 1;
        if (k >= 2) BGW_CUDA(c, cudaStreamWaitEvent(s2, ev_rest[buf], 0));
        {
          TimedScope ts(c, kTSweepChain, s2);
          // the diagonal block of step k >= 1 was swept by step k-1's
          // next-block update (the CTA of the tile holding it)
          if (k == 0) sw_diag_kernel<<<nb, kDiagThreads, 0, s2>>>(sb, k0, c->d_status);
          if ((rc = oz_panel_slice(c, oz.get(), k0, ngmax, buf, s2)) != BGW_OK) return rc;
        }
        BGW_CUDA(c, cudaEventRecord(ev_slice, s2));
        if (k >= 1) BGW_CUDA(c, cudaStreamWaitEvent(s2, ev_rest[buf ^ 1], 0));
        {
          TimedScope ts(c, kTOzAhead, s2);
          if ((rc = oz_update(c, oz.get(), k0, ngmax, buf, 1, s2)) != BGW_OK) return rc;
        }
        BGW_CUDA(c, cudaStreamWaitEvent(st, ev_slice, 0));
        {
          TimedScope ts(c, kTOzUpdate, st);
          if ((rc = oz_update(c, oz.get(), k0, ngmax, buf, 2, st)) != BGW_OK) return rc;
        }
        BGW_CUDA(c, cudaEventRecord(ev_rest[buf], st));
        BGW_CUDA(c, cudaGetLastError());
        c->launches += 4;
      }
      // join: the main stream waits for the side stream's last work
      BGW_CUDA(c, cudaEventRecord(ev_fork, s2));
      BGW_CUDA(c, cudaStreamWaitEvent(st, ev_fork, 0));
    }
    const long long nlow = (long long)ngmax * (ngmax + 1) / 2;
    sw_finish_kernel<<<dim3((unsigned)std::min<long long>((nlow + 255) / 256, 152LL * 16), nb), 256, 0, st>>>(sb);
    BGW_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  return BGW_OK;
}

// ---------------------------------------------------------------------------
int eps_form_run(Ctx* c, const bgw_cell* cell, const int32_t* d_geps, int ng, const void* chi, double* sv,
                 double2* A, void* eps, cudaStream_t st) {
  TimedScope ts(c, kTEpsForm, st);
  coulomb_sqrt_kernel<<<(ng + 255) / 256, 256, 0, st>>>(d_geps, ng, coulomb_args(cell), sv);
  const size_t n2 = (size_t)ng * ng;
  const unsigned eb = (unsigned)std::min<size_t>((n2 + 255) / 256, 152 * 16);
  eps_form_kernel<<<eb, 256, 0, st>>>(static_cast<const double2*>(chi), sv, ng, A, static_cast<double2*>(eps));
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 2;
  return BGW_OK;
}

int gj_update_run(Ctx* c, double2* A, int ng, int k0, int kb, const double2* R, const double2* Cp,
                  cudaStream_t st) {
  const int nt = (ng + TU - 1) / TU;
  const size_t upd_smem = sizeof(double2) * (TU * (NB + 1) + NB * TU);
  BGW_CUDA(c, cudaFuncSetAttribute(gj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem));
  gj_update_kernel<<<dim3(nt, nt), 256, upd_smem, st>>>(A, ng, k0, kb, R, Cp);
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 1;
  return BGW_OK;
}

__global__ void real_to_complex_kernel(const double* __restrict__ x, size_t n, double2* __restrict__ out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_double2(x[e], 0.0);
}
__global__ void real_part_kernel(const double2* __restrict__ x, size_t n, double* __restrict__ out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = x[e].x;
}

int epsinv_rflavor_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells, const int32_t* const* d_geps,
                       const void* const* chi, void* const* eps, void* const* epsinv, cudaStream_t st,
                       bool tc_update) {
  size_t total = 0;
  for (int m = 0; m < nmat; ++m) total += (size_t)ng[m] * ng[m];
  Scratch A, E;
  A.pool = E.pool = &c->pool;
  int rc;
  if ((rc = c->pool.alloc(total * sizeof(double2), &A.ptr)) != BGW_OK ||
      (eps && (rc = c->pool.alloc(total * sizeof(double2), &E.ptr)) != BGW_OK))
    return fail(c, rc, "real-flavor inverse: scratch allocation failed");
  std::vector<const void*> xin(nmat);
  std::vector<void*> ain(nmat), ein(nmat);
  size_t off = 0;
  for (int m = 0; m < nmat; ++m) {
    const size_t n2 = (size_t)ng[m] * ng[m];
    double2* a = A.as<double2>() + off;
    const unsigned gb = (unsigned)std::min<size_t>((n2 + 255) / 256, 152 * 16);
    real_to_complex_kernel<<<gb, 256, 0, st>>>(static_cast<const double*>(chi[m]), n2, a);
    xin[m] = a;
    ain[m] = a;   // eps~ is formed in place: every element is read before it is written
    ein[m] = eps ? static_cast<void*>(E.as<double2>() + off) : nullptr;
    off += n2;
  }
  BGW_CUDA(c, cudaGetLastError());
  c->launches += nmat;
  if ((rc = epsinv_batch_run(c, nmat, ng, cells, d_geps, xin.data(), eps ? ein.data() : nullptr, ain.data(), st,
                             tc_update, true)) != BGW_OK)
    return rc;
  for (int m = 0; m < nmat; ++m) {
    const size_t n2 = (size_t)ng[m] * ng[m];
    const unsigned gb = (unsigned)std::min<size_t>((n2 + 255) / 256, 152 * 16);
    real_part_kernel<<<gb, 256, 0, st>>>(static_cast<const double2*>(ain[m]), n2, static_cast<double*>(epsinv[m]));
    if (eps) real_part_kernel<<<gb, 256, 0, st>>>(static_cast<const double2*>(ein[m]), n2, static_cast<double*>(eps[m]));
  }
  BGW_CUDA(c, cudaGetLastError());
  c->launches += nmat * (eps ? 2 : 1);
  return BGW_OK;
}

int coulomb_sqrt_run(Ctx* c, const bgw_cell* cell, const int32_t* d_geps, int ng, double* sv, cudaStream_t st) {
  coulomb_sqrt_kernel<<<(ng + 255) / 256, 256, 0, st>>>(d_geps, ng, coulomb_args(cell), sv);
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 1;
  return BGW_OK;
}

int screened_w_run(Ctx* c, int nmat, const int* ng, const bgw_cell* const* cells, const int32_t* const* d_geps,
                   const void* const* epsinv, void* const* W, cudaStream_t st) {
  int ngmax = 0;
  for (int m = 0; m < nmat; ++m) ngmax = std::max(ngmax, ng[m]);
  const int nb = std::min(nmat, kWBatch);
  Scratch sv;
  sv.pool = &c->pool;
  int rc;
  if ((rc = c->pool.alloc((size_t)nb * ngmax * sizeof(double), &sv.ptr)) != BGW_OK)
    return fail(c, rc, "bgw_screened_w: scratch allocation failed");
  TimedScope ts(c, kTScreenedW, st);
  for (int m0 = 0; m0 < nmat; m0 += kWBatch) {
    const int cnt = std::min(kWBatch, nmat - m0);
    WBatch b = {};
    size_t most = 0;
    for (int k = 0; k < cnt; ++k) {
      const int m = m0 + k;
      double* svk = sv.as<double>() + (size_t)k * ngmax;
      coulomb_sqrt_kernel<<<(ng[m] + 255) / 256, 256, 0, st>>>(d_geps[m], ng[m], coulomb_args(cells[m]), svk);
      b.in[k] = static_cast<const double2*>(epsinv[m]);
      b.out[k] = static_cast<double2*>(W[m]);
      b.sv[k] = svk;
      b.ng[k] = ng[m];
      most = std::max(most, (size_t)ng[m] * ng[m]);
    }
    // up to 8 resident blocks per SM over the matrices of this launch
    const size_t per_block = (size_t)kWThreads * kWUnroll;
    const unsigned gx = (unsigned)std::min<size_t>((most + per_block - 1) / per_block,
                                                   std::max<size_t>(1, 152 * 8 / cnt));
    screened_w_kernel<<<dim3(gx, (unsigned)cnt), kWThreads, 0, st>>>(b);
    BGW_CUDA(c, cudaGetLastError());
    c->launches += cnt + 1;
  }
  return BGW_OK;
}

int coulomb_check(const bgw_cell* cell, int ng, const int32_t* geps, int* what, int* bad) {
  *what = 0;
  *bad = -1;
  const int model = cell->coulomb;
  if (model != BGW_COULOMB_BULK && model != BGW_COULOMB_SPHERE && model != BGW_COULOMB_SLAB) {
    *what = 1;
    return BGW_EINVAL;
  }
  if (model != BGW_COULOMB_BULK && !(cell->coulomb_cut > 0.0 && std::isfinite(cell->coulomb_cut))) {
    *what = 2;
    return BGW_EINVAL;
  }
  if (model == BGW_COULOMB_SPHERE) return BGW_OK;  // finite everywhere
  for (int i = 0; i < ng; ++i) {
    double k2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      double kd = 0.0;
      for (int a = 0; a < 3; ++a) kd += (geps[3 * i + a] + cell->q_frac[a]) * cell->bvec[a][d];
      k2 += kd * kd;
    }
    if (!(k2 > 0.0)) {
      *what = 3;
      *bad = i;
      return BGW_EINVAL;
    }
  }
  return BGW_OK;
}

// Allocation-free inverse: bgw_epsinv_noalloc (include/bgw.h).
//
// The Gauss-Jordan kernels above, with every scratch buffer
// (Coulomb factors, the G list, the diagonal-block inverse, the two panels and
// the status word) lives in one file-scope device array of fixed size, so the
// call makes no device allocation.  The array is part of the library's device
// image: every GPU that loads the library holds it until the process exits.
namespace {
constexpr int kNoAllocMaxNg = 4096;
// Byte offsets inside the array; each region starts on a 256-byte boundary.
constexpr size_t kNaSv = 0;                                                // double[kNoAllocMaxNg]
constexpr size_t kNaDinv = kNaSv + sizeof(double) * kNoAllocMaxNg;          // double2[NB*NB]
constexpr size_t kNaR = kNaDinv + sizeof(double2) * NB * NB;                // double2[NB*kNoAllocMaxNg]
constexpr size_t kNaC = kNaR + sizeof(double2) * NB * kNoAllocMaxNg;        // double2[kNoAllocMaxNg*NB]
constexpr size_t kNaGeps = kNaC + sizeof(double2) * NB * kNoAllocMaxNg;     // int32[3*kNoAllocMaxNg]
constexpr size_t kNaStatus = kNaGeps + sizeof(int32_t) * 3 * kNoAllocMaxNg; // int
constexpr size_t kNaBytes = kNaStatus + 256;
static_assert(kNaDinv % 256 == 0 && kNaR % 256 == 0 && kNaC % 256 == 0 && kNaGeps % 256 == 0 &&
                  kNaStatus % 256 == 0,
              "scratch regions must stay 256-byte aligned");
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
// Per device: the CUDA context the address was looked up in (its
// process-unique id) and the address.  A symbol's device address belongs to
// one context, so a new context on the device (after cudaDeviceReset, or a
// driver-API context made current by the caller) needs a new lookup.
struct NoallocAddr {
  unsigned long long ctx_id = 0;
  bool valid = false;
  void* ptr = nullptr;
};
NoallocAddr g_noalloc_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

cudaError_t driver_entry(const char* name, int version, void** fn) {
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, version, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  return (q == cudaDriverEntryPointSuccess && *fn) ? cudaSuccess : cudaErrorNotSupported;
}
}  // namespace

// The scratch itself (about 4.1 MiB).  Host code must not use this name as an
// address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch in the current device's current
// context.  Set-up: looked up once per device (with that device current) and
// again whenever the current context is not the one of the cached lookup.
static cudaError_t noalloc_scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void *a = nullptr, *b = nullptr;
    if ((e = driver_entry("cuCtxGetCurrent", 4000, &a)) != cudaSuccess) return e;
    if ((e = driver_entry("cuCtxGetId", 12000, &b)) != cudaSuccess) return e;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
  }
  CUcontext cur = nullptr;
  if (g_ctx_get_current(&cur) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  void* p = nullptr;
  if (!cur) {
    // No context bound to this thread yet: the runtime binds the device's
    // primary context on its first call that needs one.
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    if (g_ctx_get_current(&cur) != CUDA_SUCCESS || !cur) return cudaErrorDeviceUninitialized;
  }
  unsigned long long id = 0;
  if (g_ctx_get_id(cur, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  NoallocAddr& a = g_noalloc_addr[dev];
  if (!a.valid || a.ctx_id != id) {
    if (!p && (e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    a.ptr = p;
    a.ctx_id = id;
    a.valid = true;
  }
  *out = static_cast<unsigned char*>(a.ptr);
  return cudaSuccess;
}

}  // namespace bgw

extern "C" int bgw_epsinv_noalloc(const bgw_cell* cell, int ng, const int32_t* geps, const void* chi, void* eps,
                                  void* epsinv, void* stream) {
  using namespace bgw;
  if (!cell || !geps || !chi || !epsinv || ng <= 0) return BGW_EINVAL;
  if (ng > kNoAllocMaxNg) return BGW_EINVAL;
  int what, bad;
  if (coulomb_check(cell, ng, geps, &what, &bad) != BGW_OK) return BGW_EINVAL;
  unsigned char* base = nullptr;
  if (noalloc_scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return BGW_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* sv = reinterpret_cast<double*>(base + kNaSv);
  double2* dinv = reinterpret_cast<double2*>(base + kNaDinv);
  double2* R = reinterpret_cast<double2*>(base + kNaR);
  double2* Cp = reinterpret_cast<double2*>(base + kNaC);
  int32_t* dgeps = reinterpret_cast<int32_t*>(base + kNaGeps);
  int* status = reinterpret_cast<int*>(base + kNaStatus);
  // The array keeps the previous call's contents: the status word must start at 0.
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemcpyAsync(dgeps, geps, sizeof(int32_t) * 3 * (size_t)ng, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return BGW_ECUDA;
  }
  // Each launch's own status (not the thread's last error, which may hold
  // an earlier call's failure): a failed launch is reported as this call's.
  auto launch = [st](dim3 grid, dim3 block, size_t smem, auto kernel, auto... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
  };
  cudaError_t e = launch(dim3((ng + 255) / 256), dim3(256), 0, coulomb_sqrt_kernel, (const int32_t*)dgeps, ng,
                         coulomb_args(cell), sv);
  double2* A = static_cast<double2*>(epsinv);
  const size_t n2 = (size_t)ng * ng;
  const unsigned eb = (unsigned)std::min<size_t>((n2 + 255) / 256, 152 * 16);
  if (e == cudaSuccess)
    e = launch(dim3(eb), dim3(256), 0, eps_form_kernel, static_cast<const double2*>(chi), (const double*)sv, ng, A,
               static_cast<double2*>(eps));
  const int nt = (ng + TU - 1) / TU;
  const size_t upd_smem = sizeof(double2) * (TU * (NB + 1) + NB * TU);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem);
  for (int k0 = 0; k0 < ng && e == cudaSuccess; k0 += NB) {
    const int kb = std::min(NB, ng - k0);
    e = launch(dim3(1), dim3(NB, NB), 0, gj_diag_kernel, A, ng, k0, kb, dinv, status);
    if (e == cudaSuccess)
      e = launch(dim3((ng + 63) / 64, 1 + (ng + 255) / 256), dim3(256), 0, gj_panels_kernel, (const double2*)A, ng, k0,
                 kb, (const double2*)dinv, R, Cp);
    if (e == cudaSuccess)
      e = launch(dim3(nt, nt), dim3(256), upd_smem, gj_update_kernel, A, ng, k0, kb, (const double2*)R,
                 (const double2*)Cp);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();   // the failure just reported is this call's own
    return BGW_ECUDA;
  }
  return BGW_OK;
}

