// Kernels of the matrix-element step (paper, Eq. eqn_matrix_elem and the
// FFT form that follows it):
//
//   band transform   u_b(r) = sum_G c_b(G) e^{+iG.r}           (per band)
//     band_zpass     scatter the sphere onto its (gx,gy) columns, FFT along z
//     band_yxpass    per z-plane: FFT along y on the occupied gx, then along x
//   pair transform   F_p(G) = (1/N^3) sum_r conj(u_v) u_c e^{+iG.r}
//     pair_yxpass    per (z-plane, pairs): product formed on load, FFT along
//                    y keeping the epsilon-sphere ky, FFT along x keeping the
//                    epsilon-sphere (kx,ky) columns -> T[p][z][col]
//     pair_zgather   per pair: FFT along z of every kept column, gather the
//                    epsilon-sphere kz into the pair-major row M[p][:]
//
// Real-space grids are u[b][z][y][x] (x fastest), n^3 complex per band.
#pragma once
#include <algorithm>

#include "fft.cuh"
#include "runtime.h"

namespace bgw {

template <typename T> __device__ __forceinline__ cpx<T> load_c128(const double2* p) {
  double2 v = *p;
  return mk<T>(T(v.x), T(v.y));
}

// ---------------------------------------------------------------- band z
// grid (ceil(ncol/64), nb), block 64.  smem S[64][N+1].
template <typename T, int N>
__global__ void __launch_bounds__(64) band_zpass(const void* __restrict__ coef, int real_coef, int npw,
                                                 int ncol, const int* __restrict__ col_start,
                                                 const int* __restrict__ ent_col,
                                                 const int* __restrict__ ent_z,
                                                 const int* __restrict__ ent_idx,
                                                 cpx<T>* __restrict__ U1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
  constexpr int CB = 64, LD = N + 1;
  const int col0 = blockIdx.x * CB;
  const int b = blockIdx.y;
  const int tid = threadIdx.x;
  for (int i = tid; i < CB * LD; i += CB) S[i] = mk<T>(T(0), T(0));
  __syncthreads();
  const int e0 = col_start[col0];
  const int e1 = col_start[min(col0 + CB, ncol)];
  if (real_coef) {   // real flavor: real coefficients, imaginary part zero
    const double* cb = static_cast<const double*>(coef) + (size_t)b * npw;
    for (int e = e0 + tid; e < e1; e += CB) S[(ent_col[e] - col0) * LD + ent_z[e]] = mk<T>(T(cb[ent_idx[e]]), T(0));
  } else {
    const double2* cb = static_cast<const double2*>(coef) + (size_t)b * npw;
    for (int e = e0 + tid; e < e1; e += CB) S[(ent_col[e] - col0) * LD + ent_z[e]] = load_c128<T>(cb + ent_idx[e]);
  }
  __syncthreads();
  const int col = col0 + tid;
  if (col >= ncol) return;
  cpx<T> a[N];
#pragma unroll
  for (int z = 0; z < N; ++z) a[z] = S[tid * LD + z];
  fft_line<T, N, 1>(a);
  cpx<T>* out = U1 + (size_t)b * N * ncol + col;
#pragma unroll
  for (int z = 0; z < N; ++z) out[(size_t)z * ncol] = a[z];
}

// ---------------------------------------------------------------- band y,x
// grid (N, nb), block 64.  smem P[N][N+1].
template <typename T, int N>
__global__ void __launch_bounds__(64) band_yxpass(const cpx<T>* __restrict__ U1, int ncol,
                                                  const int* __restrict__ col_xy, int nxs,
                                                  const int* __restrict__ xslot,
                                                  cpx<T>* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* P = reinterpret_cast<cpx<T>*>(smem_raw);
  constexpr int LD = N + 1;
  const int z = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N * LD; i += nt) P[i] = mk<T>(T(0), T(0));
  __syncthreads();
  const cpx<T>* src = U1 + ((size_t)b * N + z) * ncol;
  for (int c = tid; c < ncol; c += nt) {
    int xy = col_xy[c];
    P[(xy / N) * LD + (xy % N)] = src[c];
  }
  __syncthreads();
  for (int s = tid; s < nxs; s += nt) {
    const int x = xslot[s];
    cpx<T> a[N];
#pragma unroll
    for (int y = 0; y < N; ++y) a[y] = P[y * LD + x];
    fft_line<T, N, 1>(a);
#pragma unroll
    for (int y = 0; y < N; ++y) P[y * LD + x] = a[y];
  }
  __syncthreads();
  for (int y = tid; y < N; y += nt) {
    cpx<T> a[N];
#pragma unroll
    for (int x = 0; x < N; ++x) a[x] = P[y * LD + x];
    fft_line<T, N, 1>(a);
#pragma unroll
    for (int x = 0; x < N; ++x) P[y * LD + x] = a[x];
  }
  __syncthreads();
  cpx<T>* dst = u + ((size_t)b * N + z) * N * N;
  for (int i = tid; i < N * N; i += nt) dst[i] = P[(i / N) * LD + (i % N)];
}

// ---------------------------------------------------------------- pair y,x
// grid (ceil(npb/ppb), N), block >= 32.  Pairs pbase .. pbase+npb-1.
// smem: Y[ppb][nys][N+1] | Tz[ppb][ncol] | colmap[N*nys] | yslot[N]
// LB (low band): every kept frequency lies in |k| < N/4 along y and x, so
// each line takes the two outer quarters of its transform (fft_quarters:
// one quarter-length sub-transform live at a time) instead of the whole
// line in registers.  FP32: at most 128 registers, so two 256-thread blocks
// share an SM (a register-limited single block leaves the SM latency-bound);
// a whole FP32 line of more than 40 points needs more, and FP64 keeps its
// registers (a cap would spill).
template <typename T, int N, bool LB>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && (LB || N <= 40)) ? 2 : 1) pair_yxpass(const cpx<T>* __restrict__ uv,
                                                   const cpx<T>* __restrict__ uc, int nc,
                                                   int pbase, int npb, int ppb, int nys, int ncol,
                                                   const int* __restrict__ g_colmap,
                                                   const int* __restrict__ g_yslot,
                                                   cpx<T>* __restrict__ Tbuf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LD = N + 1;
  cpx<T>* Y = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* Tz = Y + (size_t)ppb * nys * LD;
  int* colmap = reinterpret_cast<int*>(Tz + (size_t)ppb * ncol);
  int* yslot = colmap + N * nys;
  const int z = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  const int pl0 = blockIdx.x * ppb;                  // first local pair of this block
  const int npp = min(ppb, npb - pl0);               // pairs in this block
  for (int i = tid; i < N * nys; i += nt) colmap[i] = g_colmap[i];
  for (int i = tid; i < N; i += nt) yslot[i] = g_yslot[i];
  __syncthreads();
  const size_t plane = (size_t)N * N;
  // phase A: FFT along y of conj(u_v) u_c for every x, keep the ky slots
  for (int j = tid; j < npp * N; j += nt) {
    const int pp = j / N, x = j - pp * N;
    const int p = pbase + pl0 + pp;
    const int v = p / nc, c = p - v * nc;
    const cpx<T>* pv = uv + ((size_t)v * N + z) * plane + x;
    const cpx<T>* pc = uc + ((size_t)c * N + z) * plane + x;
    cpx<T>* yrow = Y + (size_t)pp * nys * LD + x;
    if constexpr (LB) {
      constexpr int Q = N / 4;
      cpx<T> lo[Q], hi[Q];
      fft_quarters<T, N>([&](int y) { return cmulc<T>(pv[(size_t)y * N], pc[(size_t)y * N]); }, lo, hi);
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int s0 = yslot[k], s3 = yslot[k + 3 * Q];
        if (s0 >= 0) yrow[s0 * LD] = lo[k];
        if (s3 >= 0) yrow[s3 * LD] = hi[k];
      }
    } else {
      cpx<T> a[N];
#pragma unroll
      for (int y = 0; y < N; ++y) a[y] = cmulc<T>(pv[(size_t)y * N], pc[(size_t)y * N]);
      fft_line<T, N, 1>(a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int s = yslot[k];
        if (s >= 0) yrow[s * LD] = a[k];
      }
    }
  }
  __syncthreads();
  // phase B: FFT along x of each kept ky row, keep the sphere's columns
  for (int j = tid; j < npp * nys; j += nt) {
    const int pp = j / nys, s = j - pp * nys;
    const cpx<T>* row = Y + ((size_t)pp * nys + s) * LD;
    cpx<T>* tz = Tz + (size_t)pp * ncol;
    if constexpr (LB) {
      constexpr int Q = N / 4;
      cpx<T> lo[Q], hi[Q];
      fft_quarters<T, N>([&](int x) { return row[x]; }, lo, hi);
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int c0 = colmap[k * nys + s], c3 = colmap[(k + 3 * Q) * nys + s];
        if (c0 >= 0) tz[c0] = lo[k];
        if (c3 >= 0) tz[c3] = hi[k];
      }
    } else {
      cpx<T> a[N];
#pragma unroll
      for (int x = 0; x < N; ++x) a[x] = row[x];
      fft_line<T, N, 1>(a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int col = colmap[k * nys + s];
        if (col >= 0) tz[col] = a[k];
      }
    }
  }
  __syncthreads();
  // phase C: coalesced store of the kept columns of this plane
  for (int i = tid; i < npp * ncol; i += nt) {
    const int pp = i / ncol, col = i - pp * ncol;
    Tbuf[((size_t)(pl0 + pp) * N + z) * ncol + col] = Tz[i];
  }
}

// ---------------------------------------------------------------- pair y,x (warp per pair)
// The low-band form of pair_yxpass with one warp per pair and no block-wide
// barrier between the passes: the y pass over the N x columns (lane = x),
// __syncwarp, then the x pass over the nys kept ky rows (lane = row), whose
// kept columns are staged over the warp's Y rows and stored to T in whole,
// coalesced runs.  A
// pair's two passes keep 32 lanes busy for 83 of 96 lane-lines at N = 60
// instead of the block kernel's 332 of 512, and warps of a block move on
// independently.  grid (ceil(npb / kPairWarps), N), block 32 kPairWarps.
// smem: Y[kPairWarps][nys][N+1] | colmap[N*nys] | yslot[N].
constexpr int kPairWarps = 4;
constexpr int kWarpPerPair = kPairWarpCode;   // tuner's code for pair_yxpass_warp
template <typename T, int N>
__global__ void __launch_bounds__(32 * kPairWarps, sizeof(T) == 4 ? 4 : 2)
    pair_yxpass_warp(const cpx<T>* __restrict__ uv, const cpx<T>* __restrict__ uc, int nc, int pbase, int npb,
                     int nys, int ncol, const int* __restrict__ g_colmap, const int* __restrict__ g_yslot,
                     cpx<T>* __restrict__ Tbuf) {
  static_assert(N % 4 == 0, "low-band lines need N divisible by 4");
  constexpr int LD = N + 1, Q = N / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* Y = reinterpret_cast<cpx<T>*>(smem_raw);
  int* colmap = reinterpret_cast<int*>(Y + (size_t)kPairWarps * nys * LD);
  int* yslot = colmap + N * nys;
  const int z = blockIdx.y, tid = threadIdx.x;
  for (int i = tid; i < N * nys; i += blockDim.x) colmap[i] = g_colmap[i];
  for (int i = tid; i < N; i += blockDim.x) yslot[i] = g_yslot[i];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int pl = blockIdx.x * kPairWarps + warp;     // pair of this warp inside the call's block of pairs
  if (pl >= npb) return;
  const int p = pbase + pl;
  const int v = p / nc, c = p - v * nc;
  const size_t plane = (size_t)N * N;
  const cpx<T>* pv = uv + ((size_t)v * N + z) * plane;
  const cpx<T>* pc = uc + ((size_t)c * N + z) * plane;
  cpx<T>* Yw = Y + (size_t)warp * nys * LD;
  // y pass: conj(u_v) u_c formed on load, the kept ky of every x column
  for (int x = lane; x < N; x += 32) {
    cpx<T> lo[Q], hi[Q];
    fft_quarters<T, N>([&](int y) { return cmulc<T>(pv[(size_t)y * N + x], pc[(size_t)y * N + x]); }, lo, hi);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int s0 = yslot[k], s3 = yslot[k + 3 * Q];
      if (s0 >= 0) Yw[s0 * LD + x] = lo[k];
      if (s3 >= 0) Yw[s3 * LD + x] = hi[k];
    }
  }
  __syncwarp();
  // x pass: the kept (kx, ky) columns of each kept ky row (low-band grids
  // keep at most N/2 <= 32 rows: one per lane); the columns are staged over
  // Y once every row is read and stored to T in coalesced runs
  cpx<T>* Tp = Tbuf + ((size_t)pl * N + z) * ncol;
  const int s = lane;
  cpx<T> lo[Q], hi[Q];
  if (s < nys) {
    const cpx<T>* row = Yw + (size_t)s * LD;
    fft_quarters<T, N>([&](int x) { return row[x]; }, lo, hi);
  }
  __syncwarp();
  if (s < nys) {
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int c0 = colmap[k * nys + s], c3 = colmap[(k + 3 * Q) * nys + s];
      if (c0 >= 0) Yw[c0] = lo[k];
      if (c3 >= 0) Yw[c3] = hi[k];
    }
  }
  __syncwarp();
  for (int c = lane; c < ncol; c += 32) Tp[c] = Yw[c];
}

// ---------------------------------------------------------------- pair z
// grid (npb), block 256.  smem Mrow[ng], or none with direct != 0 (a list
// too long for shared memory: the outputs go straight to M, complex only).
template <typename T, int N, bool LB>
__global__ void __launch_bounds__(256) pair_zgather(const cpx<T>* __restrict__ Tbuf, int pbase,
                                                    int ncol, int ng,
                                                    const int* __restrict__ zmap,
                                                    void* __restrict__ M, int real_out, int direct) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* Mrow = direct ? static_cast<cpx<T>*>(M) + (size_t)(pbase + blockIdx.x) * ng
                        : reinterpret_cast<cpx<T>*>(smem_raw);
  const int pl = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const T inv = T(1) / T(N * N * N);
  const cpx<T>* src = Tbuf + (size_t)pl * N * ncol;
  for (int col = tid; col < ncol; col += nt) {
    if constexpr (LB) {
      constexpr int Q = N / 4;
      cpx<T> lo[Q], hi[Q];
      fft_quarters<T, N>([&](int z) { return src[(size_t)z * ncol + col]; }, lo, hi);
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const int g0 = zmap[k * ncol + col], g3 = zmap[(k + 3 * Q) * ncol + col];
        if (g0 >= 0) Mrow[g0] = scale<T>(lo[k], inv);
        if (g3 >= 0) Mrow[g3] = scale<T>(hi[k], inv);
      }
    } else {
      cpx<T> a[N];
#pragma unroll
      for (int z = 0; z < N; ++z) a[z] = src[(size_t)z * ncol + col];
      fft_line<T, N, 1>(a);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int g = zmap[k * ncol + col];
        if (g >= 0) Mrow[g] = scale<T>(a[k], inv);
      }
    }
  }
  if (direct) return;
  __syncthreads();
  if (real_out) {   // real flavor: M is real (its imaginary part vanishes up to rounding)
    T* dst = static_cast<T*>(M) + (size_t)(pbase + pl) * ng;
    for (int i = tid; i < ng; i += nt) dst[i] = Mrow[i].x;
  } else {
    cpx<T>* dst = static_cast<cpx<T>*>(M) + (size_t)(pbase + pl) * ng;
    for (int i = tid; i < ng; i += nt) dst[i] = Mrow[i];
  }
}

// ------------------------------------------------------------ launchers
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Shared memory and threads of a pair_yxpass block holding ppb pairs.
template <typename T, int N>
static void pair_block_shape(int ppb, int nys, int ncol, int* threads, size_t* smem) {
  *smem = (size_t)ppb * nys * (N + 1) * sizeof(cpx<T>) + (size_t)ppb * ncol * sizeof(cpx<T>) +
          (size_t)(N * nys + N) * sizeof(int);
  const int t = ((ppb * N + 31) / 32) * 32;
  *threads = t > 256 ? 256 : t;
}

// Autotuner of the pairs per pair_yxpass block: each candidate runs twice on
// the first pairs of the call (the second run is timed with CUDA events on
// the call's stream) and the fastest is kept for this (grid, precision,
// epsilon-sphere shape).  Runs once per shape, outside graph capture.
template <typename T, int N, bool LB>
static int tune_pairs_per_block(const MtxelExec& x, const cpx<T>* uv, const cpx<T>* uc, cpx<T>* Tb) {
  const PairPlan* pp = x.pp;
  const int npb = (int)std::min<long long>((long long)x.nv * x.nc, std::min<long long>(x.pair_block, 4096));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 256 / N > 0 ? 256 / N : 1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 256 / N > 0 ? 256 / N : 1;
  }
  int best = 0;
  float best_ms = 1e30f;
  const int cands[] = {1, 2, 3, 4, 6, 8, 12};
  for (int p : cands) {
    int threads;
    size_t sm;
    pair_block_shape<T, N>(p, pp->nys, pp->ncol, &threads, &sm);
    if (sm > 200 * 1024 || p * N > 1024) continue;
    if (set_smem(pair_yxpass<T, N, LB>, sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, x.st);
      pair_yxpass<T, N, LB><<<dim3((npb + p - 1) / p, N), threads, sm, x.st>>>(
          uv, uc, x.nc, 0, npb, p, pp->nys, pp->ncol, pp->d_colmap, pp->d_yslot_of_k, Tb);
      cudaEventRecord(e1, x.st);
    }
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    *x.launches += 2;
    if (ms < best_ms) {
      best_ms = ms;
      best = p;
    }
  }
  if constexpr (LB) {   // the warp-per-pair kernel as one more candidate
    const size_t sm = (size_t)kPairWarps * pp->nys * (N + 1) * sizeof(cpx<T>) + (size_t)(N * pp->nys + N) * sizeof(int);
    float ms = 0.f;
    if (sm <= 200 * 1024 && set_smem(pair_yxpass_warp<T, N>, sm) == cudaSuccess) {
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, x.st);
        pair_yxpass_warp<T, N><<<dim3((npb + kPairWarps - 1) / kPairWarps, N), 32 * kPairWarps, sm, x.st>>>(
            uv, uc, x.nc, 0, npb, pp->nys, pp->ncol, pp->d_colmap, pp->d_yslot_of_k, Tb);
        cudaEventRecord(e1, x.st);
      }
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        *x.launches += 2;
        if (ms < best_ms) {
          best_ms = ms;
          best = kWarpPerPair;
        }
      } else {
        cudaGetLastError();
      }
    } else {
      cudaGetLastError();
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best > 0 ? best : (256 / N > 0 ? 256 / N : 1);
}

template <typename T, int N>
static cudaError_t band_transform(const BandPlan* bp, const void* coef, int real_coef, int nb, cpx<T>* U1,
                                  cpx<T>* u, cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  size_t sm1 = (size_t)64 * (N + 1) * sizeof(cpx<T>);
  cudaError_t e = set_smem(band_zpass<T, N>, sm1);
  if (e != cudaSuccess) return e;
  band_zpass<T, N><<<dim3((bp->ncol + 63) / 64, nb), 64, sm1, st>>>(
      coef, real_coef, bp->npw, bp->ncol, bp->d_col_start, bp->d_ent_col, bp->d_ent_z, bp->d_ent_idx, U1);
  size_t sm2 = (size_t)N * (N + 1) * sizeof(cpx<T>);
  if ((e = set_smem(band_yxpass<T, N>, sm2)) != cudaSuccess) return e;
  band_yxpass<T, N><<<dim3(N, nb), 64, sm2, st>>>(U1, bp->ncol, bp->d_col_xy, bp->nxs, bp->d_xslot, u);
  return cudaGetLastError();
}

template <typename T, int N, bool LB>
static cudaError_t mtxel_exec_lb(const MtxelExec& x) {
  using C = cpx<T>;
  C* uv = reinterpret_cast<C*>(x.uv);
  C* uc = reinterpret_cast<C*>(x.uc);
  C* U1 = reinterpret_cast<C*>(x.U1);
  C* Tb = reinterpret_cast<C*>(x.T);
  void* M = x.M;
  cudaError_t e;
  {
    TimedScope ts(x.ctx, kTBand, x.st);
    if ((e = band_transform<T, N>(x.bpv, x.cv, x.real, x.nv, U1, uv, x.st)) != cudaSuccess) return e;
    if ((e = band_transform<T, N>(x.bpc, x.cc, x.real, x.nc, U1, uc, x.st)) != cudaSuccess) return e;
  }
  *x.launches += 4;
  const PairPlan* pp = x.pp;
  int ppb = x.tuned_ppb ? *x.tuned_ppb : 0;
  if (ppb <= 0) {
    ppb = tune_pairs_per_block<T, N, LB>(x, uv, uc, Tb);
    if (x.tuned_ppb) *x.tuned_ppb = ppb;
  }
  // a variant that does not apply to this grid or precision (a forced
  // choice) falls back to the block kernel with the default pairs per block
  const bool warp_kernel = LB && ppb == kWarpPerPair;
  if (ppb >= kWarpPerPair && !warp_kernel) ppb = 256 / N > 0 ? 256 / N : 1;
  int threads = 32 * kPairWarps;
  size_t sm = 0;
  if constexpr (LB) {
    if (warp_kernel) {
      sm = (size_t)kPairWarps * pp->nys * (N + 1) * sizeof(C) + (size_t)(N * pp->nys + N) * sizeof(int);
      if ((e = set_smem(pair_yxpass_warp<T, N>, sm)) != cudaSuccess) return e;
    }
  }
  if (!warp_kernel) {
    pair_block_shape<T, N>(ppb, pp->nys, pp->ncol, &threads, &sm);
    if ((e = set_smem(pair_yxpass<T, N, LB>, sm)) != cudaSuccess) return e;
  }
  size_t smz = (size_t)pp->ng * sizeof(C);
  const int zdirect = (smz > 200 * 1024 && !x.real) ? 1 : 0;
  if (zdirect) smz = 0;
  else if ((e = set_smem(pair_zgather<T, N, LB>, smz)) != cudaSuccess) return e;
  const long long npairs = (long long)x.nv * x.nc;
  for (long long p0 = 0; p0 < npairs; p0 += x.pair_block) {
    const int npb = (int)((npairs - p0) < x.pair_block ? (npairs - p0) : x.pair_block);
    {
      TimedScope ts(x.ctx, kTPairYX, x.st);
      if constexpr (LB) {
        if (warp_kernel)
          pair_yxpass_warp<T, N><<<dim3((npb + kPairWarps - 1) / kPairWarps, N), threads, sm, x.st>>>(
              uv, uc, x.nc, (int)p0, npb, pp->nys, pp->ncol, pp->d_colmap, pp->d_yslot_of_k, Tb);
      }
      if (!warp_kernel)
        pair_yxpass<T, N, LB><<<dim3((npb + ppb - 1) / ppb, N), threads, sm, x.st>>>(
            uv, uc, x.nc, (int)p0, npb, ppb, pp->nys, pp->ncol, pp->d_colmap, pp->d_yslot_of_k, Tb);
    }
    {
      TimedScope ts(x.ctx, kTPairZ, x.st);
      pair_zgather<T, N, LB><<<npb, 256, smz, x.st>>>(Tb, (int)p0, pp->ncol, pp->ng, pp->d_zmap, M, x.real,
                                                      zdirect);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *x.launches += 2;
  }
  return cudaSuccess;
}

// The low-band kernels where the plan allows them (every kept frequency in
// |k| < N/4 on all three axes, N divisible by 4), the whole-line ones
// otherwise.
template <typename T, int N>
static cudaError_t mtxel_exec_n(const MtxelExec& x) {
  if constexpr (N % 4 == 0 && N >= 16) {
    if (x.pp->lowband) return mtxel_exec_lb<T, N, true>(x);
  }
  return mtxel_exec_lb<T, N, false>(x);
}

#define BGW_FOR_EACH_N(X) X(8) X(10) X(12) X(16) X(20) X(24) X(30) X(32) X(36) X(40) X(48) X(50) X(60) X(64)

template <typename T>
static cudaError_t mtxel_exec_t(const MtxelExec& x) {
  switch (x.n) {
#define BGW_CASE(n) case n: return mtxel_exec_n<T, n>(x);
    BGW_FOR_EACH_N(BGW_CASE)
#undef BGW_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bgw
