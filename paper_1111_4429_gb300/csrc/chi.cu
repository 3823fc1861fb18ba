// Polarizability, plain FP64 path (paper, Eq. eqn_static_xi written as the
// matrix product of Eq. eqn_static_xi_compact):
//   chi[G][G'] (+)= scale * sum_p w_p conj(M[p][G]) M[p][G'],  scale = 4/Omega
// with pair weights w_p = 1/Delta_p (static) or Delta_p/(Delta_p^2 + omega^2)
// (Eq. retarded_advanced_epsilon at E = i omega), Delta_p = E_v - E_c.
//
// chi is Hermitian, so only the lower-triangle 64x64 tiles are computed; each
// result is written to its own position and, conjugated, to the mirrored one.
// FP64 FMA on the CUDA cores: each thread holds a 4x4 block of complex
// accumulators and streams 16-pair slices of both operand tiles through
// shared memory.
#include "runtime.h"

namespace bgw {

// w[f][p] for every frequency f (nfreq = 0: one static row).
__global__ void chi_weights_kernel(const double* __restrict__ ev, const double* __restrict__ ec,
                                   int nv, int nc, int nrow, const double* __restrict__ omega,
                                   int is_static, double* __restrict__ w) {
  const long long K = (long long)nv * nc;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K * nrow) return;
  const int f = (int)(i / K);
  const long long p = i - (long long)f * K;
  const int v = (int)(p / nc), c = (int)(p - (long long)v * nc);
  const double d = ev[v] - ec[c];
  if (is_static) {
    w[i] = 1.0 / d;
  } else {
    const double om = omega[f];
    w[i] = d / fma(d, d, om * om);
  }
}

namespace {
constexpr int TB = 64;   // tile edge (G)
constexpr int KB = 16;   // pairs per shared-memory slice
}

__global__ void __launch_bounds__(256) chi_f64_kernel(const double2* __restrict__ M, long long K, int ng,
                                                      const double* __restrict__ w, double scale,
                                                      int accumulate, double2* __restrict__ chi) {
  __shared__ double2 As[KB][TB];
  __shared__ double2 Bs[KB][TB];
  // lower-triangle tile (I >= J) from the linear block index
  const long long t = blockIdx.x;
  int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
  while ((long long)I * (I + 1) / 2 > t) --I;
  const int J = (int)(t - (long long)I * (I + 1) / 2);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = I * TB, col0 = J * TB;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (long long k0 = 0; k0 < K; k0 += KB) {
#pragma unroll
    for (int q = 0; q < (KB * TB) / 256; ++q) {
      const int e = tid + 256 * q;
      const int kk = e / TB, r = e % TB;
      const long long k = k0 + kk;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (k < K) {
        const double wk = w[k];
        if (row0 + r < ng) a = M[k * ng + row0 + r];
        if (col0 + r < ng) {
          b = M[k * ng + col0 + r];
          b.x *= wk;
          b.y *= wk;
        }
      }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KB; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // acc += conj(a) * b
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(-a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int g = row0 + ty + 16 * i;
    if (g >= ng) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gp = col0 + tx + 16 * j;
      if (gp >= ng || gp > g) continue;  // lower triangle incl. diagonal
      double2 v = make_double2(acc[i][j].x * scale, acc[i][j].y * scale);
      double2* lo = chi + (size_t)g * ng + gp;
      if (accumulate) {
        const double2 old = *lo;
        v.x += old.x;
        v.y += old.y;
      }
      if (g == gp) v.y = 0.0;  // the diagonal of a Hermitian matrix is real
      *lo = v;
      if (g != gp) chi[(size_t)gp * ng + g] = make_double2(v.x, -v.y);
    }
  }
}

// Real flavor, FP64: chi[G][G'] (+)= scale sum_p w_p M[p][G] M[p][G'] with real
// M (a real SYRK: a quarter of the complex flops), lower 64x64 tiles,
// mirrored; 4x4 register blocking as the complex kernel.
__global__ void __launch_bounds__(256) chi_f64_real_kernel(const double* __restrict__ M, long long K, int ng,
                                                           const double* __restrict__ w, double scale,
                                                           int accumulate, double* __restrict__ chi) {
  __shared__ double As[KB][TB];
  __shared__ double Bs[KB][TB];
  const long long t = blockIdx.x;
  int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
  while ((long long)I * (I + 1) / 2 > t) --I;
  const int J = (int)(t - (long long)I * (I + 1) / 2);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = I * TB, col0 = J * TB;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long long k0 = 0; k0 < K; k0 += KB) {
#pragma unroll
    for (int q = 0; q < (KB * TB) / 256; ++q) {
      const int e = tid + 256 * q;
      const int kk = e / TB, r = e % TB;
      const long long k = k0 + kk;
      double a = 0.0, b = 0.0;
      if (k < K) {
        if (row0 + r < ng) a = M[k * ng + row0 + r];
        if (col0 + r < ng) b = M[k * ng + col0 + r] * w[k];
      }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KB; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int g = row0 + ty + 16 * i;
    if (g >= ng) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gp = col0 + tx + 16 * j;
      if (gp >= ng || gp > g) continue;
      double v = acc[i][j] * scale;
      double* lo = chi + (size_t)g * ng + gp;
      if (accumulate) v += *lo;
      *lo = v;
      if (g != gp) chi[(size_t)gp * ng + g] = v;
    }
  }
}

int chi_mixed_run(Ctx* c, int prec, long long K, int ng, const void* M, const double* w, int nrow,
                  double scale, int accumulate, void* chi, cudaStream_t st, bool real);

int chi_run(Ctx* c, int prec, int nv, int nc, int ng, const void* M, const double* d_ev,
            const double* d_ec, int nfreq, const double* d_omega, double scale, int accumulate,
            void* chi, cudaStream_t st, const HeadPlan* hp, const double2* h, bool real) {
  const long long K = (long long)nv * nc;
  const int nrow = nfreq > 0 ? nfreq : 1;
  Scratch w;
  w.pool = &c->pool;
  int rc = c->pool.alloc((size_t)K * nrow * sizeof(double), &w.ptr);
  if (rc != BGW_OK) return fail(c, rc, "bgw_chi_sum: weight scratch allocation failed");
  const long long nw = K * nrow;
  chi_weights_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(d_ev, d_ec, nv, nc, nrow, d_omega,
                                                                   nfreq == 0, w.as<double>());
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 1;
  if (prec != BGW_PREC_FP64) {
    if ((rc = chi_mixed_run(c, prec, K, ng, M, w.as<double>(), nrow, scale, accumulate, chi, st, real)) != BGW_OK)
      return rc;
    if (hp && hp->g0 >= 0) return head_wings(c, hp, K, ng, M, h, w.as<double>(), nrow, scale, chi, st);
    return BGW_OK;
  }
  const int nt = (ng + TB - 1) / TB;
  const long long ntiles = (long long)nt * (nt + 1) / 2;
  if (real) {
    for (int f = 0; f < nrow; ++f) {
      TimedScope ts(c, kTChiF64, st);
      chi_f64_real_kernel<<<(unsigned)ntiles, 256, 0, st>>>(static_cast<const double*>(M), K, ng,
                                                             w.as<double>() + (size_t)f * K, scale, accumulate,
                                                             static_cast<double*>(chi) + (size_t)f * ng * ng);
      BGW_CUDA(c, cudaGetLastError());
      c->launches += 1;
    }
    return BGW_OK;
  }
  for (int f = 0; f < nrow; ++f) {
    TimedScope ts(c, kTChiF64, st);
    chi_f64_kernel<<<(unsigned)ntiles, 256, 0, st>>>(static_cast<const double2*>(M), K, ng,
                                                      w.as<double>() + (size_t)f * K, scale, accumulate,
                                                      static_cast<double2*>(chi) + (size_t)f * ng * ng);
    BGW_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  return BGW_OK;
}

// ---------------------------------------------------------------------------
// Real axis (Eq. retarded_advanced_epsilon): complex pair weights
//   w_p(E) = (1/2) [1/(D - E - s i delta) + 1/(D + E + s i delta)],
// s = +1 retarded, -1 advanced, D = E_v - E_c.  chi = (4/Omega) sum_p w_p
// conj(M_p(G)) M_p(G') is no longer Hermitian, so every tile is computed.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double2 cinv(double2 z) {
  const double m = fma(z.x, z.x, z.y * z.y);
  return make_double2(z.x / m, -z.y / m);
}

__global__ void chi_weights_real_kernel(const double* __restrict__ ev, const double* __restrict__ ec, int nv,
                                        int nc, int nrow, const double* __restrict__ energy, double delta,
                                        double sgn, double2* __restrict__ w) {
  const long long K = (long long)nv * nc;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K * nrow) return;
  const int f = (int)(i / K);
  const long long p = i - (long long)f * K;
  const int v = (int)(p / nc), c = (int)(p - (long long)v * nc);
  const double d = ev[v] - ec[c];
  const double e = energy[f], sd = sgn * delta;
  const double2 a = cinv(make_double2(d - e, -sd));   // 1/(D - E - s i delta)
  const double2 b = cinv(make_double2(d + e, sd));    // 1/(D + E + s i delta)
  w[i] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
}

// chi[G][G'] (+)= scale sum_p conj(M[p][G]) w_p M[p][G'] over all 64x64 tiles
// (grid = nt^2), same register blocking as the Hermitian kernel.
__global__ void __launch_bounds__(256) chi_f64_general_kernel(const double2* __restrict__ M, long long K, int ng,
                                                              const double2* __restrict__ w, double scale,
                                                              int accumulate, double2* __restrict__ chi) {
  __shared__ double2 As[KB][TB];
  __shared__ double2 Bs[KB][TB];
  const int nt = (ng + TB - 1) / TB;
  const int I = (int)(blockIdx.x / nt), J = (int)(blockIdx.x - (unsigned)I * nt);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = I * TB, col0 = J * TB;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (long long k0 = 0; k0 < K; k0 += KB) {
#pragma unroll
    for (int q = 0; q < (KB * TB) / 256; ++q) {
      const int e = tid + 256 * q;
      const int kk = e / TB, r = e % TB;
      const long long k = k0 + kk;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (k < K) {
        if (row0 + r < ng) a = M[k * ng + row0 + r];
        if (col0 + r < ng) {
          const double2 m = M[k * ng + col0 + r], wk = w[k];
          b = make_double2(fma(wk.x, m.x, -wk.y * m.y), fma(wk.x, m.y, wk.y * m.x));
        }
      }
      As[kk][r] = a;
      Bs[kk][r] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KB; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(-a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int g = row0 + ty + 16 * i;
    if (g >= ng) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gp = col0 + tx + 16 * j;
      if (gp >= ng) continue;
      double2 v = make_double2(acc[i][j].x * scale, acc[i][j].y * scale);
      double2* dst = chi + (size_t)g * ng + gp;
      if (accumulate) {
        const double2 old = *dst;
        v.x += old.x;
        v.y += old.y;
      }
      *dst = v;
    }
  }
}

int chi_real_mixed_run(Ctx* c, int prec, long long K, int ng, const void* M, const double2* w, int nrow,
                       double scale, int accumulate, void* chi, cudaStream_t st);

int chi_real_run(Ctx* c, int prec, int nv, int nc, int ng, const void* M, const double* d_ev, const double* d_ec,
                 int nfreq, const double* d_energy, double delta, int advanced, double scale, int accumulate,
                 void* chi, cudaStream_t st) {
  const long long K = (long long)nv * nc;
  Scratch w;
  w.pool = &c->pool;
  int rc = c->pool.alloc((size_t)K * nfreq * sizeof(double2), &w.ptr);
  if (rc != BGW_OK) return fail(c, rc, "real-axis chi: weight scratch allocation failed");
  const long long nw = K * nfreq;
  chi_weights_real_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(d_ev, d_ec, nv, nc, nfreq, d_energy, delta,
                                                                        advanced ? -1.0 : 1.0, w.as<double2>());
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 1;
  if (prec != BGW_PREC_FP64)
    return chi_real_mixed_run(c, prec, K, ng, M, w.as<double2>(), nfreq, scale, accumulate, chi, st);
  const int nt = (ng + TB - 1) / TB;
  for (int f = 0; f < nfreq; ++f) {
    TimedScope ts(c, kTChiF64, st);
    chi_f64_general_kernel<<<(unsigned)(nt * nt), 256, 0, st>>>(static_cast<const double2*>(M), K, ng,
                                                                 w.as<double2>() + (size_t)f * K, scale,
                                                                 accumulate,
                                                                 static_cast<double2*>(chi) + (size_t)f * ng * ng);
    BGW_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  return BGW_OK;
}

}  // namespace bgw
