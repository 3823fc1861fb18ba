// Diagonal static COHSEX and bare exchange for one q (paper, Section "The
// Self-Energy": Eqs. cohsex-sx, cohsex-ch-sum, cohsex-ch-exact, hf-x), fed by
// the eps~^-1 of the epsilon path:
//   m_p(G) = M_{n''n}(k, -q, -G) = sum_{G2} conj(c_n''(G2 - G)) c_n(G2),
//            p = n'' n_outer + n, the inner band n'' on the k - q sphere;
//   W = eps^-1 v = V^1/2 eps~^-1 V^1/2;
//   qW_p = m_p^H W m_p,  qV_p = sum_G |m_p(G)|^2 v_G;
//   X(n)  = -(1/Omega) sum_{n'' < nocc} qV,   SX(n) = -(1/Omega) sum_{n'' < nocc} qW,
//   CH(n) = (1/(2 Omega)) sum_{n''} (qW - qV),
//   CH_exact(n) = (1/(2 Omega)) sum_{G G'} rho_n(G - G') (W - V)_{G G'},
//            rho_n(D) = <n| e^{i D.r} |n> = sum_{G2} conj(c_n(D + G2)) c_n(G2).
// The 1/Omega is the implicit normalization of a q sum with one q point.
// Plain precision: FP64 throughout.  Mixed precisions: m in FP32 (the
// matrix-element kernels' FP32 path) and W m on the tensor cores (split
// operands, FP32 segment sums, FP64 result); the forms, the sums and the
// closed form in FP64.
#include <algorithm>
#include <vector>

#include "runtime.h"

namespace bgw {

namespace {

constexpr int TQ = 64;   // tile edge (pairs x G)
constexpr int KQ = 16;   // G' per shared-memory slice

// partial[gt][p] = sum_{G in tile gt} conj(m_p(G)) (W m_p)(G); grid (ceil(K/64), ceil(ng/64)).
__global__ void __launch_bounds__(256) sigma_quad_kernel(const double2* __restrict__ M, long long K, int ng,
                                                         const double2* __restrict__ W,
                                                         double2* __restrict__ partial) {
  __shared__ double2 As[KQ][TQ];   // m_p(G') for the tile's pairs
  __shared__ double2 Bs[KQ][TQ];   // W[G][G'] for the tile's G, read as [G'][G]
  __shared__ double2 red[16][TQ + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long p0 = (long long)blockIdx.x * TQ;
  const int g0 = blockIdx.y * TQ;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < ng; k0 += KQ) {
#pragma unroll
    for (int q = 0; q < (KQ * TQ) / 256; ++q) {
      const int e = tid + 256 * q;
      const int r = e / KQ, kk = e % KQ;   // pair row r, G' = k0 + kk
      const long long p = p0 + r;
      As[kk][r] = (p < K && k0 + kk < ng) ? M[p * ng + k0 + kk] : make_double2(0.0, 0.0);
      const int c = e / KQ;                // G column c
      Bs[kk][c] = (g0 + c < ng && k0 + kk < ng) ? W[(size_t)(g0 + c) * ng + k0 + kk] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KQ; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {   // (W m)(G) += W[G][G'] m(G')
          acc[i][j].x = fma(b[j].x, a[i].x, acc[i][j].x);
          acc[i][j].x = fma(-b[j].y, a[i].y, acc[i][j].x);
          acc[i][j].y = fma(b[j].x, a[i].y, acc[i][j].y);
          acc[i][j].y = fma(b[j].y, a[i].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  // conj(m_p(G)) (W m_p)(G), summed over the thread's 4 columns, then over tx
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long p = p0 + ty + 16 * i;
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int g = g0 + tx + 16 * j;
      if (p < K && g < ng) {
        const double2 m = M[p * ng + g];
        sr = fma(m.x, acc[i][j].x, fma(m.y, acc[i][j].y, sr));
        si = fma(m.x, acc[i][j].y, fma(-m.y, acc[i][j].x, si));
      }
    }
    red[tx][ty + 16 * i] = make_double2(sr, si);
  }
  __syncthreads();
  if (tid < TQ) {
    double sr = 0.0, si = 0.0;
    for (int t = 0; t < 16; ++t) {
      sr += red[t][tid].x;
      si += red[t][tid].y;
    }
    const long long p = p0 + tid;
    if (p < K) partial[(size_t)blockIdx.y * K + p] = make_double2(sr, si);
  }
}

// qV_p = sum_G |m_p(G)|^2 v_G (one warp per pair) and qW_p from the partials.
__global__ void sigma_forms_kernel(const double2* __restrict__ M, long long K, int ng, const double* __restrict__ sv,
                                   const double2* __restrict__ partial, int ntg, double* __restrict__ qW,
                                   double* __restrict__ qV) {
  const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= K) return;
  double s = 0.0;
  for (int g = lane; g < ng; g += 32) {
    const double2 m = M[p * ng + g];
    s = fma(fma(m.x, m.x, m.y * m.y), sv[g] * sv[g], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double w = 0.0;
    for (int t = 0; t < ntg; ++t) w += partial[(size_t)t * K + p].x;   // the forms are real (W Hermitian)
    qW[p] = w;
    qV[p] = s;
  }
}

// Mixed precision: qW_p = Re sum_G conj(m_p(G)) C[p][G] with C = (W m_p) from
// the tensor cores and the FP32 m; qV_p = sum_G |m_p(G)|^2 v_G.  One warp per pair.
__global__ void sigma_forms_tc_kernel(const float2* __restrict__ M, long long K, int ng, const double* __restrict__ sv,
                                      const double2* __restrict__ C, double* __restrict__ qW,
                                      double* __restrict__ qV) {
  const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= K) return;
  double w = 0.0, s = 0.0;
  for (int g = lane; g < ng; g += 32) {
    const float2 mf = M[p * ng + g];
    const double mx = mf.x, my = mf.y;
    const double2 cw = C[p * ng + g];
    w = fma(mx, cw.x, fma(my, cw.y, w));
    s = fma(fma(mx, mx, my * my), sv[g] * sv[g], s);
  }
  for (int o = 16; o > 0; o >>= 1) {
    w += __shfl_xor_sync(0xffffffffu, w, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if (lane == 0) {
    qW[p] = w;
    qV[p] = s;
  }
}

// out[0..3][n] from the pair forms.
__global__ void sigma_sums_kernel(const double* __restrict__ qW, const double* __restrict__ qV, int ni, int no,
                                  int nocc, double inv_omega, double* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= no) return;
  double x = 0.0, sx = 0.0, ch = 0.0;
  for (int b = 0; b < ni; ++b) {
    const double w = qW[(size_t)b * no + n], v = qV[(size_t)b * no + n];
    if (b < nocc) {
      x += v;
      sx += w;
    }
    ch += w - v;
  }
  out[n] = -x * inv_omega;
  out[no + n] = -sx * inv_omega;
  out[2 * no + n] = 0.5 * ch * inv_omega;
}

// rho_n(D) for every point D of the difference box, one warp per (point, n);
// omap: outer-sphere index of G in the outer box (or -1).
__global__ void rho_kernel(const double2* __restrict__ co, int npw, const int32_t* __restrict__ go,
                           const int* __restrict__ omap, int3 olo, int3 odim, int3 dlo, int3 ddim, int no,
                           double2* __restrict__ rho) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long npts = (long long)ddim.x * ddim.y * ddim.z;
  if (w >= npts * no) return;
  const int n = (int)(w / npts);
  const long long d = w - (long long)n * npts;
  const int dz = (int)(d % ddim.z), dy = (int)((d / ddim.z) % ddim.y), dx = (int)(d / ((long long)ddim.z * ddim.y));
  const int Dx = dlo.x + dx, Dy = dlo.y + dy, Dz = dlo.z + dz;
  const double2* c = co + (size_t)n * npw;
  double re = 0.0, im = 0.0;
  for (int j = lane; j < npw; j += 32) {
    const int x = go[3 * j] + Dx - olo.x, y = go[3 * j + 1] + Dy - olo.y, z = go[3 * j + 2] + Dz - olo.z;
    if (x < 0 || y < 0 || z < 0 || x >= odim.x || y >= odim.y || z >= odim.z) continue;
    const int k = omap[((size_t)x * odim.y + y) * odim.z + z];
    if (k < 0) continue;
    const double2 a = c[k], b = c[j];   // conj(c(D + G2)) c(G2)
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) rho[w] = make_double2(re, im);
}

// rho[b0 + j][:] = M[j nb + j][:] (the band-diagonal pairs of a chunk).
__global__ void rho_diag_kernel(const double2* __restrict__ M, int nb, long long npts, double2* __restrict__ rho) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * npts) return;
  const int j = (int)(e / npts);
  const long long d = e - (long long)j * npts;
  rho[e] = M[((size_t)j * nb + j) * npts + d];
}

// CH_exact(n) = (1/(2 Omega)) Re sum_{G G'} rho_n(G - G') (W - V)_{G G'}.
// Grid (kChBlocks, ceil(no / kChBands)): each CTA reads its share of W once
// and accumulates kChBands bands; part[band][block] (fixed order, reduced by
// ch_reduce_kernel).
constexpr int kChBlocks = 304;
constexpr int kChBands = 8;

__global__ void __launch_bounds__(256) ch_exact_kernel(const double2* __restrict__ W, const double* __restrict__ sv,
                                                       const int32_t* __restrict__ geps, int ng, int no,
                                                       const double2* __restrict__ rho, int3 dlo, int3 ddim,
                                                       double* __restrict__ part) {
  __shared__ double red[kChBands][8];
  const int n0 = blockIdx.y * kChBands;
  const int nb = min(kChBands, no - n0);
  const long long npts = (long long)ddim.x * ddim.y * ddim.z;
  const long long n2 = (long long)ng * ng;
  const long long per = (n2 + gridDim.x - 1) / gridDim.x;
  const long long e0 = (long long)blockIdx.x * per, e1 = min(n2, e0 + per);
  double s[kChBands];
#pragma unroll
  for (int b = 0; b < kChBands; ++b) s[b] = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += 256) {
    const int i = (int)(e / ng), j = (int)(e - (long long)i * ng);
    const int dx = geps[3 * i] - geps[3 * j] - dlo.x, dy = geps[3 * i + 1] - geps[3 * j + 1] - dlo.y,
              dz = geps[3 * i + 2] - geps[3 * j + 2] - dlo.z;
    const size_t d = ((size_t)dx * ddim.y + dy) * ddim.z + dz;
    double2 w = W[e];
    if (i == j) w.x -= sv[i] * sv[i];
#pragma unroll
    for (int b = 0; b < kChBands; ++b)
      if (b < nb) {
        const double2 rv = rho[(size_t)(n0 + b) * npts + d];
        s[b] = fma(rv.x, w.x, fma(-rv.y, w.y, s[b]));
      }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < kChBands; ++b) {
    double v = s[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[b][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nb) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
    part[(size_t)(n0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void ch_reduce_kernel(const double* __restrict__ part, int nblk, int no, double half_inv_omega,
                                 double* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= no) return;
  double v = 0.0;
  for (int k = 0; k < nblk; ++k) v += part[(size_t)n * nblk + k];
  out[n] = v * half_inv_omega;
}

}  // namespace

int sigma_run(Ctx* c, const bgw_cell* cell, int n, int no, const BandPlan* bpo, const int32_t* go, const void* co,
              int ni, const BandPlan* bpi, const void* ci, int nocc, int ng, const int32_t* geps_host,
              const int32_t* d_geps, const PairPlan* pp_neg, const void* epsinv, int prec, double* sigma_host,
              cudaStream_t st) {
  const long long K = (long long)ni * no;
  const bool mixed = prec != BGW_PREC_FP64;
  Scratch sM, sW, sv, part, q, out, rho, omap, gox, chp;
  sM.pool = sW.pool = sv.pool = part.pool = q.pool = out.pool = rho.pool = omap.pool = gox.pool = chp.pool = &c->pool;
  const int ntg = (ng + TQ - 1) / TQ;
  // difference box of the epsilon list and index box of the outer sphere
  int glo[3], ghi[3], olo[3], ohi[3];
  for (int d = 0; d < 3; ++d) {
    glo[d] = ghi[d] = geps_host[d];
    olo[d] = ohi[d] = go[d];
  }
  for (int i = 0; i < ng; ++i)
    for (int d = 0; d < 3; ++d) {
      glo[d] = std::min(glo[d], geps_host[3 * i + d]);
      ghi[d] = std::max(ghi[d], geps_host[3 * i + d]);
    }
  const int npw_o = bpo->npw;
  for (int i = 0; i < npw_o; ++i)
    for (int d = 0; d < 3; ++d) {
      olo[d] = std::min(olo[d], go[3 * i + d]);
      ohi[d] = std::max(ohi[d], go[3 * i + d]);
    }
  const int3 dlo = make_int3(glo[0] - ghi[0], glo[1] - ghi[1], glo[2] - ghi[2]);
  const int3 ddim = make_int3(2 * (ghi[0] - glo[0]) + 1, 2 * (ghi[1] - glo[1]) + 1, 2 * (ghi[2] - glo[2]) + 1);
  const int3 o3 = make_int3(olo[0], olo[1], olo[2]);
  const int3 odim = make_int3(ohi[0] - olo[0] + 1, ohi[1] - olo[1] + 1, ohi[2] - olo[2] + 1);
  const long long npts = (long long)ddim.x * ddim.y * ddim.z;
  std::vector<int> map((size_t)odim.x * odim.y * odim.z, -1);
  for (int i = 0; i < npw_o; ++i)
    map[((size_t)(go[3 * i] - olo[0]) * odim.y + (go[3 * i + 1] - olo[1])) * odim.z + (go[3 * i + 2] - olo[2])] = i;
  int rc;
  // FP64: partial dot products [ntg][K]; mixed: the product C = W m [K][ng] (FP64)
  const size_t part_bytes = mixed ? (size_t)K * ng * sizeof(double2) : (size_t)ntg * K * sizeof(double2);
  if ((rc = c->pool.alloc((size_t)K * ng * (mixed ? sizeof(float2) : sizeof(double2)), &sM.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)ng * ng * sizeof(double2), &sW.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)ng * sizeof(double), &sv.ptr)) != BGW_OK ||
      (rc = c->pool.alloc(part_bytes, &part.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)2 * K * sizeof(double), &q.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)4 * no * sizeof(double), &out.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)npts * no * sizeof(double2), &rho.ptr)) != BGW_OK ||
      (rc = c->pool.alloc(map.size() * sizeof(int), &omap.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)npw_o * 3 * sizeof(int32_t), &gox.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)no * kChBlocks * sizeof(double), &chp.ptr)) != BGW_OK)
    return fail(c, rc, "bgw_sigma_cohsex: scratch allocation failed");
  BGW_CUDA(c, cudaMemcpyAsync(omap.ptr, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  BGW_CUDA(c, cudaMemcpyAsync(gox.ptr, go, (size_t)npw_o * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  // m_p(G) = M_{n''n}(k, -q, -G): the inner bands take the shifted-sphere role
  if ((rc = mtxel_run(c, n, prec, ni, bpi, ci, no, bpo, co, pp_neg, sM.ptr, st)) != BGW_OK) return rc;
  {
    const int ngv[1] = {ng};
    const bgw_cell* cp[1] = {cell};
    const int32_t* dg[1] = {d_geps};
    const void* ein[1] = {epsinv};
    void* wout[1] = {sW.ptr};
    if ((rc = screened_w_run(c, 1, ngv, cp, dg, ein, wout, st)) != BGW_OK) return rc;
    if ((rc = coulomb_sqrt_run(c, cell, d_geps, ng, sv.as<double>(), st)) != BGW_OK) return rc;
  }
  double* qW = q.as<double>();
  double* qV = qW + K;
  {
    TimedScope ts(c, kTSigmaForms, st);
    if (mixed) {
      // C[p][G] = sum_G' m_p(G') W[G][G'] on the tensor cores
      if ((rc = tc_rows_gemm(c, prec, (int)K, ng, ng, sM.ptr, sW.ptr, part.ptr, st)) != BGW_OK) return rc;
      sigma_forms_tc_kernel<<<(unsigned)((K * 32 + 255) / 256), 256, 0, st>>>(
          sM.as<float2>(), K, ng, sv.as<double>(), part.as<double2>(), qW, qV);
    } else {
      sigma_quad_kernel<<<dim3((unsigned)((K + TQ - 1) / TQ), ntg), 256, 0, st>>>(
          sM.as<double2>(), K, ng, sW.as<double2>(), part.as<double2>());
      sigma_forms_kernel<<<(unsigned)((K * 32 + 255) / 256), 256, 0, st>>>(
          sM.as<double2>(), K, ng, sv.as<double>(), part.as<double2>(), ntg, qW, qV);
    }
    sigma_sums_kernel<<<(no + 127) / 128, 128, 0, st>>>(qW, qV, ni, no, nocc, 1.0 / cell->omega, out.as<double>());
  }
  {
    TimedScope ts(c, kTSigmaExact, st);
    // rho_n(D) = M_{nn}(D): the pair transform of band n with itself onto the
    // difference box, on the smallest supported grid where neither the
    // product's spectrum (extent of the outer sphere's differences) nor the
    // box aliases.  Where no grid qualifies, the direct sum over the sphere.
    int nr = 0;
    for (int cand = n; cand <= 64 && nr == 0 && c->sigma_density != 0; ++cand) {
      if (!fft_size_supported(cand)) continue;
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        const int dl = glo[d] - ghi[d], dh = ghi[d] - glo[d];
        ok = ok && cand > (ohi[d] - olo[d]) + dh && dl >= -(cand / 2) && dh < cand - cand / 2 &&
             olo[d] >= -(cand / 2) && ohi[d] < cand - cand / 2;
      }
      if (ok) nr = cand;
    }
    if (nr > 0) {
      std::vector<int32_t> dlist((size_t)npts * 3);
      size_t e = 0;
      for (int x = 0; x < ddim.x; ++x)
        for (int y = 0; y < ddim.y; ++y)
          for (int z = 0; z < ddim.z; ++z, e += 3) {
            dlist[e] = dlo.x + x;
            dlist[e + 1] = dlo.y + y;
            dlist[e + 2] = dlo.z + z;
          }
      const BandPlan* bpr;
      const PairPlan* ppr;
      if ((rc = get_band_plan(c, nr, npw_o, go, st, &bpr)) != BGW_OK) return rc;
      if ((rc = get_pair_plan(c, nr, (int)npts, dlist.data(), st, &ppr)) != BGW_OK) return rc;
      constexpr int kRhoChunk = 8;
      Scratch mr;
      mr.pool = &c->pool;
      const int nbmax = std::min(no, kRhoChunk);
      if ((rc = c->pool.alloc((size_t)nbmax * nbmax * npts * sizeof(double2), &mr.ptr)) != BGW_OK)
        return fail(c, rc, "bgw_sigma_cohsex: scratch allocation failed");
      for (int b0 = 0; b0 < no; b0 += kRhoChunk) {
        const int nb = std::min(kRhoChunk, no - b0);
        const void* cb = static_cast<const double2*>(co) + (size_t)b0 * npw_o;
        if ((rc = mtxel_run(c, nr, BGW_PREC_FP64, nb, bpr, cb, nb, bpr, cb, ppr, mr.ptr, st)) != BGW_OK) return rc;
        rho_diag_kernel<<<(unsigned)(((long long)nb * npts + 255) / 256), 256, 0, st>>>(
            mr.as<double2>(), nb, npts, rho.as<double2>() + (size_t)b0 * npts);
        c->launches += 1;
      }
    } else {
      rho_kernel<<<(unsigned)((npts * no * 32 + 255) / 256), 256, 0, st>>>(
          static_cast<const double2*>(co), npw_o, gox.as<int32_t>(), omap.as<int>(), o3, odim, dlo, ddim, no,
          rho.as<double2>());
      c->launches += 1;
    }
    ch_exact_kernel<<<dim3(kChBlocks, (no + kChBands - 1) / kChBands), 256, 0, st>>>(
        sW.as<double2>(), sv.as<double>(), d_geps, ng, no, rho.as<double2>(), dlo, ddim, chp.as<double>());
    ch_reduce_kernel<<<(no + 127) / 128, 128, 0, st>>>(chp.as<double>(), kChBlocks, no, 0.5 / cell->omega,
                                                       out.as<double>() + 3 * no);
  }
  BGW_CUDA(c, cudaGetLastError());
  c->launches += mixed ? 4 : 5;
  BGW_CUDA(c, cudaMemcpyAsync(sigma_host, out.ptr, (size_t)4 * no * sizeof(double), cudaMemcpyDeviceToHost, st));
  BGW_CUDA(c, cudaStreamSynchronize(st));
  return BGW_OK;
}

}  // namespace bgw
