// Head and wings of chi at a small q0 for the mixed precisions.
//
// The q -> 0 limit is evaluated at a small q0 (Section "RPA Dielectric
// Matrix: epsilon": about 1/1000 of the zone, on a shifted grid).  There
// M_vc(G = 0) = <u_v(k+q0)|u_c(k)> is O(|q0|) while v(q0 + 0) = 4 pi/|q0|^2,
// and v(q0) chi_00 is O(1): the macroscopic response.  Single-precision FFTs
// leave absolute errors near 2^-24 |M_vc| on every G, i.e. a relative error
// near 2^-24 / |q0| on the head column, which eps~ inherits at full size.
// The mixed precisions therefore take the head column in FP64 directly from
// its definition (Eq. eqn_matrix_elem at G = 0, the convolution reduced to
// one dot product over the plane waves both spheres hold):
//   h_p = sum_{G in S_c} conj(c_v(G)) c_c(G)
// zero that column of M before the tensor-core chi, and add the head and the
// wings back in FP64:
//   chi[g0][G'] += scale sum_p w_p conj(h_p) M[p][G']   (G' != g0; mirrored)
//   chi[g0][g0] += scale sum_p w_p |h_p|^2
// Deterministic: fixed pair splits, partial sums reduced in a fixed order.
#include <cmath>
#include <unordered_map>

#include "runtime.h"

namespace bgw {

namespace {

// One warp per pair p = v * nc + c.  map[j] = index in the valence list of
// the conduction sphere's j-th G, or -1 when the valence sphere lacks it.
__global__ void head_dot_kernel(const double2* __restrict__ cv, int npw_v, const double2* __restrict__ cc,
                                int npw_c, const int32_t* __restrict__ map, int nc, long long K, int ng, int g0,
                                double2* __restrict__ h, float2* __restrict__ M) {
  const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= K) return;
  const int v = (int)(p / nc), c = (int)(p - (long long)v * nc);
  const double2* a = cv + (size_t)v * npw_v;
  const double2* b = cc + (size_t)c * npw_c;
  double re = 0.0, im = 0.0;
  for (int j = lane; j < npw_c; j += 32) {
    const int iv = map[j];
    if (iv < 0) continue;
    const double2 x = a[iv], y = b[j];
    re = fma(x.x, y.x, fma(x.y, y.y, re));   // conj(x) y
    im = fma(x.x, y.y, fma(-x.y, y.x, im));
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    h[p] = make_double2(re, im);
    M[(size_t)p * ng + g0] = make_float2(0.f, 0.f);
  }
}

constexpr int kWingThreads = 128;

// a[f][p] = w_f[p] conj(h_p) in FP32 (hi) plus the head term in FP64.
// part[f][s][G'] = sum_{p in split s} a[f][p] M_p(G') for G' != g0, the
// products in FP32 (M itself holds FP32 values) and the sum compensated
// (two-sum), so the wing carries the relative precision of M; at G' = g0
// the split sums w |h|^2 in FP64.  Grid (column tiles, splits, nrow).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  const float t = s + x;
  const float z = t - s;
  e += (s - (t - z)) + (x - z);
  s = t;
}

__global__ void __launch_bounds__(kWingThreads) head_wing_partial_kernel(
    const float2* __restrict__ M, const double2* __restrict__ h, const double* __restrict__ w, long long K, int ng,
    int g0, long long per_split, double2* __restrict__ part) {
  __shared__ float2 a_s[256];
  const int gp = blockIdx.x * kWingThreads + threadIdx.x;
  const int s = blockIdx.y, f = blockIdx.z;
  const long long p0 = (long long)s * per_split;
  const long long p1 = p0 + per_split < K ? p0 + per_split : K;
  const double* wf = w + (size_t)f * K;
  float re = 0.f, rec = 0.f, im = 0.f, imc = 0.f;
  double hre = 0.0;
  for (long long q0 = p0; q0 < p1; q0 += 256) {
    const int cnt = (int)(p1 - q0 < 256 ? p1 - q0 : 256);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += kWingThreads) {
      const double2 hp = h[q0 + t];
      const double wp = wf[q0 + t];
      a_s[t] = make_float2((float)(wp * hp.x), (float)(-wp * hp.y));   // w conj(h)
    }
    __syncthreads();
    if (gp < ng) {
      if (gp == g0) {
        for (int t = 0; t < cnt; ++t) {
          const double2 hp = h[q0 + t];
          hre = fma(wf[q0 + t], fma(hp.x, hp.x, hp.y * hp.y), hre);
        }
      } else {
        const float2* mp = M + (size_t)q0 * ng + gp;
        for (int t = 0; t < cnt; ++t) {
          const float2 m = mp[(size_t)t * ng];
          const float2 a = a_s[t];
          two_sum_acc(re, rec, fmaf(a.x, m.x, -a.y * m.y));
          two_sum_acc(im, imc, fmaf(a.x, m.y, a.y * m.x));
        }
      }
    }
  }
  if (gp < ng)
    part[((size_t)f * gridDim.y + s) * ng + gp] =
        gp == g0 ? make_double2(hre, 0.0) : make_double2((double)re + (double)rec, (double)im + (double)imc);
}

__global__ void head_wing_apply_kernel(const double2* __restrict__ part, int nsplit, int ng, int g0, double scale,
                                       double2* __restrict__ chi) {
  const int gp = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (gp >= ng) return;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    const double2 x = part[((size_t)f * nsplit + s) * ng + gp];
    re += x.x;
    im += x.y;
  }
  double2* cf = chi + (size_t)f * ng * ng;
  if (gp == g0) {
    double2& d = cf[(size_t)g0 * ng + g0];
    d.x += scale * re;   // sum_p w_p |h_p|^2 is real
    return;
  }
  double2& r = cf[(size_t)g0 * ng + gp];
  r.x += scale * re;
  r.y += scale * im;
  double2& c = cf[(size_t)gp * ng + g0];
  c.x += scale * re;
  c.y -= scale * im;
}

}  // namespace

int head_prepare(Ctx* c, const bgw_cell* cell, int npw_v, const int32_t* gv, int npw_c, const int32_t* gc, int ng,
                 const int32_t* geps, int prec, cudaStream_t st, HeadPlan* out) {
  out->g0 = -1;
  out->d_map = nullptr;
  out->npw_c = npw_c;
  if (prec == BGW_PREC_FP64 || c->head_mode == 0) return BGW_OK;
  int g0 = -1;
  for (int i = 0; i < ng && g0 < 0; ++i)
    if (geps[3 * i] == 0 && geps[3 * i + 1] == 0 && geps[3 * i + 2] == 0) g0 = i;
  if (g0 < 0) return BGW_OK;
  if (c->head_mode == -1) {
    // Automatic: where v(q + 0) diverges (bulk, slab) and |q| < 0.02 min |b_i|.
    if (cell->coulomb == BGW_COULOMB_SPHERE) return BGW_OK;
    double q2 = 0.0, bmin = INFINITY;
    for (int d = 0; d < 3; ++d) {
      double kd = 0.0, bb = 0.0;
      for (int a = 0; a < 3; ++a) {
        kd += cell->q_frac[a] * cell->bvec[a][d];
        bb += cell->bvec[d][a] * cell->bvec[d][a];
      }
      q2 += kd * kd;
      bmin = std::fmin(bmin, std::sqrt(bb));
    }
    if (!(std::sqrt(q2) < 0.02 * bmin)) return BGW_OK;
  }
  const uint64_t key = hash_bytes(gc, (size_t)npw_c * 12, hash_bytes(gv, (size_t)npw_v * 12, hash_bytes(&npw_c, sizeof(int))));
  auto it = c->head_maps.find(key);
  if (it == c->head_maps.end()) {
    std::unordered_map<uint64_t, int> index;
    index.reserve((size_t)npw_v * 2);
    auto pack = [](const int32_t* g) {
      return ((uint64_t)(uint32_t)(g[0] + (1 << 20)) << 42) | ((uint64_t)(uint32_t)(g[1] + (1 << 20)) << 21) |
             (uint64_t)(uint32_t)(g[2] + (1 << 20));
    };
    for (int i = 0; i < npw_v; ++i) index.emplace(pack(gv + 3 * i), i);
    std::vector<int32_t> map(npw_c);
    for (int j = 0; j < npw_c; ++j) {
      auto f = index.find(pack(gc + 3 * j));
      map[j] = f == index.end() ? -1 : f->second;
    }
    const void* d;
    int rc = upload_cached(c, map.data(), map.size() * sizeof(int32_t), st, &d);
    if (rc != BGW_OK) return rc;
    it = c->head_maps.emplace(key, static_cast<const int32_t*>(d)).first;
  }
  out->g0 = g0;
  out->d_map = it->second;
  return BGW_OK;
}

int head_dot(Ctx* c, const HeadPlan* hp, int nv, const void* cv, int npw_v, int nc, const void* cc, int ng,
             void* M, double2* h, cudaStream_t st) {
  const long long K = (long long)nv * nc;
  const long long threads = K * 32;
  TimedScope ts(c, kTHeadDot, st);
  head_dot_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      static_cast<const double2*>(cv), npw_v, static_cast<const double2*>(cc), hp->npw_c, hp->d_map, nc, K, ng,
      hp->g0, h, static_cast<float2*>(M));
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 1;
  return BGW_OK;
}

int head_wings(Ctx* c, const HeadPlan* hp, long long K, int ng, const void* M, const double2* h, const double* w,
               int nrow, double scale, void* chi, cudaStream_t st) {
  const int tiles = (ng + kWingThreads - 1) / kWingThreads;
  // About two waves of 152 SMs over (tiles x splits), at least 64 pairs per split.
  long long nsplit = std::max<long long>(1, std::min<long long>((2 * 152 * 8) / std::max(1, tiles), K / 64));
  nsplit = std::min<long long>(nsplit, 1024);
  const long long per = (K + nsplit - 1) / nsplit;
  nsplit = (K + per - 1) / per;
  Scratch part;
  part.pool = &c->pool;
  int rc = c->pool.alloc((size_t)nrow * nsplit * ng * sizeof(double2), &part.ptr);
  if (rc != BGW_OK) return fail(c, rc, "chi head: scratch allocation failed");
  TimedScope ts(c, kTHeadWings, st);
  head_wing_partial_kernel<<<dim3((unsigned)tiles, (unsigned)nsplit, (unsigned)nrow), kWingThreads, 0, st>>>(
      static_cast<const float2*>(M), h, w, K, ng, hp->g0, per, part.as<double2>());
  head_wing_apply_kernel<<<dim3((unsigned)((ng + 127) / 128), (unsigned)nrow), 128, 0, st>>>(
      part.as<double2>(), (int)nsplit, ng, hp->g0, scale, static_cast<double2*>(chi));
  BGW_CUDA(c, cudaGetLastError());
  c->launches += 2;
  return BGW_OK;
}

}  // namespace bgw
