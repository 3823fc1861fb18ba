// Host side of the matrix-element step (Eq. eqn_matrix_elem, evaluated by
// the FFT form that follows it): plans of the pruned transforms and the
// scratch layout of one evaluation (kernels in mtxel_kernels.cuh).
#include <algorithm>
#include <map>
#include <vector>

#include "fft.cuh"
#include "runtime.h"

namespace bgw {

bool fft_size_supported(int n) {
  for (int s : kSupportedN)
    if (s == n) return true;
  return false;
}

static inline int wrap(int g, int n) { return ((g % n) + n) % n; }

template <typename V>
static int upload_vec(Ctx* c, const std::vector<V>& v, cudaStream_t st, V** dev) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(1, v.size()) * sizeof(V);
  int rc = c->pool.alloc_keep(bytes, &p);
  if (rc != BGW_OK) return fail(c, rc, "plan upload: device allocation of %zu bytes failed", bytes);
  if (!v.empty()) BGW_CUDA(c, cudaMemcpyAsync(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, st));
  *dev = static_cast<V*>(p);
  return BGW_OK;
}

// Band transform plan: the sphere's (gx,gy) columns with their (gz, index)
// entries, and the distinct gx (the only x columns the y pass must touch).
int get_band_plan(Ctx* c, int n, int npw, const int32_t* g, cudaStream_t st, const BandPlan** out) {
  uint64_t key = hash_bytes(g, (size_t)npw * 3 * sizeof(int32_t), hash_bytes(&n, sizeof(n)));
  auto it = c->band_plans.find(key);
  if (it != c->band_plans.end() && it->second->npw == npw) {
    *out = it->second.get();
    return BGW_OK;
  }
  std::map<int, std::vector<std::pair<int, int>>> cols;  // xy -> (z, idx)
  std::vector<char> xs(n, 0);
  for (int i = 0; i < npw; ++i) {
    int x = wrap(g[3 * i], n), y = wrap(g[3 * i + 1], n), z = wrap(g[3 * i + 2], n);
    cols[y * n + x].push_back({z, i});
    xs[x] = 1;
  }
  auto plan = std::make_unique<BandPlan>();
  plan->n = n;
  plan->npw = npw;
  plan->ncol = (int)cols.size();
  std::vector<int> ent_col, ent_z, ent_idx, col_start, col_xy, xslot;
  int ci = 0;
  for (auto& kv : cols) {
    col_start.push_back((int)ent_col.size());
    col_xy.push_back(kv.first);
    for (auto& e : kv.second) {
      ent_col.push_back(ci);
      ent_z.push_back(e.first);
      ent_idx.push_back(e.second);
    }
    ++ci;
  }
  col_start.push_back((int)ent_col.size());
  for (int x = 0; x < n; ++x)
    if (xs[x]) xslot.push_back(x);
  plan->nxs = (int)xslot.size();
  int rc;
  if ((rc = upload_vec(c, ent_col, st, &plan->d_ent_col)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, ent_z, st, &plan->d_ent_z)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, ent_idx, st, &plan->d_ent_idx)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, col_start, st, &plan->d_col_start)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, col_xy, st, &plan->d_col_xy)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, xslot, st, &plan->d_xslot)) != BGW_OK) return rc;
  *out = plan.get();
  c->band_plans[key] = std::move(plan);
  return BGW_OK;
}

// Pair transform plan: the epsilon sphere's distinct ky (y-pass outputs), its
// (kx,ky) columns (x-pass outputs) and the kz of each column (z-pass outputs
// scattered to the caller's G order).
int get_pair_plan(Ctx* c, int n, int ng, const int32_t* geps, cudaStream_t st, const PairPlan** out) {
  uint64_t key = hash_bytes(geps, (size_t)ng * 3 * sizeof(int32_t), hash_bytes(&n, sizeof(n), 7));
  auto it = c->pair_plans.find(key);
  if (it != c->pair_plans.end() && it->second->ng == ng) {
    *out = it->second.get();
    return BGW_OK;
  }
  std::vector<int> yslot_of_k(n, -1);
  std::map<int, int> colidx;  // y*n + x -> column
  for (int i = 0; i < ng; ++i) {
    int x = wrap(geps[3 * i], n), y = wrap(geps[3 * i + 1], n);
    yslot_of_k[y] = 0;
    colidx.emplace(y * n + x, 0);
  }
  int nys = 0;
  for (int k = 0; k < n; ++k)
    if (yslot_of_k[k] >= 0) yslot_of_k[k] = nys++;
  int ncol = 0;
  for (auto& kv : colidx) kv.second = ncol++;
  std::vector<int> colmap((size_t)n * nys, -1), zmap((size_t)n * ncol, -1);
  for (auto& kv : colidx) {
    int y = kv.first / n, x = kv.first % n;
    colmap[(size_t)x * nys + yslot_of_k[y]] = kv.second;
  }
  for (int i = 0; i < ng; ++i) {
    int x = wrap(geps[3 * i], n), y = wrap(geps[3 * i + 1], n), z = wrap(geps[3 * i + 2], n);
    zmap[(size_t)z * ncol + colidx[y * n + x]] = i;
  }
  auto plan = std::make_unique<PairPlan>();
  plan->n = n;
  plan->ng = ng;
  plan->ncol = ncol;
  plan->nys = nys;
  // The low-band kernels take only the outer quarters k < n/4 and k >= 3n/4
  // of every line: allowed when each kept frequency on each axis is there.
  auto in_band = [n](int k) { return 4 * k < n || 4 * k >= 3 * n; };
  plan->lowband = n % 4 == 0;
  for (int i = 0; i < ng && plan->lowband; ++i)
    for (int d = 0; d < 3; ++d)
      if (!in_band(wrap(geps[3 * i + d], n))) plan->lowband = false;
  int rc;
  if ((rc = upload_vec(c, yslot_of_k, st, &plan->d_yslot_of_k)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, colmap, st, &plan->d_colmap)) != BGW_OK) return rc;
  if ((rc = upload_vec(c, zmap, st, &plan->d_zmap)) != BGW_OK) return rc;
  *out = plan.get();
  c->pair_plans[key] = std::move(plan);
  return BGW_OK;
}

// Upper bound of the pair-transform intermediate T held at once.
static const size_t kPairScratchBytes = size_t(4) << 30;

int mtxel_run(Ctx* c, int n, int prec, int nv, const BandPlan* bpv, const void* cv, int nc,
              const BandPlan* bpc, const void* cc, const PairPlan* pp, void* M, cudaStream_t st, bool real) {
  const size_t cs = prec == BGW_PREC_FP64 ? 16 : 8;
  const size_t n3 = (size_t)n * n * n;
  const long long npairs = (long long)nv * nc;
  const size_t per_pair = (size_t)n * pp->ncol * cs;
  long long pb = (long long)(kPairScratchBytes / per_pair);
  if (pb < 1) pb = 1;
  if (pb > npairs) pb = npairs;
  Scratch uv, uc, U1, T;
  uv.pool = uc.pool = U1.pool = T.pool = &c->pool;
  int rc;
  const int ncolmax = std::max(bpv->ncol, bpc->ncol);
  const int nbmax = std::max(nv, nc);
  if ((rc = c->pool.alloc(nv * n3 * cs, &uv.ptr)) != BGW_OK ||
      (rc = c->pool.alloc(nc * n3 * cs, &uc.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)nbmax * n * ncolmax * cs, &U1.ptr)) != BGW_OK ||
      (rc = c->pool.alloc((size_t)pb * per_pair, &T.ptr)) != BGW_OK)
    return fail(c, rc, "bgw_mtxel: scratch allocation failed (grids %zu B, intermediate %zu B)",
                (size_t)(nv + nc) * n3 * cs, (size_t)pb * per_pair);
  MtxelExec x;
  x.n = n;
  x.nv = nv;
  x.nc = nc;
  x.bpv = bpv;
  x.bpc = bpc;
  x.pp = pp;
  x.cv = cv;
  x.cc = cc;
  x.real = real ? 1 : 0;
  x.uv = uv.ptr;
  x.uc = uc.ptr;
  x.U1 = U1.ptr;
  x.T = T.ptr;
  x.pair_block = (int)pb;
  x.M = M;
  x.st = st;
  x.launches = &c->launches;
  x.ctx = c;
  // Pairs per pair_yxpass block: autotuned once per shape, or the default
  // (as many pairs as 256 threads hold) when tuning is off.
  const int ppb_default = std::max(1, 256 / n);
  int* slot = &c->tuned_ppb[std::make_tuple(n, prec == BGW_PREC_FP64 ? 0 : 1, pp->nys, pp->ncol)];
  if (!c->autotune && *slot <= 0) *slot = ppb_default;
  int forced = 0;   // a kernel chosen by BGW_OPT_PAIR_KERNEL (the table is left alone)
  if (c->pair_kernel >= 0) {
    forced = c->pair_kernel == 0 ? ppb_default : kPairWarpCode;
    slot = &forced;
  }
  x.tuned_ppb = slot;
  cudaError_t e = prec == BGW_PREC_FP64 ? mtxel_exec_f64(x) : mtxel_exec_f32(x);
  if (e != cudaSuccess) return cuda_fail(c, e, "bgw_mtxel kernels");
  return BGW_OK;
}

}  // namespace bgw
