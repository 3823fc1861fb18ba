// extern "C" entry points declared in include/bgw.h: argument checks, plan
// lookup, scratch management and the order of the kernel launches.
#include <cstddef>
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <string>

#include <algorithm>
#include <new>
#include <set>
#include <tuple>
#include <functional>
#include <vector>

#include "runtime.h"

using namespace bgw;

namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

Ctx* impl(bgw_ctx* c) { return c ? &c->impl : nullptr; }

// The Python binding mirrors this layout field by field.
static_assert(offsetof(bgw_cell, fft) == 104 && offsetof(bgw_cell, coulomb) == 116 &&
                  offsetof(bgw_cell, coulomb_cut) == 120 && sizeof(bgw_cell) == 128,
              "bgw_cell layout");

int check_cell(Ctx* c, const bgw_cell* cell, int* n) {
  if (!cell) return fail(c, BGW_EINVAL, "cell is NULL");
  if (cell->fft[0] != cell->fft[1] || cell->fft[1] != cell->fft[2])
    return fail(c, BGW_EUNSUPPORTED, "FFT grid %dx%dx%d: only cubic grids are implemented", cell->fft[0],
                cell->fft[1], cell->fft[2]);
  if (!fft_size_supported(cell->fft[0]))
    return fail(c, BGW_EUNSUPPORTED, "FFT grid %d has no kernel (supported: 8 10 12 16 20 24 30 32 36 40 48 50 60 64)",
                cell->fft[0]);
  if (!(cell->omega > 0.0) || !isfinite(cell->omega)) return fail(c, BGW_EINVAL, "cell volume must be > 0");
  *n = cell->fft[0];
  return BGW_OK;
}

// G components in [-n/2, n/2), no duplicates; returns max |G_d| per axis.
int check_glist(Ctx* c, const char* name, int cnt, const int32_t* g, int n, int gmax[3]) {
  if (cnt <= 0) return fail(c, BGW_EINVAL, "%s: count must be >= 1", name);
  if (!g) return fail(c, BGW_EINVAL, "%s is NULL", name);
  const int lo = -(n / 2), hi = n - n / 2;  // [lo, hi)
  gmax[0] = gmax[1] = gmax[2] = 0;
  std::vector<int64_t> keys(cnt);
  for (int i = 0; i < cnt; ++i) {
    for (int d = 0; d < 3; ++d) {
      const int v = g[3 * i + d];
      if (v < lo || v >= hi)
        return fail(c, BGW_EINVAL, "%s[%d] component %d = %d outside [-n/2, n/2) for n = %d", name, i, d, v, n);
      gmax[d] = std::max(gmax[d], std::abs(v));
    }
    keys[i] = ((int64_t)(g[3 * i] - lo) * n + (g[3 * i + 1] - lo)) * n + (g[3 * i + 2] - lo);
  }
  std::sort(keys.begin(), keys.end());
  if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
    return fail(c, BGW_EINVAL, "%s holds a duplicate G vector", name);
  return BGW_OK;
}

int check_energies(Ctx* c, int nv, const double* ev, int nc, const double* ec) {
  if (!ev || !ec) return fail(c, BGW_EINVAL, "energies are NULL");
  for (int i = 0; i < nv; ++i)
    if (!isfinite(ev[i]) || (i && ev[i] < ev[i - 1])) return fail(c, BGW_EINVAL, "ev must be finite and ascending");
  for (int i = 0; i < nc; ++i)
    if (!isfinite(ec[i]) || (i && ec[i] < ec[i - 1])) return fail(c, BGW_EINVAL, "ec must be finite and ascending");
  if (!(ev[nv - 1] < ec[0]))
    return fail(c, BGW_EINVAL, "Delta = E_v - E_c must be < 0 for every pair (max ev %g >= min ec %g)",
                ev[nv - 1], ec[0]);
  return BGW_OK;
}

int check_real_axis(Ctx* c, int nfreq, const double* energy, double delta, int advanced) {
  if (nfreq <= 0 || !energy) return fail(c, BGW_EINVAL, "real axis: need nfreq >= 1 frequencies");
  for (int f = 0; f < nfreq; ++f)
    if (!isfinite(energy[f])) return fail(c, BGW_EINVAL, "energy[%d] is not finite", f);
  if (!(delta > 0.0) || !isfinite(delta)) return fail(c, BGW_EINVAL, "broadening delta must be finite and > 0");
  if (advanced != 0 && advanced != 1) return fail(c, BGW_EINVAL, "advanced must be 0 (retarded) or 1");
  return BGW_OK;
}

int check_prec(Ctx* c, int prec) {
  if (prec != BGW_PREC_FP64 && prec != BGW_PREC_MIX_FP16 && prec != BGW_PREC_MIX_BF16)
    return fail(c, BGW_EINVAL, "unknown precision %d", prec);
  return BGW_OK;
}

// Splits a precision argument into the precision and the real-flavor flag.
int split_flavor(Ctx* c, int* prec, bool* real) {
  *real = (*prec & BGW_FLAVOR_REAL) != 0;
  *prec &= ~BGW_FLAVOR_REAL;
  return check_prec(c, *prec);
}

int check_q(Ctx* c, const bgw_cell* cell, int ng, const int32_t* geps) {
  int what, bad;
  if (coulomb_check(cell, ng, geps, &what, &bad) == BGW_OK) return BGW_OK;
  if (what == 1) return fail(c, BGW_EINVAL, "unknown Coulomb model %d", cell->coulomb);
  if (what == 2) return fail(c, BGW_EINVAL, "Coulomb cut length %g must be finite and > 0", cell->coulomb_cut);
  return fail(c, BGW_EINVAL, "|q+G| = 0 at geps[%d]: the %s Coulomb factor diverges", bad,
              cell->coulomb == BGW_COULOMB_SLAB ? "slab-truncated" : "bare");
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Largest epsilon sphere the gather kernel can hold in shared memory.
int max_ng(int prec) { return (int)((227 * 1024) / (prec == BGW_PREC_FP64 ? 16 : 8)); }

int validate_mtxel(Ctx* c, const bgw_cell* cell, int nv, int npw_v, const int32_t* gv, const void* cv, int nc,
                   int npw_c, const int32_t* gc, const void* cc, int ng, const int32_t* geps, int prec, void* M,
                   int* n_out) {
  int n, rc;
  if ((rc = check_cell(c, cell, &n)) != BGW_OK) return rc;
  if ((rc = check_prec(c, prec)) != BGW_OK) return rc;
  if (nv <= 0 || nc <= 0) return fail(c, BGW_EINVAL, "nv and nc must be >= 1");
  if (nv > 65535 || nc > 65535) return fail(c, BGW_EUNSUPPORTED, "at most 65535 bands per side");
  if ((long long)nv * nc > 0x7fffffffLL) return fail(c, BGW_EUNSUPPORTED, "nv * nc exceeds 2^31 - 1");
  if (!cv || !cc || !M) return fail(c, BGW_EINVAL, "coefficient or output pointer is NULL");
  if (ng > max_ng(prec)) return fail(c, BGW_EUNSUPPORTED, "ng = %d exceeds %d for this precision", ng, max_ng(prec));
  int mv[3], mc[3], me[3];
  if ((rc = check_glist(c, "gv", npw_v, gv, n, mv)) != BGW_OK) return rc;
  if ((rc = check_glist(c, "gc", npw_c, gc, n, mc)) != BGW_OK) return rc;
  if ((rc = check_glist(c, "geps", ng, geps, n, me)) != BGW_OK) return rc;
  for (int d = 0; d < 3; ++d)
    if (n <= mv[d] + mc[d] + me[d])
      return fail(c, BGW_EINVAL,
                  "FFT grid %d aliases on axis %d: need n > max|Gv| + max|Gc| + max|Geps| = %d + %d + %d", n, d,
                  mv[d], mc[d], me[d]);
  *n_out = n;
  return BGW_OK;
}

// Runs body (launches on st and streams forked from it) directly the first
// time a key is seen -- plans, tuning and pool blocks are made then -- and
// captures a second, unexecuted pass into a CUDA graph; later calls with the
// key replay the graph.  Pool blocks handed out during the capture stay
// pinned for the graph's life.  With BGW_OPT_TIMING on, or on the legacy
// default stream (not capturable), every call runs directly.
int run_graphed(Ctx* c, uint64_t key, cudaStream_t st, const std::function<int()>& body) {
  if (!c->use_graphs || c->timing.on || st == nullptr || st == cudaStreamLegacy) return body();
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    BGW_CUDA(c, cudaGraphLaunch(it->second.exec, st));
    c->launches += it->second.kernels;
    c->graph_replays += 1;
    return BGW_OK;
  }
  int rc = body();
  if (rc != BGW_OK) return rc;
  if (c->graphs.size() >= kMaxGraphs) return BGW_OK;   // no more pinned scratch: run directly
  c->pool.set_pinning(true);
  const uint64_t l0 = c->launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = body();
    e = cudaStreamEndCapture(st, &graph);
  }
  c->pool.set_pinning(false);
  const uint64_t captured = c->launches - l0;
  c->launches = l0;  // captured launches did not run
  if (e != cudaSuccess || rc != BGW_OK || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    c->pool.abandon_pins();   // no graph refers to them
    c->err.clear();
    return BGW_OK;  // the direct run's results stand; the next call runs directly again
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->pool.abandon_pins();
    return BGW_OK;
  }
  c->graphs[key].exec = exec;
  c->graphs[key].kernels = captured;
  return BGW_OK;
}

// The mixed precisions invert with the tensor-core trailing update unless
// BGW_OPT_INVERSE selects otherwise; the plain FP64 path uses FP64 FMA.
bool use_tc_inverse(Ctx* c, int prec) {
  if (c->inverse_mode == 0) return false;
  if (c->inverse_mode == 1) return true;
  return prec != BGW_PREC_FP64;
}

// Precision of the tensor-core inverse for a call of precision prec: seven
// slices (FP64-level updates, near 2^-48) unless the option asks for five
// (near 2^-34); the mixed precisions take the next diagonal block and the
// panel product in double FP32 (about 2^-46), FP64 inputs in FP64.
// Recorded in the context for the inverse that follows.
void set_run_slices(Ctx* c, int prec) {
  c->run_slices = c->update_slices ? c->update_slices : 7;
  c->run_ff_chain = c->double_fp32 == 1 || (c->double_fp32 == -1 && prec != BGW_PREC_FP64) || c->run_slices < 7;
}

int init_device(Ctx* c) {
  if (c->twiddles_ready) return BGW_OK;
  BGW_CUDA(c, mtxel_init_f64());
  BGW_CUDA(c, mtxel_init_f32());
  c->twiddles_ready = true;
  return BGW_OK;
}

}  // namespace

extern "C" {

int bgw_create(bgw_ctx** out, int device, uint64_t hbm_budget_bytes) {
  if (!out) return BGW_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BGW_ECUDA;
  }
  DeviceGuard g(device);
  if (!g.ok) return BGW_ECUDA;
  bgw_ctx* c = new (std::nothrow) bgw_ctx(hbm_budget_bytes);
  if (!c) return BGW_ENOMEM;
  c->impl.device = device;
  if (cudaMalloc(&c->impl.d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->impl.d_status, 0, sizeof(int)) != cudaSuccess || init_device(&c->impl) != BGW_OK) {
    cudaGetLastError();
    if (c->impl.d_status) cudaFree(c->impl.d_status);
    delete c;
    return BGW_ECUDA;
  }
  *out = c;
  return BGW_OK;
}

int bgw_destroy(bgw_ctx* ctx) {
  if (!ctx) return BGW_EINVAL;
  DeviceGuard g(ctx->impl.device);
  cudaDeviceSynchronize();
  timing_collect(&ctx->impl);
  for (cudaEvent_t e : ctx->impl.timing.free_events) cudaEventDestroy(e);
  for (auto& kv : ctx->impl.graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (ctx->impl.side) cudaStreamDestroy(ctx->impl.side);
  for (cudaEvent_t e : ctx->impl.la_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->impl.copy_st) cudaStreamDestroy(ctx->impl.copy_st);
  for (cudaEvent_t e : ctx->impl.copy_ev)
    if (e) cudaEventDestroy(e);
  ctx->impl.graphs.clear();
  ctx->impl.pool.unpin_all();
  cudaFree(ctx->impl.d_status);
  delete ctx;
  return BGW_OK;
}

const char* bgw_last_error(bgw_ctx* ctx) {
  if (!ctx) return "context is NULL";
  return ctx->impl.err.c_str();
}

int bgw_sync(bgw_ctx* ctx, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BGW_CUDA(c, cudaStreamSynchronize(st));
  int s = 0;
  BGW_CUDA(c, cudaMemcpy(&s, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (s != kDevOk) {
    BGW_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (s == kDevZeroPivot) return fail(c, BGW_ENUMERIC, "zero or non-finite pivot in the inversion");
    if (s == kDevTimeout) return fail(c, BGW_ETIMEOUT, "a bounded device wait gave up");
    return fail(c, BGW_ECUDA, "device status %d", s);
  }
  return BGW_OK;
}

int bgw_mem_stats(bgw_ctx* ctx, uint64_t* in_use, uint64_t* high_water) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (in_use) *in_use = c->pool.in_use();
  if (high_water) *high_water = c->pool.high_water();
  return BGW_OK;
}

int bgw_launch_count(bgw_ctx* ctx, uint64_t* launches) {
  Ctx* c = impl(ctx);
  if (!c || !launches) return BGW_EINVAL;
  *launches = c->launches;
  return BGW_OK;
}

int bgw_graph_stats(bgw_ctx* ctx, uint64_t* graphs, uint64_t* replays) {
  Ctx* c = impl(ctx);
  if (!c || !graphs || !replays) return BGW_EINVAL;
  uint64_t n = 0;
  for (const auto& kv : c->graphs) n += kv.second.exec ? 1 : 0;
  *graphs = n;
  *replays = c->graph_replays;
  return BGW_OK;
}

int bgw_set_option(bgw_ctx* ctx, int option, int64_t value) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (option == BGW_OPT_CHI_SEGMENT_PAIRS) {
    if (value < 0 || value > (1 << 24)) return fail(c, BGW_EINVAL, "segment pairs must be in [0, 2^24]");
    if (value > 0 && value < 32) return fail(c, BGW_EINVAL, "segment pairs must be >= 32");
    c->chi_segment_pairs = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_CHI_CHUNK_PAIRS) {
    if (value < 0 || value > (1 << 30)) return fail(c, BGW_EINVAL, "chunk pairs must be in [0, 2^30]");
    c->chi_chunk_pairs = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_INVERSE) {
    if (value < -1 || value > 1) return fail(c, BGW_EINVAL, "inverse mode is -1, 0 or 1");
    c->inverse_mode = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_DOUBLE_FP32) {
    if (value < -1 || value > 1) return fail(c, BGW_EINVAL, "double-FP32 mode is -1, 0 or 1");
    c->double_fp32 = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_UPDATE_SLICES) {
    if (value != 0 && value != 5 && value != 7) return fail(c, BGW_EINVAL, "update slices are 0, 5 or 7");
    c->update_slices = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_SIGMA_DENSITY) {
    if (value < -1 || value > 1) return fail(c, BGW_EINVAL, "density mode is -1, 0 or 1");
    c->sigma_density = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_HEAD) {
    if (value < -1 || value > 1) return fail(c, BGW_EINVAL, "head mode is -1, 0 or 1");
    c->head_mode = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_AUTOTUNE) {
    if (value != 0 && value != 1) return fail(c, BGW_EINVAL, "autotune is 0 or 1");
    c->autotune = value == 1;
    return BGW_OK;
  }
  if (option == BGW_OPT_PAIR_KERNEL) {
    if (value < -1 || value > 1) return fail(c, BGW_EINVAL, "pair kernel is -1, 0 or 1");
    c->pair_kernel = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_UPDATE_ITEMS) {
    if (value < -1 || value > 1) return fail(c, BGW_EINVAL, "update items are -1, 0 or 1");
    c->update_items = (int)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_WAIT_LIMIT_NS) {
    if (value < 0 || value > 10000000000LL) return fail(c, BGW_EINVAL, "wait limit must be in [0, 1e10] ns");
    c->wait_ns = (unsigned long long)value;
    return BGW_OK;
  }
  if (option == BGW_OPT_TIMING) {
    if (value != 0 && value != 1) return fail(c, BGW_EINVAL, "timing is 0 or 1");
    c->timing.on = value == 1;
    return BGW_OK;
  }
  return fail(c, BGW_EINVAL, "unknown option %d", option);
}

int bgw_timing_report(bgw_ctx* ctx, char* buf, size_t len, int reset) {
  Ctx* c = impl(ctx);
  if (!c || !buf || len == 0) return BGW_EINVAL;
  DeviceGuard g(c->device);
  timing_collect(c);
  std::string out = "{";
  bool first = true;
  for (auto& kv : c->timing.acc) {
    char item[160];
    snprintf(item, sizeof(item), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", timed_name(kv.first),
             kv.second.first, kv.second.second);
    out += item;
    first = false;
  }
  out += "}";
  snprintf(buf, len, "%s", out.c_str());
  if (reset) c->timing.acc.clear();
  return BGW_OK;
}

int bgw_mtxel(bgw_ctx* ctx, const bgw_cell* cell, int nv, int npw_v, const int32_t* gv, const void* cv, int nc,
              int npw_c, const int32_t* gc, const void* cc, int ng, const int32_t* geps, int prec, void* M,
              void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  int n, rc;
  bool real;
  if ((rc = split_flavor(c, &prec, &real)) != BGW_OK) return rc;
  if ((rc = validate_mtxel(c, cell, nv, npw_v, gv, cv, nc, npw_c, gc, cc, ng, geps, prec, M, &n)) != BGW_OK)
    return rc;
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const BandPlan *bpv, *bpc;
  const PairPlan* pp;
  if ((rc = get_band_plan(c, n, npw_v, gv, st, &bpv)) != BGW_OK) return rc;
  if ((rc = get_band_plan(c, n, npw_c, gc, st, &bpc)) != BGW_OK) return rc;
  if ((rc = get_pair_plan(c, n, ng, geps, st, &pp)) != BGW_OK) return rc;
  return mtxel_run(c, n, prec, nv, bpv, cv, nc, bpc, cc, pp, M, st, real);
}

int bgw_chi_sum(bgw_ctx* ctx, const bgw_cell* cell, int nv, int nc, int ng, const void* M, const double* ev,
                const double* ec, int nfreq, const double* omega, int prec, int accumulate, void* chi,
                void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  int rc;
  bool real;
  if (!cell || !(cell->omega > 0.0)) return fail(c, BGW_EINVAL, "cell is NULL or has no volume");
  if ((rc = split_flavor(c, &prec, &real)) != BGW_OK) return rc;
  if (nv <= 0 || nc <= 0 || ng <= 0) return fail(c, BGW_EINVAL, "nv, nc, ng must be >= 1");
  if (!M || !chi) return fail(c, BGW_EINVAL, "M or chi is NULL");
  if (nfreq < 0 || (nfreq > 0 && !omega)) return fail(c, BGW_EINVAL, "bad frequency list");
  for (int f = 0; f < nfreq; ++f)
    if (!isfinite(omega[f])) return fail(c, BGW_EINVAL, "omega[%d] is not finite", f);
  if ((rc = check_energies(c, nv, ev, nc, ec)) != BGW_OK) return rc;
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const void *dev_ev, *dev_ec, *dev_om = nullptr;
  if ((rc = upload_cached(c, ev, nv * sizeof(double), st, &dev_ev)) != BGW_OK) return rc;
  if ((rc = upload_cached(c, ec, nc * sizeof(double), st, &dev_ec)) != BGW_OK) return rc;
  if (nfreq > 0 && (rc = upload_cached(c, omega, nfreq * sizeof(double), st, &dev_om)) != BGW_OK) return rc;
  return chi_run(c, prec, nv, nc, ng, M, static_cast<const double*>(dev_ev), static_cast<const double*>(dev_ec),
                 nfreq, static_cast<const double*>(dev_om), 4.0 / cell->omega, accumulate, chi, st, nullptr, nullptr,
                 real);
}

int bgw_chi_sum_real(bgw_ctx* ctx, const bgw_cell* cell, int nv, int nc, int ng, const void* M, const double* ev,
                     const double* ec, int nfreq, const double* energy, double delta, int advanced, int prec,
                     int accumulate, void* chi, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  int rc;
  if (!cell || !(cell->omega > 0.0)) return fail(c, BGW_EINVAL, "cell is NULL or has no volume");
  if (prec & BGW_FLAVOR_REAL)
    return fail(c, BGW_EUNSUPPORTED, "the real-axis response has complex chi: no real flavor");
  if ((rc = check_prec(c, prec)) != BGW_OK) return rc;
  if (nv <= 0 || nc <= 0 || ng <= 0) return fail(c, BGW_EINVAL, "nv, nc, ng must be >= 1");
  if (!M || !chi) return fail(c, BGW_EINVAL, "M or chi is NULL");
  if ((rc = check_real_axis(c, nfreq, energy, delta, advanced)) != BGW_OK) return rc;
  if ((rc = check_energies(c, nv, ev, nc, ec)) != BGW_OK) return rc;
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const void *dev_ev, *dev_ec, *dev_e;
  if ((rc = upload_cached(c, ev, nv * sizeof(double), st, &dev_ev)) != BGW_OK) return rc;
  if ((rc = upload_cached(c, ec, nc * sizeof(double), st, &dev_ec)) != BGW_OK) return rc;
  if ((rc = upload_cached(c, energy, nfreq * sizeof(double), st, &dev_e)) != BGW_OK) return rc;
  return chi_real_run(c, prec, nv, nc, ng, M, static_cast<const double*>(dev_ev), static_cast<const double*>(dev_ec),
                      nfreq, static_cast<const double*>(dev_e), delta, advanced, 4.0 / cell->omega, accumulate, chi,
                      st);
}

int bgw_epsinv_general(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng, const int32_t* const* geps,
                       const void* const* chi, void* const* eps, void* const* epsinv, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (nmat <= 0 || !cells || !ng || !geps || !chi || !epsinv) return fail(c, BGW_EINVAL, "NULL argument array");
  int rc;
  for (int m = 0; m < nmat; ++m) {
    if (ng[m] <= 0 || !geps[m] || !chi[m] || !epsinv[m])
      return fail(c, BGW_EINVAL, "matrix %d: bad size or NULL pointer", m);
    if (ng[m] > kGeneralMaxNg)
      return fail(c, BGW_EUNSUPPORTED, "matrix %d: ng = %d exceeds %d for the general inverse", m, ng[m],
                  kGeneralMaxNg);
    if ((rc = check_q(c, &cells[m], ng[m], geps[m])) != BGW_OK) return rc;
  }
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<const int32_t*> dgeps(nmat);
  std::vector<const bgw_cell*> cp(nmat);
  for (int m = 0; m < nmat; ++m) {
    const void* dg;
    if ((rc = upload_cached(c, geps[m], (size_t)ng[m] * 3 * sizeof(int32_t), st, &dg)) != BGW_OK) return rc;
    dgeps[m] = static_cast<const int32_t*>(dg);
    cp[m] = &cells[m];
  }
  set_run_slices(c, BGW_PREC_FP64);
  return epsinv_general_run(c, nmat, ng, cp.data(), dgeps.data(), chi, eps, epsinv, st, c->inverse_mode == 1);
}

int bgw_epsinv_rflavor(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng, const int32_t* const* geps,
                       const void* const* chi, void* const* eps, void* const* epsinv, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (nmat <= 0 || !cells || !ng || !geps || !chi || !epsinv) return fail(c, BGW_EINVAL, "NULL argument array");
  int rc;
  for (int m = 0; m < nmat; ++m) {
    if (ng[m] <= 0 || !geps[m] || !chi[m] || !epsinv[m])
      return fail(c, BGW_EINVAL, "matrix %d: bad size or NULL pointer", m);
    if ((rc = check_q(c, &cells[m], ng[m], geps[m])) != BGW_OK) return rc;
  }
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<const int32_t*> dgeps(nmat);
  std::vector<const bgw_cell*> cp(nmat);
  for (int m = 0; m < nmat; ++m) {
    const void* dg;
    if ((rc = upload_cached(c, geps[m], (size_t)ng[m] * 3 * sizeof(int32_t), st, &dg)) != BGW_OK) return rc;
    dgeps[m] = static_cast<const int32_t*>(dg);
    cp[m] = &cells[m];
  }
  set_run_slices(c, BGW_PREC_FP64);
  return epsinv_rflavor_run(c, nmat, ng, cp.data(), dgeps.data(), chi, eps, epsinv, st, c->inverse_mode == 1);
}

int bgw_epsinv(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng, const int32_t* const* geps,
               const void* const* chi, void* const* eps, void* const* epsinv, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (nmat <= 0 || !cells || !ng || !geps || !chi || !epsinv) return fail(c, BGW_EINVAL, "NULL argument array");
  int rc;
  for (int m = 0; m < nmat; ++m) {
    if (ng[m] <= 0 || !geps[m] || !chi[m] || !epsinv[m])
      return fail(c, BGW_EINVAL, "matrix %d: bad size or NULL pointer", m);
    if ((rc = check_q(c, &cells[m], ng[m], geps[m])) != BGW_OK) return rc;
  }
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<const int32_t*> dgeps(nmat);
  std::vector<const bgw_cell*> cp(nmat);
  for (int m = 0; m < nmat; ++m) {
    const void* dg;
    if ((rc = upload_cached(c, geps[m], (size_t)ng[m] * 3 * sizeof(int32_t), st, &dg)) != BGW_OK) return rc;
    dgeps[m] = static_cast<const int32_t*>(dg);
    cp[m] = &cells[m];
  }
  set_run_slices(c, BGW_PREC_FP64);
  auto body = [&]() {
    return epsinv_batch_run(c, nmat, ng, cp.data(), dgeps.data(), chi, eps, epsinv, st, c->inverse_mode == 1);
  };
  // Repeated calls with the same arguments replay a CUDA graph of the
  // sweep (about five launches per 32-column step on three streams): the
  // graph's edges replace the streams' event waits.
  uint64_t key = hash_bytes("epsinv", 6, hash_bytes(&nmat, sizeof(nmat)));
  key = hash_bytes(&st, sizeof(st), key);
  const int modes[5] = {c->inverse_mode, c->update_slices, c->run_slices, c->run_ff_chain ? 1 : 0, c->update_items};
  key = hash_bytes(modes, sizeof(modes), key);
  key = hash_bytes(ng, nmat * sizeof(int), key);
  key = hash_bytes(cells, nmat * sizeof(bgw_cell), key);
  for (int m = 0; m < nmat; ++m) {
    const void* ptrs[4] = {chi[m], eps ? eps[m] : nullptr, epsinv[m], dgeps[m]};
    key = hash_bytes(ptrs, sizeof(ptrs), key);
  }
  return run_graphed(c, key, st, body);
}

int bgw_screened_w(bgw_ctx* ctx, int nmat, const bgw_cell* cells, const int* ng, const int32_t* const* geps,
                   const void* const* epsinv, void* const* W, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (nmat <= 0 || !cells || !ng || !geps || !epsinv || !W) return fail(c, BGW_EINVAL, "NULL argument array");
  int rc;
  for (int m = 0; m < nmat; ++m) {
    if (ng[m] <= 0 || !geps[m] || !epsinv[m] || !W[m])
      return fail(c, BGW_EINVAL, "matrix %d: bad size or NULL pointer", m);
    if (ng[m] > 65535) return fail(c, BGW_EUNSUPPORTED, "matrix %d: ng = %d exceeds 65535", m, ng[m]);
    if ((rc = check_q(c, &cells[m], ng[m], geps[m])) != BGW_OK) return rc;
    if (W[m] != epsinv[m]) {
      const size_t bytes = (size_t)ng[m] * ng[m] * sizeof(double2);
      const char *a = static_cast<const char*>(epsinv[m]), *b = static_cast<const char*>(W[m]);
      if (a < b + bytes && b < a + bytes) return fail(c, BGW_EINVAL, "matrix %d: W overlaps epsinv", m);
    }
  }
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<const int32_t*> dgeps(nmat);
  std::vector<const bgw_cell*> cp(nmat);
  for (int m = 0; m < nmat; ++m) {
    const void* dg;
    if ((rc = upload_cached(c, geps[m], (size_t)ng[m] * 3 * sizeof(int32_t), st, &dg)) != BGW_OK) return rc;
    dgeps[m] = static_cast<const int32_t*>(dg);
    cp[m] = &cells[m];
  }
  return screened_w_run(c, nmat, ng, cp.data(), dgeps.data(), epsinv, W, st);
}

}  // extern "C"

namespace {

// The whole batch, in stream order on st (no host synchronization once the
// plans and uploads of its arguments are cached).
int run_batch(Ctx* c, int nq, const bgw_problem* pr, int nfreq, const double* dev_om, int prec,
              void* const* epsinv, const std::vector<const void*>& dev_ev, const std::vector<const void*>& dev_ec,
              const std::vector<const void*>& dev_geps, cudaStream_t st) {
  const int nrow = nfreq > 0 ? nfreq : 1;
  const size_t cs = prec == BGW_PREC_FP64 ? 16 : 8;
  size_t mbytes = 0, cbytes = 0;
  for (int q = 0; q < nq; ++q) {
    mbytes = std::max(mbytes, (size_t)pr[q].nv * pr[q].nc * pr[q].ng * cs);
    cbytes = std::max(cbytes, (size_t)nrow * pr[q].ng * pr[q].ng * sizeof(double2));
  }
  Scratch sM, sChi;
  sM.pool = sChi.pool = &c->pool;
  int rc;
  if ((rc = c->pool.alloc(mbytes, &sM.ptr)) != BGW_OK || (rc = c->pool.alloc(cbytes, &sChi.ptr)) != BGW_OK)
    return fail(c, rc, "bgw_epsilon_batch: scratch allocation failed (M %zu B, chi %zu B)", mbytes, cbytes);
  for (int q = 0; q < nq; ++q) {
    const bgw_problem& p = pr[q];
    const int n = p.cell.fft[0];
    const BandPlan *bpv, *bpc;
    const PairPlan* pp;
    if ((rc = get_band_plan(c, n, p.npw_v, p.gv, st, &bpv)) != BGW_OK) return rc;
    if ((rc = get_band_plan(c, n, p.npw_c, p.gc, st, &bpc)) != BGW_OK) return rc;
    if ((rc = get_pair_plan(c, n, p.ng, p.geps, st, &pp)) != BGW_OK) return rc;
    if ((rc = mtxel_run(c, n, prec, p.nv, bpv, p.cv, p.nc, bpc, p.cc, pp, sM.ptr, st)) != BGW_OK) return rc;
    HeadPlan hp;
    Scratch sH;
    sH.pool = &c->pool;
    if ((rc = head_prepare(c, &p.cell, p.npw_v, p.gv, p.npw_c, p.gc, p.ng, p.geps, prec, st, &hp)) != BGW_OK)
      return rc;
    if (hp.g0 >= 0) {
      if ((rc = c->pool.alloc((size_t)p.nv * p.nc * sizeof(double2), &sH.ptr)) != BGW_OK)
        return fail(c, rc, "head scratch");
      if ((rc = head_dot(c, &hp, p.nv, p.cv, p.npw_v, p.nc, p.cc, p.ng, sM.ptr, sH.as<double2>(), st)) != BGW_OK)
        return rc;
    }
    if ((rc = chi_run(c, prec, p.nv, p.nc, p.ng, sM.ptr, static_cast<const double*>(dev_ev[q]),
                      static_cast<const double*>(dev_ec[q]), nfreq, dev_om, 4.0 / p.cell.omega, 0, sChi.ptr, st,
                      &hp, sH.as<double2>())) != BGW_OK)
      return rc;
    const size_t n2 = (size_t)p.ng * p.ng * sizeof(double2);
    std::vector<int> ngv(nrow, p.ng);
    std::vector<const bgw_cell*> cp(nrow, &p.cell);
    std::vector<const int32_t*> gv(nrow, static_cast<const int32_t*>(dev_geps[q]));
    std::vector<const void*> chis(nrow);
    std::vector<void*> invs(nrow);
    for (int f = 0; f < nrow; ++f) {
      chis[f] = static_cast<char*>(sChi.ptr) + f * n2;
      invs[f] = static_cast<char*>(epsinv[q]) + f * n2;
    }
    set_run_slices(c, prec);
    if ((rc = epsinv_batch_run(c, nrow, ngv.data(), cp.data(), gv.data(), chis.data(), nullptr,
                               invs.data(), st, use_tc_inverse(c, prec))) != BGW_OK)
      return rc;
  }
  return BGW_OK;
}

}  // namespace

extern "C" int bgw_epsilon_batch(bgw_ctx* ctx, int nq, const bgw_problem* problems, int nfreq, const double* omega,
                                 int prec, void* const* epsinv, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  if (nq <= 0 || !problems || !epsinv) return fail(c, BGW_EINVAL, "bad batch arguments");
  if (prec & BGW_FLAVOR_REAL) return fail(c, BGW_EUNSUPPORTED, "bgw_epsilon_batch: complex flavor only");
  if (nfreq < 0 || (nfreq > 0 && !omega)) return fail(c, BGW_EINVAL, "bad frequency list");
  for (int f = 0; f < nfreq; ++f)
    if (!isfinite(omega[f])) return fail(c, BGW_EINVAL, "omega[%d] is not finite", f);
  int rc, n;
  for (int q = 0; q < nq; ++q) {
    const bgw_problem& p = problems[q];
    if ((rc = validate_mtxel(c, &p.cell, p.nv, p.npw_v, p.gv, p.cv, p.nc, p.npw_c, p.gc, p.cc, p.ng, p.geps, prec,
                             epsinv[q], &n)) != BGW_OK)
      return fail(c, rc, "problem %d: %s", q, c->err.c_str());
    if ((rc = check_energies(c, p.nv, p.ev, p.nc, p.ec)) != BGW_OK) return fail(c, rc, "problem %d: %s", q, c->err.c_str());
    if ((rc = check_q(c, &p.cell, p.ng, p.geps)) != BGW_OK) return fail(c, rc, "problem %d: %s", q, c->err.c_str());
    if (!is_device_ptr(p.cv) || !is_device_ptr(p.cc) || !is_device_ptr(epsinv[q]))
      return fail(c, BGW_EINVAL, "problem %d: cv, cc and epsinv must be device arrays", q);
  }
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Key of the argument set: sizes, pointers and host-array contents.
  uint64_t key = hash_bytes(&nq, sizeof(nq), hash_bytes(&prec, sizeof(prec), hash_bytes(&nfreq, sizeof(nfreq))));
  if (nfreq > 0) key = hash_bytes(omega, nfreq * sizeof(double), key);
  key = hash_bytes(&st, sizeof(st), key);
  const int modes[6] = {c->inverse_mode, c->head_mode, c->update_slices, c->double_fp32, c->pair_kernel,
                         c->update_items};
  key = hash_bytes(modes, sizeof(modes), key);
  for (int q = 0; q < nq; ++q) {
    const bgw_problem& p = problems[q];
    key = hash_bytes(&p.cell, sizeof(p.cell), key);
    const void* ptrs[3] = {p.cv, p.cc, epsinv[q]};
    key = hash_bytes(ptrs, sizeof(ptrs), key);
    const int dims[4] = {p.nv, p.npw_v, p.nc, p.npw_c};
    key = hash_bytes(dims, sizeof(dims), key);
    key = hash_bytes(p.gv, (size_t)p.npw_v * 12, key);
    key = hash_bytes(p.gc, (size_t)p.npw_c * 12, key);
    key = hash_bytes(p.geps, (size_t)p.ng * 12, key);
    key = hash_bytes(p.ev, (size_t)p.nv * 8, key);
    key = hash_bytes(p.ec, (size_t)p.nc * 8, key);
  }
  auto it = c->use_graphs ? c->graphs.find(key) : c->graphs.end();
  if (it != c->graphs.end()) {
    BGW_CUDA(c, cudaGraphLaunch(it->second.exec, st));
    c->launches += it->second.kernels;
    c->graph_replays += 1;
    return BGW_OK;
  }
  // Uploads of the small host arrays (cached by content).
  const void* dev_om = nullptr;
  if (nfreq > 0 && (rc = upload_cached(c, omega, nfreq * sizeof(double), st, &dev_om)) != BGW_OK) return rc;
  std::vector<const void*> dev_ev(nq), dev_ec(nq), dev_geps(nq);
  for (int q = 0; q < nq; ++q) {
    const bgw_problem& p = problems[q];
    if ((rc = upload_cached(c, p.ev, p.nv * sizeof(double), st, &dev_ev[q])) != BGW_OK) return rc;
    if ((rc = upload_cached(c, p.ec, p.nc * sizeof(double), st, &dev_ec[q])) != BGW_OK) return rc;
    if ((rc = upload_cached(c, p.geps, (size_t)p.ng * 12, st, &dev_geps[q])) != BGW_OK) return rc;
  }
  // Direct run: produces this call's results, creates the plans, tunes and
  // fills the pool with the blocks the capture below will reuse.
  if ((rc = run_batch(c, nq, problems, nfreq, static_cast<const double*>(dev_om), prec, epsinv, dev_ev, dev_ec,
                      dev_geps, st)) != BGW_OK)
    return rc;
  if (st == nullptr || st == cudaStreamLegacy) return BGW_OK;  // the legacy stream cannot be captured
  if (!c->use_graphs || c->graphs.size() >= kMaxGraphs) return BGW_OK;
  const bool timing = c->timing.on;
  c->timing.on = false;
  c->pool.set_pinning(true);
  const uint64_t l0 = c->launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = run_batch(c, nq, problems, nfreq, static_cast<const double*>(dev_om), prec, epsinv, dev_ev, dev_ec,
                   dev_geps, st);
    e = cudaStreamEndCapture(st, &graph);
  }
  c->pool.set_pinning(false);
  c->timing.on = timing;
  const uint64_t captured = c->launches - l0;
  c->launches = l0;  // captured launches did not run
  if (e != cudaSuccess || rc != BGW_OK || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    c->pool.abandon_pins();   // no graph refers to them
    c->err.clear();
    return BGW_OK;  // results of the direct run stand; the next call runs directly again
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->pool.abandon_pins();
    return BGW_OK;
  }
  c->graphs[key].exec = exec;
  c->graphs[key].kernels = captured;
  return BGW_OK;
}

namespace {

// Frequencies of one whole-path call: the imaginary axis (nfreq = 0: static)
// or the real axis with broadening (bgw_epsilon_real).
struct FreqArgs {
  bool real = false;
  int nfreq = 0;
  const double* w = nullptr;   // omega (imaginary axis) or E (real axis), host
  double delta = 0.0;
  int advanced = 0;
};

int epsilon_run(bgw_ctx* ctx, const bgw_cell* cell, int nv, int npw_v, const int32_t* gv, const void* cv,
                const double* ev, int nc, int npw_c, const int32_t* gc, const void* cc, const double* ec, int ng,
                const int32_t* geps, const FreqArgs& fa, int prec, int nc_chunk, void* chi, void* epsinv,
                void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  int n, rc;
  bool rf;   // real flavor
  if ((rc = split_flavor(c, &prec, &rf)) != BGW_OK) return rc;
  if (rf && fa.real) return fail(c, BGW_EUNSUPPORTED, "the real-axis response has complex chi: no real flavor");
  if ((rc = validate_mtxel(c, cell, nv, npw_v, gv, cv, nc, npw_c, gc, cc, ng, geps, prec, epsinv, &n)) != BGW_OK)
    return rc;
  if ((rc = check_energies(c, nv, ev, nc, ec)) != BGW_OK) return rc;
  if ((rc = check_q(c, cell, ng, geps)) != BGW_OK) return rc;
  const int nfreq = fa.nfreq;
  const double* omega = fa.w;
  if (fa.real) {
    if ((rc = check_real_axis(c, nfreq, omega, fa.delta, fa.advanced)) != BGW_OK) return rc;
    if (ng > kGeneralMaxNg)
      return fail(c, BGW_EUNSUPPORTED, "ng = %d exceeds %d for the general inverse", ng, kGeneralMaxNg);
  } else if (nfreq < 0 || (nfreq > 0 && !omega)) {
    return fail(c, BGW_EINVAL, "bad frequency list");
  }
  if (nc_chunk <= 0 || nc_chunk > nc) nc_chunk = nc;
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool cv_dev = is_device_ptr(cv), cc_dev = is_device_ptr(cc);
  const bool chi_dev = chi && is_device_ptr(chi), inv_dev = is_device_ptr(epsinv);
  auto body = [&]() -> int {
    int rc;
    const int nrow = nfreq > 0 ? nfreq : 1;
    // element sizes: coefficients, M, chi and eps~^-1 are real in the real flavor
    const size_t coef = rf ? 8 : 16;
    const size_t cs = (prec == BGW_PREC_FP64 ? 16 : 8) / (rf ? 2 : 1);
    const size_t n2 = (size_t)ng * ng * (rf ? sizeof(double) : sizeof(double2));
    Scratch s_cv, s_cc, s_M, s_chi, s_inv;
    s_cv.pool = s_cc.pool = s_M.pool = s_chi.pool = s_inv.pool = &c->pool;
    const void* d_cv = cv;
    const void* d_cc = cc;
    if (!cv_dev) {
      if ((rc = c->pool.alloc((size_t)nv * npw_v * coef, &s_cv.ptr)) != BGW_OK) return fail(c, rc, "cv staging");
      BGW_CUDA(c, cudaMemcpyAsync(s_cv.ptr, cv, (size_t)nv * npw_v * coef, cudaMemcpyHostToDevice, st));
      d_cv = s_cv.ptr;
    }
    // Host conduction coefficients are copied chunk by chunk on a copy stream,
    // one chunk ahead of the chunk being transformed: the copies overlap the
    // matrix elements and chi of the chunk before (forked from and joined
    // back to the call's stream by events, so graph capture keeps them).
    const bool cc_chunked = !cc_dev && nc_chunk < nc;
    auto copy_chunk = [&](int c0, cudaEvent_t done) -> int {
      const int ncc = std::min(nc_chunk, nc - c0);
      const size_t off = (size_t)c0 * npw_c * coef, bytes = (size_t)ncc * npw_c * coef;
      BGW_CUDA(c, cudaMemcpyAsync(static_cast<char*>(s_cc.ptr) + off, static_cast<const char*>(cc) + off, bytes,
                                  cudaMemcpyHostToDevice, c->copy_st));
      BGW_CUDA(c, cudaEventRecord(done, c->copy_st));
      return BGW_OK;
    };
    if (!cc_dev) {
      if ((rc = c->pool.alloc((size_t)nc * npw_c * coef, &s_cc.ptr)) != BGW_OK) return fail(c, rc, "cc staging");
      if (cc_chunked) {
        if (!c->copy_st) {
          BGW_CUDA(c, cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking));
          for (auto& e : c->copy_ev) BGW_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        // the staging block may still be read by earlier work on the stream
        BGW_CUDA(c, cudaEventRecord(c->copy_ev[0], st));
        BGW_CUDA(c, cudaStreamWaitEvent(c->copy_st, c->copy_ev[0], 0));
        if ((rc = copy_chunk(0, c->copy_ev[1])) != BGW_OK) return rc;
      } else {
        BGW_CUDA(c, cudaMemcpyAsync(s_cc.ptr, cc, (size_t)nc * npw_c * coef, cudaMemcpyHostToDevice, st));
      }
      d_cc = s_cc.ptr;
    }
    void* d_chi = chi_dev ? chi : nullptr;
    if (!d_chi) {
      if ((rc = c->pool.alloc(nrow * n2, &s_chi.ptr)) != BGW_OK) return fail(c, rc, "chi scratch");
      d_chi = s_chi.ptr;
    }
    void* d_inv = inv_dev ? epsinv : nullptr;
    if (!d_inv) {
      if ((rc = c->pool.alloc(nrow * n2, &s_inv.ptr)) != BGW_OK) return fail(c, rc, "epsinv scratch");
      d_inv = s_inv.ptr;
    }
    if ((rc = c->pool.alloc((size_t)nv * nc_chunk * ng * cs, &s_M.ptr)) != BGW_OK) return fail(c, rc, "M scratch");
    const BandPlan *bpv, *bpc;
    const PairPlan* pp;
    if ((rc = get_band_plan(c, n, npw_v, gv, st, &bpv)) != BGW_OK) return rc;
    if ((rc = get_band_plan(c, n, npw_c, gc, st, &bpc)) != BGW_OK) return rc;
    if ((rc = get_pair_plan(c, n, ng, geps, st, &pp)) != BGW_OK) return rc;
    const void *dev_ev, *dev_ec, *dev_om = nullptr, *dev_geps;
    if ((rc = upload_cached(c, ev, nv * sizeof(double), st, &dev_ev)) != BGW_OK) return rc;
    if ((rc = upload_cached(c, ec, nc * sizeof(double), st, &dev_ec)) != BGW_OK) return rc;
    if (nfreq > 0 && (rc = upload_cached(c, omega, nfreq * sizeof(double), st, &dev_om)) != BGW_OK) return rc;
    if ((rc = upload_cached(c, geps, (size_t)ng * 3 * sizeof(int32_t), st, &dev_geps)) != BGW_OK) return rc;
    HeadPlan hp;
    Scratch s_h;
    s_h.pool = &c->pool;
    if (!fa.real && !rf && (rc = head_prepare(c, cell, npw_v, gv, npw_c, gc, ng, geps, prec, st, &hp)) != BGW_OK) return rc;
    if (hp.g0 >= 0 && (rc = c->pool.alloc((size_t)nv * nc_chunk * sizeof(double2), &s_h.ptr)) != BGW_OK)
      return fail(c, rc, "head scratch");
    for (int c0 = 0, k = 0; c0 < nc; c0 += nc_chunk, ++k) {
      const int ncc = std::min(nc_chunk, nc - c0);
      const void* cc0 = static_cast<const char*>(d_cc) + (size_t)c0 * npw_c * coef;
      if (cc_chunked) {
        // next chunk's copy first (its event was last waited on by chunk k - 1),
        // then wait for this chunk's
        if (c0 + nc_chunk < nc && (rc = copy_chunk(c0 + nc_chunk, c->copy_ev[1 + (k + 1) % 2])) != BGW_OK) return rc;
        BGW_CUDA(c, cudaStreamWaitEvent(st, c->copy_ev[1 + k % 2], 0));
      }
      if ((rc = mtxel_run(c, n, prec, nv, bpv, d_cv, ncc, bpc, cc0, pp, s_M.ptr, st, rf)) != BGW_OK) return rc;
      if (hp.g0 >= 0 &&
          (rc = head_dot(c, &hp, nv, d_cv, npw_v, ncc, cc0, ng, s_M.ptr, s_h.as<double2>(), st)) != BGW_OK)
        return rc;
      if (fa.real)
        rc = chi_real_run(c, prec, nv, ncc, ng, s_M.ptr, static_cast<const double*>(dev_ev),
                          static_cast<const double*>(dev_ec) + c0, nfreq, static_cast<const double*>(dev_om), fa.delta,
                          fa.advanced, 4.0 / cell->omega, c0 > 0, d_chi, st);
      else
        rc = chi_run(c, prec, nv, ncc, ng, s_M.ptr, static_cast<const double*>(dev_ev),
                     static_cast<const double*>(dev_ec) + c0, nfreq, static_cast<const double*>(dev_om),
                     4.0 / cell->omega, c0 > 0, d_chi, st, &hp, s_h.as<double2>(), rf);
      if (rc != BGW_OK) return rc;
    }
    {
      std::vector<int> ngv(nrow, ng);
      std::vector<const bgw_cell*> cp(nrow, cell);
      std::vector<const int32_t*> gv2(nrow, static_cast<const int32_t*>(dev_geps));
      std::vector<const void*> chis(nrow);
      std::vector<void*> invs(nrow);
      for (int f = 0; f < nrow; ++f) {
        chis[f] = static_cast<char*>(d_chi) + f * n2;
        invs[f] = static_cast<char*>(d_inv) + f * n2;
      }
      set_run_slices(c, prec);
      if (fa.real)
        rc = epsinv_general_run(c, nrow, ngv.data(), cp.data(), gv2.data(), chis.data(), nullptr, invs.data(), st,
                                use_tc_inverse(c, prec));
      else if (rf)
        rc = epsinv_rflavor_run(c, nrow, ngv.data(), cp.data(), gv2.data(), chis.data(), nullptr, invs.data(), st,
                                use_tc_inverse(c, prec));
      else
        rc = epsinv_batch_run(c, nrow, ngv.data(), cp.data(), gv2.data(), chis.data(), nullptr, invs.data(), st,
                              use_tc_inverse(c, prec));
      if (rc != BGW_OK) return rc;
    }
    if (chi && !chi_dev) BGW_CUDA(c, cudaMemcpyAsync(chi, d_chi, nrow * n2, cudaMemcpyDeviceToHost, st));
    if (!inv_dev) BGW_CUDA(c, cudaMemcpyAsync(epsinv, d_inv, nrow * n2, cudaMemcpyDeviceToHost, st));
    return BGW_OK;
  };
  // Repeated calls with the same arguments replay a CUDA graph of the whole
  // path (copies included) when every host buffer is page-locked: the key
  // holds the sizes, the pointers and the small host arrays' contents; the
  // large coefficient and result buffers are read and written in place.
  auto pinned_or_dev = [](const void* p) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged || at.type == cudaMemoryTypeHost;
  };
  const bool graphable = pinned_or_dev(cv) && pinned_or_dev(cc) && pinned_or_dev(chi) && pinned_or_dev(epsinv);
  if (graphable) {
    uint64_t key = hash_bytes("epsilon", 7, hash_bytes(cell, sizeof(bgw_cell)));
    const int dims[10] = {nv, npw_v, nc, npw_c, ng, nfreq, prec | (rf ? BGW_FLAVOR_REAL : 0), nc_chunk,
                          fa.real ? 1 : 0, fa.advanced};
    key = hash_bytes(dims, sizeof(dims), key);
    key = hash_bytes(&fa.delta, sizeof(double), key);
    if (nfreq > 0) key = hash_bytes(omega, nfreq * sizeof(double), key);
    const void* ptrs[5] = {cv, cc, chi, epsinv, (const void*)st};
    key = hash_bytes(ptrs, sizeof(ptrs), key);
    const int modes[6] = {c->inverse_mode, c->head_mode, c->update_slices, c->double_fp32, c->pair_kernel,
                         c->update_items};
    key = hash_bytes(modes, sizeof(modes), key);
    key = hash_bytes(gv, (size_t)npw_v * 12, key);
    key = hash_bytes(gc, (size_t)npw_c * 12, key);
    key = hash_bytes(geps, (size_t)ng * 12, key);
    key = hash_bytes(ev, (size_t)nv * 8, key);
    key = hash_bytes(ec, (size_t)nc * 8, key);
    rc = run_graphed(c, key, st, body);
  } else {
    rc = body();
  }
  if (rc != BGW_OK) return rc;
  if (!inv_dev || (chi && !chi_dev)) return bgw_sync(ctx, stream);
  return BGW_OK;
}

}  // namespace

extern "C" {

int bgw_epsilon(bgw_ctx* ctx, const bgw_cell* cell, int nv, int npw_v, const int32_t* gv, const void* cv,
                const double* ev, int nc, int npw_c, const int32_t* gc, const void* cc, const double* ec, int ng,
                const int32_t* geps, int nfreq, const double* omega, int prec, int nc_chunk, void* chi,
                void* epsinv, void* stream) {
  FreqArgs fa;
  fa.nfreq = nfreq;
  fa.w = omega;
  return epsilon_run(ctx, cell, nv, npw_v, gv, cv, ev, nc, npw_c, gc, cc, ec, ng, geps, fa, prec, nc_chunk, chi,
                     epsinv, stream);
}

int bgw_epsilon_real(bgw_ctx* ctx, const bgw_cell* cell, int nv, int npw_v, const int32_t* gv, const void* cv,
                     const double* ev, int nc, int npw_c, const int32_t* gc, const void* cc, const double* ec,
                     int ng, const int32_t* geps, int nfreq, const double* energy, double delta, int advanced,
                     int prec, int nc_chunk, void* chi, void* epsinv, void* stream) {
  FreqArgs fa;
  fa.real = true;
  fa.nfreq = nfreq;
  fa.w = energy;
  fa.delta = delta;
  fa.advanced = advanced;
  return epsilon_run(ctx, cell, nv, npw_v, gv, cv, ev, nc, npw_c, gc, cc, ec, ng, geps, fa, prec, nc_chunk, chi,
                     epsinv, stream);
}

int bgw_sigma_cohsex(bgw_ctx* ctx, const bgw_cell* cell, int no, int npw_o, const int32_t* go, const void* co, int ni,
                     int npw_i, const int32_t* gi, const void* ci, int nocc, int ng, const int32_t* geps,
                     const void* epsinv, int prec, double* sigma, void* stream) {
  Ctx* c = impl(ctx);
  if (!c) return BGW_EINVAL;
  int n, rc;
  if ((rc = check_cell(c, cell, &n)) != BGW_OK) return rc;
  if ((rc = check_prec(c, prec)) != BGW_OK) return rc;
  if (ng > max_ng(prec)) return fail(c, BGW_EUNSUPPORTED, "ng = %d exceeds %d", ng, max_ng(prec));
  if (no <= 0 || ni <= 0 || nocc < 0 || nocc > ni) return fail(c, BGW_EINVAL, "need no, ni >= 1 and 0 <= nocc <= ni");
  if ((long long)no * ni > 0x7fffffffLL) return fail(c, BGW_EUNSUPPORTED, "no * ni exceeds 2^31 - 1");
  if (!co || !ci || !epsinv || !sigma) return fail(c, BGW_EINVAL, "NULL coefficient, epsinv or output pointer");
  if (!is_device_ptr(co) || !is_device_ptr(ci) || !is_device_ptr(epsinv))
    return fail(c, BGW_EINVAL, "co, ci and epsinv must be device arrays");
  if (ng > max_ng(BGW_PREC_FP64)) return fail(c, BGW_EUNSUPPORTED, "ng = %d exceeds %d", ng, max_ng(BGW_PREC_FP64));
  int mo[3], mi[3], me[3];
  if ((rc = check_glist(c, "go", npw_o, go, n, mo)) != BGW_OK) return rc;
  if ((rc = check_glist(c, "gi", npw_i, gi, n, mi)) != BGW_OK) return rc;
  if ((rc = check_glist(c, "geps", ng, geps, n, me)) != BGW_OK) return rc;
  for (int d = 0; d < 3; ++d)
    if (n <= mo[d] + mi[d] + me[d])
      return fail(c, BGW_EINVAL, "FFT grid %d aliases on axis %d: need n > max|Gi| + max|Go| + max|Geps|", n, d);
  if ((rc = check_q(c, cell, ng, geps)) != BGW_OK) return rc;
  DeviceGuard g(c->device);
  if (!g.ok) return fail(c, BGW_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> neg((size_t)ng * 3);
  for (size_t i = 0; i < neg.size(); ++i) neg[i] = -geps[i];
  {   // -G must stay inside [-n/2, n/2) as well
    int tmp[3];
    if ((rc = check_glist(c, "-geps", ng, neg.data(), n, tmp)) != BGW_OK) return rc;
  }
  const BandPlan *bpo, *bpi;
  const PairPlan* pp;
  if ((rc = get_band_plan(c, n, npw_o, go, st, &bpo)) != BGW_OK) return rc;
  if ((rc = get_band_plan(c, n, npw_i, gi, st, &bpi)) != BGW_OK) return rc;
  if ((rc = get_pair_plan(c, n, ng, neg.data(), st, &pp)) != BGW_OK) return rc;
  const void* dg;
  if ((rc = upload_cached(c, geps, (size_t)ng * 3 * sizeof(int32_t), st, &dg)) != BGW_OK) return rc;
  return sigma_run(c, cell, n, no, bpo, go, co, ni, bpi, ci, nocc, ng, geps, static_cast<const int32_t*>(dg), pp,
                   epsinv, prec, sigma, st);
}

int bgw_real_coefficients(int nb, int npw, const void* c, const double* energies, double tol, double* out) {
  if (nb <= 0 || npw <= 0 || !c || !energies || !out || !(tol >= 0.0)) return BGW_EINVAL;
  const double* z = static_cast<const double*>(c);   // interleaved (re, im)
  std::vector<double> v(npw);
  std::vector<std::vector<double>> basis;
  for (int start = 0; start < nb;) {
    int stop = start + 1;
    while (stop < nb && std::fabs(energies[stop] - energies[stop - 1]) <= tol) ++stop;
    const int n = stop - start;
    basis.clear();
    for (int b = start; b < stop && (int)basis.size() < n; ++b) {
      for (int part = 0; part < 2 && (int)basis.size() < n; ++part) {
        double norm0 = 0.0;
        for (int k = 0; k < npw; ++k) {
          v[k] = z[2 * ((size_t)b * npw + k) + part];
          norm0 += v[k] * v[k];
        }
        for (const auto& q : basis) {   // modified Gram-Schmidt
          double d = 0.0;
          for (int k = 0; k < npw; ++k) d += q[k] * v[k];
          for (int k = 0; k < npw; ++k) v[k] -= d * q[k];
        }
        double nr = 0.0;
        for (int k = 0; k < npw; ++k) nr += v[k] * v[k];
        nr = std::sqrt(nr);
        if (nr > 1e-8 * std::max(std::sqrt(norm0), 1e-300)) {
          for (int k = 0; k < npw; ++k) v[k] /= nr;
          basis.push_back(v);
        }
      }
    }
    if ((int)basis.size() < n) return BGW_ENUMERIC;
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < npw; ++k) out[(size_t)(start + i) * npw + k] = basis[i][k];
    start = stop;
  }
  return BGW_OK;
}

int bgw_frequency_grid(double spacing, double low_cutoff, double high_cutoff, double increment, int max_points,
                       double* out, int* npoints) {
  if (!npoints || !(spacing > 0.0) || !(increment >= 0.0) || !(low_cutoff >= 0.0) || !(high_cutoff >= low_cutoff) ||
      !isfinite(spacing) || !isfinite(increment) || !isfinite(high_cutoff))
    return BGW_EINVAL;
  const double tol = 1e-12;
  int n = 0;
  auto put = [&](double e) {
    if (out && n < max_points) out[n] = e;
    ++n;
  };
  double e = 0.0;
  for (long long k = 0; (double)k * spacing <= low_cutoff * (1 + tol) + tol; ++k) {
    e = (double)k * spacing;
    put(e);
    if (n > (1 << 24)) return BGW_EINVAL;
  }
  double step = spacing;
  for (;;) {
    step += increment;
    e += step;
    if (e > high_cutoff * (1 + tol) + tol) break;
    put(e);
    if (n > (1 << 24)) return BGW_EINVAL;
  }
  *npoints = n;
  return (out && n > max_points) ? BGW_ENOMEM : BGW_OK;
}

}  // extern "C"
