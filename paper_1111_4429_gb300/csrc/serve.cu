// Serving loop for eps~^-1 requests (bgw_serve_* in include/bgw.h).  Each
// request is one q-point's whole path: Eq. eqn_static_xi separates in q,
// so q-points are independent epsilon calculations (Section "Parallelization
// and Performance"); requests are admitted against an estimate of their
// largest arrays, as each of the paper's runs estimates its memory needs
// (Section "Memory estimation").
//
// A scheduler thread owns `max_slots` slots; each slot is a context (its own
// scratch pool, plans and tuning) with its own CUDA stream.  Requests are
// copied into pinned host memory at submit time and wait in a FIFO.  The
// scheduler admits the oldest waiting request whenever a slot is free and
// the request's HBM estimate fits in what the budget has left, so requests
// that arrive while others run join the device as soon as a slot and memory
// free up, and their kernels overlap with the running ones (continuous
// batching across streams).  Completion is detected by polling each slot's
// event; the result is then copied to the caller's buffer and the request's
// latency (submit -> result on the host) recorded.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

namespace bgw {
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  bgw_cell cell;
  int nv = 0, npw_v = 0, nc = 0, npw_c = 0, ng = 0;
  std::vector<int32_t> gv, gc, geps;
  std::vector<double> ev, ec;
  void* h_coef = nullptr;     // pinned: cv then cc (c128)
  void* h_out = nullptr;      // pinned staging of eps~^-1 (when the caller's buffer is not pinned)
  void* user_out = nullptr;   // caller's host eps~^-1 [ng][ng]
  bool user_pinned = false;
  uint64_t est = 0;           // admission estimate (bytes)
  enum State { kQueued, kRunning, kDone } state = kQueued;
  bgw_result res{};
  Clock::time_point t_submit, t_admit;
  // device buffers (from the slot's pool) while running
  void* d_cv = nullptr;
  void* d_cc = nullptr;
  void* d_inv = nullptr;
};

struct Slot {
  bgw_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  std::shared_ptr<Req> req;
};

}  // namespace

struct Server {
  int device = 0;
  bgw_serve_opts opts{};
  uint64_t budget = 0;
  uint64_t in_use = 0;  // sum of admitted estimates
  std::vector<Slot> slots;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  std::string err;
  // Pinned host buffers are reused: cudaFreeHost may synchronize the device,
  // which would stall every running request.
  std::multimap<size_t, void*> pinned_free;
  std::mutex pin_mu;
  void* pinned_get(size_t bytes) {
    const size_t sz = (bytes + (size_t(2) << 20) - 1) / (size_t(2) << 20) * (size_t(2) << 20);
    {
      std::lock_guard<std::mutex> lk(pin_mu);
      auto it = pinned_free.find(sz);
      if (it != pinned_free.end()) {
        void* p = it->second;
        pinned_free.erase(it);
        pinned_size[p] = sz;
        return p;
      }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, sz, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    std::lock_guard<std::mutex> lk(pin_mu);
    pinned_size[p] = sz;
    return p;
  }
  void pinned_put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(pin_mu);
    auto it = pinned_size.find(p);
    if (it == pinned_size.end()) return;
    pinned_free.emplace(it->second, p);
    pinned_size.erase(it);
  }
  std::unordered_map<void*, size_t> pinned_size;
};

namespace {

// Device bytes one request needs at most: coefficients, band grids and the
// band z-pass intermediate, the pair intermediate, M, the chi operand planes,
// workspace and weights, chi and eps~^-1 and the inverse's panels.
size_t count_columns(const std::vector<int32_t>& g, int n) {
  std::set<int> cols;
  for (size_t i = 0; i + 2 < g.size(); i += 3) cols.insert((((g[i + 1] % n) + n) % n) * n + (((g[i] % n) + n) % n));
  return cols.size();
}

uint64_t estimate_bytes(const Req& r, int prec) {
  const uint64_t n = r.cell.fft[0];
  const uint64_t cs = prec == BGW_PREC_FP64 ? 16 : 8;
  const uint64_t K = (uint64_t)r.nv * r.nc;
  const uint64_t grids = (uint64_t)(r.nv + r.nc) * n * n * n * cs;
  const uint64_t ncol_eps = count_columns(r.geps, (int)n);
  const uint64_t ncol_wfn = std::max(count_columns(r.gv, (int)n), count_columns(r.gc, (int)n));
  const uint64_t u1 = (uint64_t)std::max(r.nv, r.nc) * n * ncol_wfn * cs;
  const uint64_t T = std::min<uint64_t>(K * n * ncol_eps * cs, uint64_t(4) << 30);
  const uint64_t M = K * r.ng * cs;
  // operand planes (at most 4 GiB per chunk), per-tile FP32 partials, weights
  const uint64_t ngpad = (r.ng + 127) / 128 * 128;
  const uint64_t chi_mixed = prec == BGW_PREC_FP64 ? 0
                             : std::min<uint64_t>(8 * ngpad * K, uint64_t(4) << 30) + (uint64_t(1) << 30) + K * 8;
  const uint64_t mats = 3ull * r.ng * r.ng * 16 + 2ull * r.ng * 32 * 16;
  const uint64_t coef = ((uint64_t)r.nv * r.npw_v + (uint64_t)r.nc * r.npw_c) * 16;
  return grids + u1 + T + M + chi_mixed + mats + coef + (64ull << 20);
}

void finish(Server* s, Slot& sl, int status) {
  std::shared_ptr<Req> r = sl.req;
  if (status == BGW_OK && !r->user_pinned && r->user_out)
    memcpy(r->user_out, r->h_out, (size_t)r->ng * r->ng * 16);
  Ctx* c = &sl.ctx->impl;
  if (r->d_cv) c->pool.release(r->d_cv);
  if (r->d_cc) c->pool.release(r->d_cc);
  if (r->d_inv) c->pool.release(r->d_inv);
  r->d_cv = r->d_cc = r->d_inv = nullptr;
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->res.status = status;
  r->res.latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
  r->res.queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
  r->res.hbm_bytes = r->est;
  r->state = Req::kDone;
  s->in_use -= r->est;
  s->pinned_put(r->h_coef);
  s->pinned_put(r->h_out);
  r->h_coef = r->h_out = nullptr;
  sl.req.reset();
  // keep the slot's cached scratch within the budget when others need room
  if (s->budget && c->pool.reserved() > s->budget / std::max<size_t>(1, s->slots.size())) c->pool.trim();
  s->cv_done.notify_all();
}

// Enqueue one request's work on its slot (asynchronous).
int launch(Server* s, Slot& sl) {
  Req& r = *sl.req;
  Ctx* c = &sl.ctx->impl;
  const size_t bcv = (size_t)r.nv * r.npw_v * 16, bcc = (size_t)r.nc * r.npw_c * 16;
  const size_t bout = (size_t)r.ng * r.ng * 16;
  int rc;
  if ((rc = c->pool.alloc(bcv, &r.d_cv)) != BGW_OK || (rc = c->pool.alloc(bcc, &r.d_cc)) != BGW_OK ||
      (rc = c->pool.alloc(bout, &r.d_inv)) != BGW_OK)
    return rc;
  if (cudaMemcpyAsync(r.d_cv, r.h_coef, bcv, cudaMemcpyHostToDevice, sl.st) != cudaSuccess ||
      cudaMemcpyAsync(r.d_cc, static_cast<char*>(r.h_coef) + bcv, bcc, cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
    return BGW_ECUDA;
  rc = bgw_epsilon(sl.ctx, &r.cell, r.nv, r.npw_v, r.gv.data(), r.d_cv, r.ev.data(), r.nc, r.npw_c, r.gc.data(),
                   r.d_cc, r.ec.data(), r.ng, r.geps.data(), 0, nullptr, s->opts.prec, 0, nullptr, r.d_inv, sl.st);
  if (rc != BGW_OK) return rc;
  void* dst = r.user_pinned ? r.user_out : r.h_out;
  if (cudaMemcpyAsync(dst, r.d_inv, bout, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess) return BGW_ECUDA;
  if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return BGW_ECUDA;
  return BGW_OK;
}

void worker_main(Server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // completions
    for (auto& sl : s->slots) {
      if (!sl.req) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      lk.unlock();
      int status = q == cudaSuccess ? bgw_sync(sl.ctx, sl.st) : BGW_ECUDA;
      cudaGetLastError();
      finish(s, sl, status);
      lk.lock();
      progress = true;
    }
    // admission: oldest first, while a slot and the budget allow
    while (!s->queue.empty()) {
      Slot* free_slot = nullptr;
      for (auto& sl : s->slots)
        if (!sl.req) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      std::shared_ptr<Req> r = s->queue.front();
      if (s->budget && r->est > s->budget) {  // can never fit
        s->queue.pop_front();
        r->state = Req::kDone;
        r->res.status = BGW_ENOMEM;
        r->res.hbm_bytes = r->est;
        s->cv_done.notify_all();
        progress = true;
        continue;
      }
      if (s->budget && s->in_use + r->est > s->budget) break;
      s->queue.pop_front();
      r->state = Req::kRunning;
      r->t_admit = Clock::now();
      s->in_use += r->est;
      free_slot->req = r;
      lk.unlock();
      int rc = launch(s, *free_slot);
      if (rc != BGW_OK) {
        cudaStreamSynchronize(free_slot->st);
        cudaGetLastError();
        finish(s, *free_slot, rc);
      }
      lk.lock();
      progress = true;
    }
    if (!progress) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
  }
}

}  // namespace
}  // namespace bgw

using bgw::Server;

extern "C" {

int bgw_serve_open(bgw_ctx* ctx, const bgw_serve_opts* opts, bgw_server** out) {
  if (!ctx || !opts || !out || opts->max_slots <= 0 || opts->max_slots > 64) return BGW_EINVAL;
  const int device = ctx->impl.device;
  if (opts->prec != BGW_PREC_FP64 && opts->prec != BGW_PREC_MIX_FP16 && opts->prec != BGW_PREC_MIX_BF16)
    return BGW_EINVAL;
  *out = nullptr;
  auto s = std::make_unique<Server>();
  s->device = device;
  s->opts = *opts;
  if (cudaSetDevice(device) != cudaSuccess) return BGW_ECUDA;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return BGW_ECUDA;
  s->budget = opts->hbm_budget_bytes ? opts->hbm_budget_bytes : (uint64_t)fr * 9 / 10;
  s->slots.resize(opts->max_slots);
  for (auto& sl : s->slots) {
    int rc = bgw_create(&sl.ctx, device, 0);
    if (rc != BGW_OK) return rc;
    // requests bring their own device buffers (one-shot pool blocks), so a
    // graph per argument set would pin scratch without being replayed
    sl.ctx->impl.use_graphs = false;
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      return BGW_ECUDA;
  }
  Server* raw = s.release();
  raw->worker = std::thread(bgw::worker_main, raw);
  *out = reinterpret_cast<bgw_server*>(raw);
  return BGW_OK;
}

int bgw_serve_submit(bgw_server* srv, const bgw_request* req, uint64_t* ticket) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !req || !ticket || !req->epsinv_out) return BGW_EINVAL;
  const bgw_problem& p = req->problem;
  if (p.nv <= 0 || p.nc <= 0 || p.ng <= 0 || p.npw_v <= 0 || p.npw_c <= 0 || !p.gv || !p.gc || !p.geps || !p.cv ||
      !p.cc || !p.ev || !p.ec)
    return BGW_EINVAL;
  auto r = std::make_shared<bgw::Req>();
  r->cell = p.cell;
  r->nv = p.nv;
  r->npw_v = p.npw_v;
  r->nc = p.nc;
  r->npw_c = p.npw_c;
  r->ng = p.ng;
  r->gv.assign(p.gv, p.gv + 3 * (size_t)p.npw_v);
  r->gc.assign(p.gc, p.gc + 3 * (size_t)p.npw_c);
  r->geps.assign(p.geps, p.geps + 3 * (size_t)p.ng);
  r->ev.assign(p.ev, p.ev + p.nv);
  r->ec.assign(p.ec, p.ec + p.nc);
  const size_t bcv = (size_t)p.nv * p.npw_v * 16, bcc = (size_t)p.nc * p.npw_c * 16;
  cudaSetDevice(s->device);
  r->h_coef = s->pinned_get(bcv + bcc);
  if (!r->h_coef) return BGW_ENOMEM;
  memcpy(r->h_coef, p.cv, bcv);
  memcpy(static_cast<char*>(r->h_coef) + bcv, p.cc, bcc);
  r->user_out = req->epsinv_out;
  cudaPointerAttributes a;
  r->user_pinned = cudaPointerGetAttributes(&a, req->epsinv_out) == cudaSuccess && a.type == cudaMemoryTypeHost;
  cudaGetLastError();
  if (!r->user_pinned) {
    r->h_out = s->pinned_get((size_t)p.ng * p.ng * 16);
    if (!r->h_out) {
      s->pinned_put(r->h_coef);
      return BGW_ENOMEM;
    }
  }
  r->est = bgw::estimate_bytes(*r, s->opts.prec);
  r->t_submit = bgw::Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  s->cv_work.notify_all();
  return BGW_OK;
}

int bgw_serve_poll(bgw_server* srv, uint64_t ticket, int timeout_ms, bgw_result* out) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !out) return BGW_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return BGW_EINVAL;
  std::shared_ptr<bgw::Req> r = it->second;
  const auto deadline = bgw::Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (r->state != bgw::Req::kDone) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != bgw::Req::kDone)
      return BGW_EBUSY;
  }
  *out = r->res;
  s->reqs.erase(ticket);
  return BGW_OK;
}

int bgw_serve_cancel(bgw_server* srv, uint64_t ticket) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return BGW_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return BGW_EINVAL;
  std::shared_ptr<bgw::Req> r = it->second;
  if (r->state != bgw::Req::kQueued) return BGW_EBUSY;
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (q->get() == r.get()) {
      s->queue.erase(q);
      break;
    }
  r->state = bgw::Req::kDone;
  r->res.status = BGW_ECANCELED;
  s->pinned_put(r->h_coef);
  s->pinned_put(r->h_out);
  r->h_coef = r->h_out = nullptr;
  s->cv_done.notify_all();
  return BGW_OK;
}

int bgw_serve_close(bgw_server* srv) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return BGW_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // queued requests are canceled; running ones finish first
    for (auto& r : s->queue) {
      r->state = bgw::Req::kDone;
      r->res.status = BGW_ECANCELED;
      s->pinned_put(r->h_coef);
      s->pinned_put(r->h_out);
      r->h_coef = r->h_out = nullptr;
    }
    s->queue.clear();
  }
  // wait for in-flight requests (bounded by their own completion)
  for (;;) {
    bool busy = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& sl : s->slots) busy |= (bool)sl.req;
    }
    if (!busy) break;
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (auto& sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.ctx) bgw_destroy(sl.ctx);
  }
  for (auto& kv : s->pinned_free) cudaFreeHost(kv.second);
  for (auto& kv : s->pinned_size) cudaFreeHost(kv.first);
  delete s;
  return BGW_OK;
}

}  // extern "C"
