// Context runtime: device-memory pool with a budget, error state, cached
// uploads of small host arrays.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "runtime.h"

namespace bgw {

uint64_t fnv1a(const void* data, size_t bytes, uint64_t h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

int fail(Ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int cuda_fail(Ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, BGW_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(c, BGW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ Pool
size_t Pool::round(size_t b) {
  if (b == 0) b = 1;
  const size_t small = 64 << 10, big = 2 << 20;
  if (b <= big) return (b + small - 1) / small * small;
  return (b + big - 1) / big * big;
}

Pool::~Pool() {
  for (auto& kv : free_) cudaFree(kv.second);
  for (auto& kv : live_) cudaFree(kv.first);
}

int Pool::alloc(size_t bytes, void** out) {
  const size_t sz = round(bytes);
  auto it = free_.find(sz);
  if (it != free_.end()) {
    void* p = it->second;
    free_.erase(it);
    live_[p] = sz;
    in_use_ += sz;
    if (in_use_ > high_water_) high_water_ = in_use_;
    if (pinning_) pinned_[p] = sz;
    *out = p;
    return BGW_OK;
  }
  if (pinning_) return BGW_EBUSY;  // no new device memory while a graph is being captured
  if (budget_ && reserved_ + sz > budget_) {
    trim();
    if (reserved_ + sz > budget_) return BGW_ENOMEM;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trim();
    e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? BGW_ENOMEM : BGW_ECUDA;
    }
  }
  reserved_ += sz;
  live_[p] = sz;
  in_use_ += sz;
  if (in_use_ > high_water_) high_water_ = in_use_;
  *out = p;
  return BGW_OK;
}

void Pool::release(void* p) {
  auto it = live_.find(p);
  if (it == live_.end()) return;
  in_use_ -= it->second;
  free_.emplace(it->second, p);
  live_.erase(it);
}

void Pool::trim() {
  if (free_.empty()) return;
  // Blocks on the free list may still be read by queued work of the stream
  // that released them; wait for the device before giving them back.
  cudaDeviceSynchronize();
  std::multimap<size_t, void*> keep;
  for (auto& kv : free_) {
    if (pinned_.count(kv.second)) {
      keep.emplace(kv.first, kv.second);
      continue;
    }
    cudaFree(kv.second);
    reserved_ -= kv.first;
  }
  free_.swap(keep);
}

// ------------------------------------------------------------ timing
const char* timed_name(int n) {
  static const char* names[kTNumNames] = {"band_transform", "pair_yxpass", "pair_zgather", "chi_f64",
                                          "chi_split", "chi_tc", "chi_reduce", "eps_form", "inverse",
                                          "oz_update", "sweep_chain"};
  return (n >= 0 && n < kTNumNames) ? names[n] : "?";
}

static cudaEvent_t take_event(Ctx* c) {
  if (!c->timing.free_events.empty()) {
    cudaEvent_t e = c->timing.free_events.back();
    c->timing.free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

TimedScope::TimedScope(Ctx* c, int name, cudaStream_t st) : c_(c), name_(name), st_(st) {
  if (!c_->timing.on) return;
  a_ = take_event(c_);
  if (a_ && cudaEventRecord(a_, st_) != cudaSuccess) {
    cudaGetLastError();
    a_ = nullptr;
  }
}

TimedScope::~TimedScope() {
  if (!a_) return;
  cudaEvent_t b = take_event(c_);
  if (!b || cudaEventRecord(b, st_) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  c_->timing.pending.push_back({name_, a_, b});
}

void timing_collect(Ctx* c) {
  for (auto& r : c->timing.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      auto& a = c->timing.acc[r.name];
      a.first += 1;
      a.second += ms;
    } else {
      cudaGetLastError();
    }
    c->timing.free_events.push_back(r.a);
    c->timing.free_events.push_back(r.b);
  }
  c->timing.pending.clear();
}

// ------------------------------------------------------------ uploads
int upload_cached(Ctx* c, const void* host, size_t bytes, cudaStream_t st, const void** dev) {
  uint64_t key = fnv1a(host, bytes, fnv1a(&bytes, sizeof(bytes)));
  auto it = c->uploads.find(key);
  if (it != c->uploads.end()) {
    *dev = it->second;
    return BGW_OK;
  }
  void* p = nullptr;
  int rc = c->pool.alloc(bytes, &p);
  if (rc != BGW_OK) return fail(c, rc, "upload of %zu bytes: device allocation failed", bytes);
  // Stream-ordered: the block may come from the pool's free list and still
  // be read by earlier work on this stream.
  cudaError_t e = cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    c->pool.release(p);
    return cuda_fail(c, e, "cudaMemcpyAsync (upload)");
  }
  c->uploads[key] = p;
  *dev = p;
  return BGW_OK;
}

}  // namespace bgw
