// Context runtime: device-memory pool with a budget, error state, cached
// uploads of small host arrays.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "runtime.h"

namespace bgw {

// Content hash of the cache keys: four independent 64-bit lanes over 32-byte
// blocks with the multiply-rotate round of xxHash64 (so the multiplies of the
// lanes overlap instead of forming one chain), the tail byte by byte, and
// MurmurHash3's fmix64 finalizer.  About 8x faster than a byte-serial hash on
// the G lists hashed by every call.
namespace {
constexpr uint64_t kP1 = 0x9E3779B185EBCA87ull, kP2 = 0xC2B2AE3D27D4EB4Full, kP3 = 0x165667B19E3779F9ull;
inline uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }
inline uint64_t round64(uint64_t acc, uint64_t in) { return rotl64(acc + in * kP2, 31) * kP1; }
inline uint64_t fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}
}  // namespace

uint64_t hash_bytes(const void* data, size_t bytes, uint64_t h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t a = h + kP1 + kP2, b = h + kP2, c = h, d = h - kP1;
  size_t i = 0;
  for (; i + 32 <= bytes; i += 32) {
    uint64_t w[4];
    memcpy(w, p + i, 32);
    a = round64(a, w[0]);
    b = round64(b, w[1]);
    c = round64(c, w[2]);
    d = round64(d, w[3]);
  }
  uint64_t t = rotl64(a, 1) + rotl64(b, 7) + rotl64(c, 12) + rotl64(d, 18);
  for (; i < bytes; ++i) t = rotl64(t ^ (p[i] * kP3), 11) * kP1;
  return fmix64(t ^ (uint64_t)bytes);
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

int sm_count(Ctx* c) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = 152;
  }
  return n;
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

int Pool::alloc(size_t bytes, void** out) { return alloc_impl(bytes, out, false); }
int Pool::alloc_keep(size_t bytes, void** out) { return alloc_impl(bytes, out, true); }

int Pool::alloc_impl(size_t bytes, void** out, bool keep) {
  const size_t sz = round(bytes);
  auto it = free_.end();
  const auto range = free_.equal_range(sz);
  for (auto j = range.first; j != range.second; ++j)
    if (!keep || !pinned_.count(j->second)) {
      it = j;
      break;
    }
  if (it != free_.end()) {
    void* p = it->second;
    free_.erase(it);
    live_[p] = sz;
    in_use_ += sz;
    if (in_use_ > high_water_) high_water_ = in_use_;
    if (pinning_ && pinned_.emplace(p, sz).second) capture_pins_.push_back(p);
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
                                          "oz_update", "sweep_chain", "head_dot", "head_wings",
                                          "screened_w", "pivot", "sigma_forms", "sigma_exact", "oz_update_ahead"};
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
  uint64_t key = hash_bytes(host, bytes, hash_bytes(&bytes, sizeof(bytes)));
  auto it = c->uploads.find(key);
  if (it != c->uploads.end()) {
    *dev = it->second;
    return BGW_OK;
  }
  void* p = nullptr;
  int rc = c->pool.alloc_keep(bytes, &p);
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
