// Runtime pieces of libvl: workspace arena, error plumbing, occupancy queries.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "vl_internal.h"

namespace vl {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void Arena::init(char* base, size_t size) {
  base_ = base;
  size_ = size;
  free_.clear();
  used_.clear();
  in_use_ = peak_ = 0;
  free_[0] = size;
}

void* Arena::alloc(size_t bytes) {
  bytes = align_up(bytes ? bytes : 1, 256);
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second >= bytes) {
      size_t off = it->first, sz = it->second;
      free_.erase(it);
      if (sz > bytes) free_[off + bytes] = sz - bytes;
      used_[off] = bytes;
      in_use_ += bytes;
      if (in_use_ > peak_) peak_ = in_use_;
      return base_ + off;
    }
  }
  return nullptr;
}

void Arena::release(void* p) {
  if (!p) return;
  size_t off = static_cast<char*>(p) - base_;
  auto u = used_.find(off);
  if (u == used_.end()) return;
  size_t sz = u->second;
  used_.erase(u);
  in_use_ -= sz;
  auto nx = free_.lower_bound(off);
  if (nx != free_.end() && nx->first == off + sz) {   // merge with the next block
    sz += nx->second;
    free_.erase(nx);
  }
  auto pv = free_.lower_bound(off);
  if (pv != free_.begin()) {
    --pv;
    if (pv->first + pv->second == off) {   // merge with the previous block
      pv->second += sz;
      return;
    }
  }
  free_[off] = sz;
}

vl_status cuda_fail(Ctx* c, cudaError_t e, const char* what) {
  if (c) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error in %s: %s", what, cudaGetErrorString(e));
    c->last_error = buf;
  }
  return VL_ERR_CUDA;
}

vl_status fail(Ctx* c, vl_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

vl_status check_dev_status(Ctx* c, const char* what) {
  VL_CUDA(c, cudaMemcpyAsync(c->hstatus, c->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->prof.on && c->prof.pending.size() > 256) prof_drain(c);
  if (c->hstatus->code != 0) {
    const int code = c->hstatus->code, row = c->hstatus->row;
    VL_CUDA(c, status_clear(c));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    char buf[256];
    if (code == VL_ERR_NOT_SPD)
      snprintf(buf, sizeof buf, "%s: NOT_SPD at row %d", what, row);
    else if (code == VL_ERR_TIMEOUT)
      snprintf(buf, sizeof buf, "%s: bounded device wait timed out at row %d", what, row);
    else
      snprintf(buf, sizeof buf, "%s: device error %d at row %d", what, code, row);
    return fail(c, (vl_status)code, buf);
  }
  return VL_OK;
}

static cudaEvent_t pool_get(Ctx* c) {
  if (!c->prof.pool.empty()) {
    cudaEvent_t e = c->prof.pool.back();
    c->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(Ctx* ctx, const char* key, int t) : c(ctx) {
  if (!c->prof.on) return;
  Profiler::Pending p{key, t, pool_get(c), pool_get(c)};
  cudaEventRecord(p.a, c->stream);
  c->prof.pending.push_back(p);
  idx = (int)c->prof.pending.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx < 0) return;
  cudaEventRecord(c->prof.pending[idx].b, c->stream);
}

void prof_drain(Ctx* c) {
  for (auto& p : c->prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& a = c->prof.acc[{p.key, p.t}];
      a.ms += ms;
      a.launches += 1;
    } else {
      cudaGetLastError();
    }
    c->prof.pool.push_back(p.a);
    c->prof.pool.push_back(p.b);
  }
  c->prof.pending.clear();
}

void prof_release(Ctx* c) {
  prof_drain(c);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  c->prof.pool.clear();
}

// Cached per (device, kernel, block, smem): grid solves ask once per launch.
int resident_blocks(Ctx* c, const void* kernel, int block, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  const auto key = std::make_tuple(c->device, kernel, block, smem);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second * c->num_sms;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  per_sm = std::max(1, per_sm);
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = per_sm;
  return per_sm * c->num_sms;
}

}  // namespace vl
