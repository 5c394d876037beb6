// cms_prof.cu - per-kernel device timing: while enabled, every kernel the
// library launches is bracketed by CUDA events recorded on its own stream;
// and the NVTX ranges the C entry points open.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cms_internal.h"

namespace cms {
namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};

struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
};

Profiler& prof() {
  static Profiler* p = new Profiler();   // never destroyed: events may outlive static teardown
  return *p;
}

}  // namespace

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }

NvtxRange::~NvtxRange() { nvtxRangePop(); }

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  if (!p.on) return;
  a_ = p.get();
  b_ = p.get();
  if (!a_ || !b_) { a_ = b_ = nullptr; return; }
  cudaEventRecord(a_, s_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  cudaEventRecord(b_, s_);
  p.recs.push_back(Rec{name_, a_, b_});
}

}  // namespace cms

using namespace cms;

extern "C" {

cms_status cms_profile_enable(int32_t on) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  for (const Rec& r : p.recs) {
    cudaEventSynchronize(r.b);
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.recs.clear();
  p.on = on != 0;
  return CMS_OK;
}

cms_status cms_profile_summary(char* buf, size_t len, size_t* needed) {
  Profiler& p = prof();
  std::map<std::string, std::pair<int64_t, double>> agg;
  {
    std::lock_guard<std::mutex> lock(p.mu);
    for (const Rec& r : p.recs) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) {
        set_error("cms_profile_summary: event wait failed");
        return CMS_ERR_CUDA;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      auto& v = agg[r.name];
      v.first += 1;
      v.second += ms;
    }
  }
  std::string out = "{";
  bool first = true;
  for (const auto& kv : agg) {
    char tmp[256];
    std::snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f}", first ? "" : ", ",
                  kv.first.c_str(), static_cast<long long>(kv.second.first), kv.second.second);
    out += tmp;
    first = false;
  }
  out += "}";
  if (needed) *needed = out.size() + 1;
  if (buf && len > 0) {
    const size_t m = std::min(len - 1, out.size());
    std::memcpy(buf, out.data(), m);
    buf[m] = '\0';
    if (m < out.size()) { set_error("cms_profile_summary: buffer too small"); return CMS_ERR_INVALID_ARG; }
  }
  return CMS_OK;
}

}  // extern "C"
