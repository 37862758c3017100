// profile.cu -- kernel launch accounting and optional per-kernel timing.
//
// Every launch in the library goes through a LaunchScope, which counts it and,
// while timing is enabled, records a CUDA event pair around it on the
// launching stream.  splat_profile_read() waits for the recorded events and
// returns per-kernel launch counts and summed durations.  Events are pooled
// and reused.  Timing must be off while a stream is being captured into a
// graph (event records would become graph nodes).
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace splat {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_mu;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::string g_only;  // time only this kernel ("" = all)
std::atomic<int> g_has_only{0};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

LaunchScope::LaunchScope(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
  count_launch(1);
  if (g_timing.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_has_only.load(std::memory_order_relaxed) && g_only != name_) return;
    a_ = take_event();
    if (a_ && cudaEventRecord(a_, s_) != cudaSuccess) {
      g_pool.push_back(a_);
      a_ = nullptr;
    }
  }
}

LaunchScope::~LaunchScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (b && cudaEventRecord(b, s_) == cudaSuccess) {
    g_recs.push_back(Rec{name_, a_, b});
  } else {
    g_pool.push_back(a_);
    if (b) g_pool.push_back(b);
  }
}

}  // namespace splat

using namespace splat;

extern "C" uint64_t splat_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

extern "C" int splat_profile_enable(int on) {
  g_timing.store(on ? 1 : 0, std::memory_order_relaxed);
  return SPLAT_OK;
}

extern "C" int splat_profile_select(const char* kernel) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_only = kernel ? kernel : "";
  g_has_only.store(g_only.empty() ? 0 : 1);
  return SPLAT_OK;
}

extern "C" int splat_profile_read(char* names, size_t names_bytes, int64_t* launches, double* ms, int32_t max_kernels,
                                  int32_t* n_kernels) {
  if (!n_kernels || max_kernels < 0 || (max_kernels > 0 && (!names || !launches || !ms)))
    return fail(SPLAT_EINVAL, "splat_profile_read: bad argument");
  std::vector<Rec> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    recs.swap(g_recs);
  }
  std::vector<std::string> keys;
  std::vector<int64_t> cnt;
  std::vector<double> tot;
  int rc = SPLAT_OK;
  for (const Rec& r : recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      rc = fail(SPLAT_ECUDA, "splat_profile_read: event query failed");
      t = 0.f;
    }
    size_t k = 0;
    while (k < keys.size() && keys[k] != r.name) ++k;
    if (k == keys.size()) {
      keys.emplace_back(r.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[k] += 1;
    tot[k] += t;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Rec& r : recs) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
  }
  *n_kernels = (int32_t)keys.size();
  std::string joined;
  for (size_t k = 0; k < keys.size() && (int32_t)k < max_kernels; ++k) {
    launches[k] = cnt[k];
    ms[k] = tot[k];
    joined += keys[k];
    joined += '\n';
  }
  if (max_kernels > 0 && names_bytes > 0) {
    const size_t n = joined.size() < names_bytes - 1 ? joined.size() : names_bytes - 1;
    std::memcpy(names, joined.data(), n);
    names[n] = '\0';
  }
  return rc;
}
