// Kernel-family timing (diagnostics).  While enabled, launch sites bracket their kernels
// with CUDA events recorded on the launching stream and note the launch's algorithmic
// work (flops or bytes, as defined by the family); fosb_profile_read waits for the
// recorded events and returns the family's total device time, launch count and work.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fosb_internal.h"

namespace fosb {

namespace {
struct Rec {
  cudaEvent_t a, b;
  double work;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::map<std::string, std::vector<Rec>> g_recs;
}  // namespace

bool profiling() { return g_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(const char* family, cudaStream_t s, double work) : fam_(family), s_(s), work_(work) {
  if (!profiling()) return;
  if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) return;
  if (cudaEventRecord(a_, s_) == cudaSuccess) active_ = true;
}

ProfScope::~ProfScope() {
  if (!active_) return;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> lock(g_mu);
  g_recs[fam_].push_back(Rec{a_, b_, work_});
}

}  // namespace fosb

extern "C" {

fosb_status fosb_profile_enable(int on) {
  fosb::g_on.store(on != 0);
  return FOSB_OK;
}

fosb_status fosb_profile_read(const char* family, double* total_ms, int64_t* launches, double* work) {
  if (!family) return fosb::fail(FOSB_ERR_INVALID_ARG, "fosb_profile_read: NULL family");
  std::vector<fosb::Rec> recs;
  {
    std::lock_guard<std::mutex> lock(fosb::g_mu);
    auto it = fosb::g_recs.find(family);
    if (it != fosb::g_recs.end()) {
      recs.swap(it->second);
      fosb::g_recs.erase(it);
    }
  }
  double ms_total = 0.0, w = 0.0;
  for (auto& r : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ms_total += ms;
    w += r.work;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (total_ms) *total_ms = ms_total;
  if (launches) *launches = int64_t(recs.size());
  if (work) *work = w;
  return FOSB_OK;
}

}  // extern "C"
