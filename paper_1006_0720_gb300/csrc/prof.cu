// Kernel timing hooks and the launch counter used by the measurements.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace pdfgb {

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::string g_only;  // empty: every kernel
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<long long> g_launches{0};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool prof_timing() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

void prof_count(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

long long prof_launches() { return g_launches.load(std::memory_order_relaxed); }

void prof_launch(const char* name, cudaStream_t st, void (*launch)(void*), void* ctx) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!launch) return;
  if (!g_on) {
    launch(ctx);
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_only.empty() && g_only != name) {
    launch(ctx);
    return;
  }
  Rec r{name, take_event(), take_event()};
  cudaEventRecord(r.a, st);
  launch(ctx);
  cudaEventRecord(r.b, st);
  g_recs.push_back(r);
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return PDF_OK;
}

extern "C" pdf_status pdf_profile_only(const char* kernel) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_only = kernel ? kernel : "";
  return PDF_OK;
}

extern "C" pdf_status pdf_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Rec& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return PDF_OK;
}

extern "C" pdf_status pdf_profile_query(const char* kernel, int64_t* launches, double* total_ms) {
  if (!kernel || !launches || !total_ms) return fail(PDF_EINVAL, "pdf_profile_query: NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = 0;
  double ms = 0.0;
  for (Rec& r : g_recs) {
    if (std::string(r.name) != kernel) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "pdf_profile_query");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "pdf_profile_query");
    ms += t;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  return PDF_OK;
}

extern "C" int64_t pdf_kernel_launches(void) { return g_launches.load(); }
