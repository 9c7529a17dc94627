// Status strings, error bookkeeping and device queries of the C ABI.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gsp {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct Slot {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> used;
};
Slot g_slots[PROF_COUNT];
std::vector<cudaEvent_t> g_pool;
cudaEvent_t g_open[PROF_COUNT] = {};

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
const char* kProfNames[PROF_COUNT] = {"bins", "level0", "box_hist", "cast", "mttkrp_xy",
                                      "mttkrp_lst", "als_small", "tables", "range_query",
                                      "range_query_backward", "adam", "struct_tables",
                                      "struct_side", "struct_bins", "solve"};
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void prof_begin(int id, cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_relaxed) || id < 0 || id >= PROF_COUNT) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e = take_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) g_open[id] = e;
}

void prof_end(int id, cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_relaxed) || id < 0 || id >= PROF_COUNT) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t b = g_open[id];
  g_open[id] = nullptr;
  if (!b) return;
  cudaEvent_t e = take_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) g_slots[id].used.emplace_back(b, e);
}

int& last_cuda_error() {
  static thread_local int e = 0;
  return e;
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
    cached[dev] = n;
  }
  return cached[dev];
}

}  // namespace gsp

extern "C" int gsp_profile_enable(int on) {
  gsp::g_prof_on.store(on ? 1 : 0);
  return GSP_OK;
}

extern "C" void gsp_profile_reset(void) {
  std::lock_guard<std::mutex> lk(gsp::g_prof_mu);
  for (auto& sl : gsp::g_slots) {
    for (auto& pr : sl.used) {
      gsp::g_pool.push_back(pr.first);
      gsp::g_pool.push_back(pr.second);
    }
    sl.used.clear();
  }
}

extern "C" int gsp_profile_read(int id, int64_t* h_launches, double* h_total_ms) {
  if (id < 0 || id >= gsp::PROF_COUNT || !h_launches || !h_total_ms) return GSP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(gsp::g_prof_mu);
  double total = 0.0;
  for (auto& pr : gsp::g_slots[id].used) {
    GSP_CUDA(cudaEventSynchronize(pr.second));
    float ms = 0.0f;
    GSP_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
    total += ms;
  }
  *h_launches = static_cast<int64_t>(gsp::g_slots[id].used.size());
  *h_total_ms = total;
  return GSP_OK;
}

extern "C" const char* gsp_profile_name(int id) {
  if (id < 0 || id >= gsp::PROF_COUNT) return "";
  return gsp::kProfNames[id];
}

extern "C" uint64_t gsp_kernel_launches(void) { return gsp::g_launches.load(); }

extern "C" const char* gsp_strerror(int status) {
  switch (status) {
    case GSP_OK: return "ok";
    case GSP_ERR_INVALID_ARG: return "invalid argument";
    case GSP_ERR_CUDA: return "CUDA runtime error";
    case GSP_ERR_WORKSPACE: return "workspace too small";
    case GSP_ERR_NONFINITE: return "non-finite data";
    case GSP_ERR_NUMERIC: return "least-squares system could not be solved";
    case GSP_ERR_TIMEOUT: return "bounded device wait ran out";
    case GSP_ERR_UNSUPPORTED: return "unsupported on this device or build";
    default: return "unknown status";
  }
}

extern "C" int gsp_last_cuda_error(void) { return gsp::last_cuda_error(); }

extern "C" int gsp_version(void) { return 20000; }
