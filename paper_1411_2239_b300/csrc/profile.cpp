// Per-kernel CUDA-event instrumentation (see rv_profile_enable in rv.h).
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "profile.h"
#include "rv_internal.h"

namespace {
struct Pending { std::string name; cudaEvent_t a, b; };
struct Stat { std::string name; uint64_t launches; double ms; };
std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<Stat> g_stats;
std::vector<cudaEvent_t> g_free;
thread_local const char* t_name = nullptr;
thread_local cudaEvent_t t_begin = nullptr;
std::atomic<uint64_t> g_launches{0};

cudaEvent_t get_event() {
  if (!g_free.empty()) { cudaEvent_t e = g_free.back(); g_free.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void rv_prof_begin(const char* name, cudaStream_t s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  t_name = name;
  t_begin = get_event();
  cudaEventRecord(t_begin, s);
}

void rv_prof_end(cudaStream_t s) {
  if (!g_on || !t_begin) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = get_event();
  cudaEventRecord(e, s);
  g_pending.push_back({t_name, t_begin, e});
  t_begin = nullptr;
}

bool rv_prof_enabled() { return g_on; }

void rv_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" void rv_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
}

extern "C" uint64_t rv_launch_count(void) { return g_launches.load(); }

extern "C" int rv_profile_collect(rv_kernel_stat* out, int max) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    bool found = false;
    for (auto& st : g_stats)
      if (st.name == p.name) { st.launches++; st.ms += ms; found = true; break; }
    if (!found) g_stats.push_back({p.name, 1, (double)ms});
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  int n = (int)g_stats.size();
  for (int i = 0; i < n && i < max && out; ++i) {
    memset(&out[i], 0, sizeof(rv_kernel_stat));
    strncpy(out[i].name, g_stats[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = g_stats[i].launches;
    out[i].total_ms = g_stats[i].ms;
  }
  g_stats.clear();
  return n;
}

namespace {
std::mutex g_once_mu;
bool g_once_done[RV_MAX_DEVICES][RV_ONCE_SLOTS];
int g_sms[RV_MAX_DEVICES];
}  // namespace

rv_status rv_once_per_device(int slot, rv_status (*fn)()) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rv_fail(RV_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= RV_MAX_DEVICES || slot < 0 || slot >= RV_ONCE_SLOTS)
    return rv_fail(RV_EINVAL, "device %d beyond the %d the library supports", dev, RV_MAX_DEVICES);
  std::lock_guard<std::mutex> lk(g_once_mu);
  if (g_once_done[dev][slot]) return RV_OK;
  rv_status st = fn();
  if (st == RV_OK) g_once_done[dev][slot] = true;
  return st;
}

int rv_num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RV_MAX_DEVICES) return 148;
  std::lock_guard<std::mutex> lk(g_once_mu);
  if (!g_sms[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 148;
    g_sms[dev] = sms;
  }
  return g_sms[dev];
}
