#include <map>
#include <mutex>
#include <string>
#include <vector>
#include <atomic>
#include "profile.cuh"
#include "../../include/az.h"

namespace az {
namespace {
struct Pending { cudaEvent_t a, b; };
struct Entry { int64_t launches = 0; double ms = 0; double bytes = 0; std::vector<Pending> pend; };
std::mutex mu;
std::map<std::string, Entry> tab;
std::vector<cudaEvent_t> pool, used;
std::atomic<int64_t> launches{0};
std::atomic<bool> enabled{false};
}  // namespace

void prof_count(int64_t n) { launches += n; }
bool prof_enabled() { return enabled.load(); }
cudaEvent_t prof_event() {
  std::lock_guard<std::mutex> g(mu);
  cudaEvent_t e;
  if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
  else cudaEventCreate(&e);
  used.push_back(e);
  return e;
}
void prof_record(const char* name, cudaEvent_t a, cudaEvent_t b, double bytes, int64_t n) {
  std::lock_guard<std::mutex> g(mu);
  Entry& en = tab[name];
  en.launches += n;
  en.bytes += bytes;
  en.pend.push_back({a, b});
}
}  // namespace az

using namespace az;

extern "C" {

int64_t az_launch_count(void) { return launches.load(); }

void az_profile_begin(void) {
  std::lock_guard<std::mutex> g(mu);
  tab.clear();
  for (cudaEvent_t e : used) pool.push_back(e);
  used.clear();
  enabled = true;
}

az_status az_profile_end(void) {
  enabled = false;
  std::lock_guard<std::mutex> g(mu);
  for (auto& kv : tab) {
    for (auto& p : kv.second.pend) {
      if (cudaEventSynchronize(p.b) != cudaSuccess) return AZ_ERR_CUDA;
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return AZ_ERR_CUDA;
      kv.second.ms += ms;
    }
    kv.second.pend.clear();
  }
  return AZ_OK;
}

az_status az_profile_query(int32_t i, char* name, int32_t name_len, int64_t* nlaunch, double* ms, double* bytes) {
  std::lock_guard<std::mutex> g(mu);
  if (i < 0 || i >= (int32_t)tab.size()) return AZ_ERR_ARG;
  auto it = tab.begin();
  std::advance(it, i);
  if (name && name_len > 0) {
    std::snprintf(name, name_len, "%s", it->first.c_str());
  }
  if (nlaunch) *nlaunch = it->second.launches;
  if (ms) *ms = it->second.ms;
  if (bytes) *bytes = it->second.bytes;
  return AZ_OK;
}

}  // extern "C"
