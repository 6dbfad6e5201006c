#include "profiler.h"

#include <atomic>
#include <map>
#include <mutex>
#include <sstream>
#include <vector>

namespace helm {

namespace {
struct Rec {
  std::string name;
  cudaEvent_t a, b;
  double bytes, flops;
};
std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::string g_prefix;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

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

unsigned long long launch_count() { return g_launches.load(); }

void profile_begin(const std::string& prefix) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = true;
  g_prefix = prefix;
  for (auto& r : g_recs) { g_pool.push_back(r.a); g_pool.push_back(r.b); }
  g_recs.clear();
}

std::string profile_end() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  struct Agg { long n = 0; double ms = 0, bytes = 0, flops = 0; };
  std::map<std::string, Agg> agg;
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      Agg& a = agg[r.name];
      a.n += 1;
      a.ms += ms;
      a.bytes += r.bytes;
      a.flops += r.flops;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  std::ostringstream os;
  os.precision(17);
  os << "{";
  bool first = true;
  for (auto& kv : agg) {
    if (!first) os << ", ";
    first = false;
    os << "\"" << kv.first << "\": {\"launches\": " << kv.second.n << ", \"ms\": " << kv.second.ms
       << ", \"bytes\": " << kv.second.bytes << ", \"flops\": " << kv.second.flops << "}";
  }
  os << "}";
  return os.str();
}

Launch::Launch(const char* name, cudaStream_t st, double bytes, double flops, int kernels) : st_(st) {
  g_launches.fetch_add((unsigned long long)kernels);
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || std::string(name).compare(0, g_prefix.size(), g_prefix) != 0) return;
  Rec r{name, take_event(), take_event(), bytes, flops};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  slot_ = (int)g_recs.size() - 1;
}

Launch::~Launch() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot_ < (int)g_recs.size()) cudaEventRecord(g_recs[slot_].b, st_);
}

}  // namespace helm
