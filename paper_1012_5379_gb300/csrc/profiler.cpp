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
std::atomic<int> g_gen{0};
thread_local std::vector<GraphRec>* t_sink = nullptr;
thread_local int* t_sink_kernels = nullptr;
struct Agg { long n = 0; double ms = 0, bytes = 0, flops = 0; };
std::map<std::string, Agg> g_harvested;

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

void capture_sink_begin(std::vector<GraphRec>* recs, int* kernels) {
  t_sink = recs;
  t_sink_kernels = kernels;
}
void capture_sink_end() {
  t_sink = nullptr;
  t_sink_kernels = nullptr;
}
void count_launches(int kernels) { g_launches.fetch_add((unsigned long long)kernels); }
int profile_generation() { return g_gen.load(); }
void bump_launch_generation() { g_gen.fetch_add(1); }
bool profiling() { return g_on; }

void harvest(const std::vector<GraphRec>& recs) {
  if (recs.empty()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  for (const auto& r : recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();  // do not leave a sticky error for the caller's checks
      continue;
    }
    {
      Agg& a = g_harvested[r.name];
      a.n += 1;
      a.ms += ms;
      a.bytes += r.bytes;
      a.flops += r.flops;
    }
  }
}

void release(std::vector<GraphRec>& recs) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : recs) { g_pool.push_back(r.a); g_pool.push_back(r.b); }
  recs.clear();
}

void profile_begin(const std::string& prefix) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = true;
  g_prefix = prefix;
  g_gen.fetch_add(1);
  g_harvested.clear();
  for (auto& r : g_recs) { g_pool.push_back(r.a); g_pool.push_back(r.b); }
  g_recs.clear();
}

std::string profile_end() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  g_gen.fetch_add(1);
  std::map<std::string, Agg> agg = g_harvested;
  g_harvested.clear();
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
  if (t_sink) {
    *t_sink_kernels += kernels;
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (std::string(name).compare(0, g_prefix.size(), g_prefix) != 0) return;
    GraphRec r{name, take_event(), take_event(), bytes, flops};
    // an external record is a real event-record node of the captured graph
    cudaEventRecordWithFlags(r.a, st, cudaEventRecordExternal);
    t_sink->push_back(r);
    slot_ = (int)t_sink->size() - 1;
    graph_ = true;
    return;
  }
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
  if (graph_) {
    if (t_sink && slot_ < (int)t_sink->size()) cudaEventRecordWithFlags((*t_sink)[slot_].b, st_, cudaEventRecordExternal);
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot_ < (int)g_recs.size()) cudaEventRecord(g_recs[slot_].b, st_);
}

}  // namespace helm
