// Launch accounting: a process-wide count of the kernels this library launched and,
// when enabled, CUDA-event timing of launches whose class name starts with a chosen
// prefix, together with the algorithmic bytes and flops of each launch.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace helm {

unsigned long long launch_count();
void profile_begin(const std::string& prefix);
// Stops profiling, waits for the recorded events and returns a JSON object
// {"class": {"launches": n, "ms": t, "bytes": b, "flops": f}, ...}.
std::string profile_end();

// CUDA-graph support: while a capture sink is set on the calling thread, launches
// are counted into it and timed launches become event-record nodes of the graph;
// after a replay of that graph has completed, harvest() adds their times.
struct GraphRec {
  std::string name;
  cudaEvent_t a, b;
  double bytes, flops;
};
void capture_sink_begin(std::vector<GraphRec>* recs, int* kernels);
void capture_sink_end();
void harvest(const std::vector<GraphRec>& recs);
void release(std::vector<GraphRec>& recs);
void count_launches(int kernels);
int profile_generation();     // changes whenever profiling starts or stops, or launch choices change
void bump_launch_generation();  // launch choices changed: captured graphs are stale
bool profiling();

// Brackets one kernel launch (or a short sequence of launches counted as `kernels`).
class Launch {
 public:
  Launch(const char* name, cudaStream_t st, double bytes, double flops, int kernels = 1);
  ~Launch();
  Launch(const Launch&) = delete;
  Launch& operator=(const Launch&) = delete;

 private:
  int slot_ = -1;
  bool graph_ = false;
  cudaStream_t st_;
};

}  // namespace helm
