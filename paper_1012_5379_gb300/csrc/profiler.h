// Launch accounting: a process-wide count of the kernels this library launched and,
// when enabled, CUDA-event timing of launches whose class name starts with a chosen
// prefix, together with the algorithmic bytes and flops of each launch.
#pragma once
#include <cuda_runtime.h>

#include <string>

namespace helm {

unsigned long long launch_count();
void profile_begin(const std::string& prefix);
// Stops profiling, waits for the recorded events and returns a JSON object
// {"class": {"launches": n, "ms": t, "bytes": b, "flops": f}, ...}.
std::string profile_end();

// Brackets one kernel launch (or a short sequence of launches counted as `kernels`).
class Launch {
 public:
  Launch(const char* name, cudaStream_t st, double bytes, double flops, int kernels = 1);
  ~Launch();
  Launch(const Launch&) = delete;
  Launch& operator=(const Launch&) = delete;

 private:
  int slot_ = -1;
  cudaStream_t st_;
};

}  // namespace helm
