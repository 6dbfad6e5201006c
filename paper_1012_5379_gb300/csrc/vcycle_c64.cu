// Complex FP32 (HELM_C64) instantiation of the V-cycle kernels.
#include "vcycle_launch.cuh"
namespace helm {
HELM_VCYCLE_INST(float2)

int vcycle_take_error() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_vcycle_error, sizeof(int)) != cudaSuccess) return 1;
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_vcycle_error, &z, sizeof(int));
  }
  return v;
}
}
