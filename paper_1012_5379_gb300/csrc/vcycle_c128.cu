// Complex FP64 (HELM_C128) instantiation of the V-cycle kernels.
#include "vcycle_launch.cuh"
namespace helm {
HELM_VCYCLE_INST(double2)

// This translation unit's copy of the V-cycle error flag (the complex128 kernels'):
// read and clear.
int vcycle_take_error_c128() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_vcycle_error, sizeof(int)) != cudaSuccess) return 1;
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_vcycle_error, &z, sizeof(int));
  }
  return v;
}
}
