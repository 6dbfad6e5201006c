// Complex FP32 (HELM_C64) instantiation of the V-cycle kernels.
#include "vcycle_launch.cuh"
namespace helm {
HELM_VCYCLE_INST(float2)

// The error flag is a file-scope device variable, one copy per translation unit: this
// one (the complex64 kernels') and the complex128 unit's are read and cleared together.
int vcycle_take_error() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_vcycle_error, sizeof(int)) != cudaSuccess) return 1;
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_vcycle_error, &z, sizeof(int));
  }
  const int w = vcycle_take_error_c128();
  return v ? v : w;
}
}
