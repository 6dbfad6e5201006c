// Complex FP32 (HELM_C64) instantiation of the V-cycle kernels.
#include "vcycle_launch.cuh"
namespace helm {
HELM_VCYCLE_INST(float2)
}
