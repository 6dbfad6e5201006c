// Complex FP64 (HELM_C128) instantiation of the V-cycle kernels.
#include "vcycle_launch.cuh"
namespace helm {
HELM_VCYCLE_INST(double2)
}
