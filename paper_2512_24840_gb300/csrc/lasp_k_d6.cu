// FP32 CUDA-core kernels for Legendre degree D = 6.
#define LASP_DEFINE_LAUNCHERS
#include "lasp_launch.cuh"

namespace lasp {
LASP_INSTANTIATE(6)
}  // namespace lasp
