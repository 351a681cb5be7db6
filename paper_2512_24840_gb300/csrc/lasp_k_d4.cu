// FP32 CUDA-core kernels for Legendre degree D = 4.
#define LASP_DEFINE_LAUNCHERS
#include "lasp_launch.cuh"

namespace lasp {
LASP_INSTANTIATE(4)
}  // namespace lasp
