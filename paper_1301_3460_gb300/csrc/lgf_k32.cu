// FP32 instantiation of the iteration kernels (FP32 phase of the mixed mode).
#include "lgf_launch_impl.cuh"

namespace lgf {
LGF_INSTANTIATE(float)
}  // namespace lgf
