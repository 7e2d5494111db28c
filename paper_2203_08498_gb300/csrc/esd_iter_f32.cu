// FP32 instantiation of the iteration kernels (inner solves of the iterative refinement).
#include "esd_iter.cuh"

namespace esd {
ESD_INSTANTIATE_ITER(float)
}  // namespace esd
