// The persistent and group kernels of 6x6 blocks in FP32 (mixed precision) (newton.cuh).
#include "newton.cuh"

namespace pf {
PF_NEWTON_INSTANTIATE(6, float)
}  // namespace pf
