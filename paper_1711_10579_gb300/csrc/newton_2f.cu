// The persistent and group kernels of 2x2 blocks in FP32 (mixed precision) (newton.cuh).
#include "newton.cuh"

namespace pf {
PF_NEWTON_INSTANTIATE(2, float)
}  // namespace pf
