// The persistent and group kernels of 2x2 blocks in FP64 (newton.cuh).
#include "newton.cuh"

namespace pf {
PF_NEWTON_INSTANTIATE(2, double)
}  // namespace pf
