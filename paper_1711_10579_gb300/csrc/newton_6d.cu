// The persistent and group kernels of 6x6 blocks in FP64 (newton.cuh).
#include "newton.cuh"

namespace pf {
PF_NEWTON_INSTANTIATE(6, double)
}  // namespace pf
