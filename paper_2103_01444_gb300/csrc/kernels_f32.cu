// Coupled-step kernels with float population storage.
#include "lbm_kernels.cuh"

namespace pemlbm {
PEMLBM_INSTANTIATE(float)
}  // namespace pemlbm
