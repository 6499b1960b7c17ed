// Coupled-step kernels with double population storage.
#include "lbm_kernels.cuh"

namespace pemlbm {
PEMLBM_INSTANTIATE(double)
}  // namespace pemlbm
