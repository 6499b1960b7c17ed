// Coupled-step kernels with __half population storage.
#include "lbm_kernels.cuh"

namespace pemlbm {
PEMLBM_INSTANTIATE(__half)
}  // namespace pemlbm
