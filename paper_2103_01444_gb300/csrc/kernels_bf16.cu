// Coupled-step kernels with __nv_bfloat16 population storage.
#include "lbm_kernels.cuh"

namespace pemlbm {
PEMLBM_INSTANTIATE(__nv_bfloat16)
}  // namespace pemlbm
