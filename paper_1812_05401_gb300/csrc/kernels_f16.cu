// Kernels for f16 population storage.
#define VPLBM_STORE vplbm::kF16
#define VPLBM_SUFFIX f16
#include "vplbm_kernels_impl.cuh"
