// Kernels for f64 population storage.
#define VPLBM_STORE vplbm::kF64
#define VPLBM_SUFFIX f64
#include "vplbm_kernels_impl.cuh"
