// Kernels for f32 population storage.
#define VPLBM_STORE vplbm::kF32
#define VPLBM_SUFFIX f32
#include "vplbm_kernels_impl.cuh"
