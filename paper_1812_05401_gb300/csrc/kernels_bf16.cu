// Kernels for bf16 population storage.
#define VPLBM_STORE vplbm::kBF16
#define VPLBM_SUFFIX bf16
#include "vplbm_kernels_impl.cuh"
