// Host-side launchers of the per-storage kernel instantiations.
#pragma once

#include <cuda_runtime.h>

#include "vplbm_params.h"

namespace vplbm {

#define VPLBM_DECLARE_LAUNCHERS(SUFFIX)                                                         \
  cudaError_t launch_fused_##SUFFIX(int coll, const StepParams& p, cudaStream_t st);            \
  cudaError_t launch_group_##SUFFIX(const StepParams* d_params,                                 \
                                    const GroupTile* d_table, int n_blocks, long long k,         \
                                    int mode, cudaStream_t st);                                 \
  cudaError_t launch_moments_##SUFFIX(const StepParams& p, double* rho, double* ux, double* uy, \
                                      cudaStream_t st);                                         \
  cudaError_t launch_momentum_exchange_##SUFFIX(const StepParams& p, const MeArgs& m,            \
                                                cudaStream_t st);                               \
  cudaError_t launch_init_##SUFFIX(const StepParams& p, void* dst, const double* u, double rho0, \
                                   double u0x, double u0y, cudaStream_t st);                    \
  cudaError_t launch_ghost_init_##SUFFIX(const StepParams& p, const void* src, void* ghost,     \
                                        void* z, cudaStream_t st);                              \
  cudaError_t launch_export_##SUFFIX(const StepParams& p, const void* src, double* f,           \
                                     cudaStream_t st);                                          \
  cudaError_t launch_import_##SUFFIX(const StepParams& p, void* dst, const double* f,           \
                                     cudaStream_t st);

VPLBM_DECLARE_LAUNCHERS(f64)
VPLBM_DECLARE_LAUNCHERS(f32)
VPLBM_DECLARE_LAUNCHERS(f16)
VPLBM_DECLARE_LAUNCHERS(bf16)

}  // namespace vplbm
