// Instantiates the kernels of one storage type (VPLBM_STORE, VPLBM_SUFFIX)
// and defines its launchers.
#include "vplbm_device.cuh"
#include "vplbm_launch.h"

#define VPLBM_CAT2(a, b) a##b
#define VPLBM_CAT(a, b) VPLBM_CAT2(a, b)
#define VPLBM_FN(name) VPLBM_CAT(name, VPLBM_SUFFIX)

namespace vplbm {

static dim3 node_grid(const StepParams& p) {
  return dim3((p.nx + kBlockX - 1) / kBlockX, (p.ny + kBlockY - 1) / kBlockY);
}

template <int COLL>
static cudaError_t launch_fused_coll(const StepParams& p, cudaStream_t st) {
  if (p.mode == kModeAAPush) {
    fused_step_kernel<VPLBM_STORE, COLL, kModeAAPush><<<p.n_tiles, dim3(kLanes, warps_per_block(VPLBM_STORE)), 0, st>>>(p);
  } else if (p.mode == kModeAALocal) {
    fused_step_kernel<VPLBM_STORE, COLL, kModeAALocal><<<p.n_tiles, dim3(kLanes, warps_per_block(VPLBM_STORE)), 0, st>>>(p);
  } else {
    fused_step_kernel<VPLBM_STORE, COLL, kModeAB><<<p.n_tiles, dim3(kLanes, warps_per_block(VPLBM_STORE)), 0, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_fused_)(int coll, const StepParams& p, cudaStream_t st) {
  return coll == kTrt ? launch_fused_coll<kTrt>(p, st) : launch_fused_coll<kMrt>(p, st);
}

cudaError_t VPLBM_FN(launch_group_)(const StepParams* d_params, const GroupTile* d_table,
                                    int n_blocks, long long k, int mode, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  const dim3 blk(kLanes, warps_per_block(VPLBM_STORE));
  if (mode == kModeAAPush)
    fused_group_kernel<VPLBM_STORE, kModeAAPush><<<n_blocks, blk, 0, st>>>(d_params, d_table, k);
  else if (mode == kModeAALocal)
    fused_group_kernel<VPLBM_STORE, kModeAALocal><<<n_blocks, blk, 0, st>>>(d_params, d_table, k);
  else
    fused_group_kernel<VPLBM_STORE, kModeAB><<<n_blocks, blk, 0, st>>>(d_params, d_table, k);
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_moments_)(const StepParams& p, double* rho, double* ux, double* uy,
                                      cudaStream_t st) {
  StepParams q = p;
  q.ghost_dst = nullptr;  // read only: the outlet state is not advanced
  moments_kernel<VPLBM_STORE><<<node_grid(q), dim3(kBlockX, kBlockY), 0, st>>>(q, rho, ux, uy);
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_momentum_exchange_)(const StepParams& p, const MeArgs& m, cudaStream_t st) {
  momentum_exchange_kernel<VPLBM_STORE><<<kMeBlocks, kThreads, 0, st>>>(p, m);
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_init_)(const StepParams& p, void* dst, const double* u, double rho0,
                                   double u0x, double u0y, cudaStream_t st) {
  init_kernel<VPLBM_STORE><<<node_grid(p), dim3(kBlockX, kBlockY), 0, st>>>(p, dst, u, rho0, u0x, u0y);
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_ghost_init_)(const StepParams& p, const void* src, void* ghost, void* z,
                                         cudaStream_t st) {
  ghost_init_kernel<VPLBM_STORE><<<(3 * p.ny + 255) / 256, 256, 0, st>>>(p, src, ghost, z);
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_export_)(const StepParams& p, const void* src, double* f, cudaStream_t st) {
  export_kernel<VPLBM_STORE><<<node_grid(p), dim3(kBlockX, kBlockY), 0, st>>>(p, src, f);
  return cudaGetLastError();
}

cudaError_t VPLBM_FN(launch_import_)(const StepParams& p, void* dst, const double* f, cudaStream_t st) {
  import_kernel<VPLBM_STORE><<<node_grid(p), dim3(kBlockX, kBlockY), 0, st>>>(p, dst, f);
  return cudaGetLastError();
}

}  // namespace vplbm
