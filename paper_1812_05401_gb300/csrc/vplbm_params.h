// Parameters shared between the host runtime and the device kernels of the
// VP-LBM solver.
#pragma once

#include <stdint.h>

namespace vplbm {

enum { kF64 = 0, kF32 = 1, kF16 = 2, kBF16 = 3 };
// Collision kernels: kTrt, the two-rate form (SRT, and MRT whose even
// moments relax at one rate and odd moments at another, as the printed S
// does); kMrt, the moment-space form for any other rates.
enum { kTrt = 0, kMrt = 1 };
enum { kBcPeriodic = 0, kBcInletOutlet = 1, kBcFreeSlip = 2, kBcInletConvective = 3 };
// Streaming schemes of the fused step: A/B buffers (pull from src, write dst),
// or in-place AA-pattern streaming on one buffer, whose steps alternate
// between a push step (pull from the opposite slots of the neighbours, push
// to their own slots) and a local step (read own slots, write the opposite
// slots of the same node).
enum { kModeAB = 0, kModeAAPush = 1, kModeAALocal = 2 };

constexpr int kMaxBodies = 8;
// Fused-step tiles: a block is warps_per_block(storage) warps; each warp
// covers one row segment of 32 lanes x npt(storage) consecutive nodes and
// rows_per_warp rows (warps_per_block apart), so a tile is (32 npt) x tile_y
// nodes, tile_y = warps_per_block x rows_per_warp. npt makes each lane's
// access 16 bytes for FP32/FP64 storage (8 bytes for the 16-bit forms). The
// tile height (8, 16 or 32 rows) is chosen per solver: 32 for grids with
// enough tiles to fill the GPU several times over, shorter ones for grids
// that would leave most of the last wave of blocks idle.
constexpr int kLanes = 32;
constexpr int kWarpsMax = 8;
constexpr int kThreads = kLanes * kWarpsMax;  // also the block of the generic reduction kernels
constexpr int kTileRowsMin = 8;
constexpr int kTileRowsMax = 32;
// Warps per fused-step block: 8 for the 8- and 4-byte stores, 4 for the
// 16-bit stores. The 16-bit kernels are bound by instruction issue; with
// half-size blocks a warp does twice the rows per tile and fewer warps wait
// at the per-tile reduction barrier (16384 x 4096 FP16 step 0.4461 vs
// 0.4408 ms; the FP32 step loses 1% with 4 warps and keeps 8).
__host__ __device__ constexpr int warps_per_block(int storage) {
  return storage == kF16 || storage == kBF16 ? 4 : 8;
}
__host__ __device__ constexpr int threads_per_block(int storage) {
  return kLanes * warps_per_block(storage);
}
// Resident blocks per SM the fused kernel is compiled for: 3 for the 8- and
// 4-byte stores (80 registers per thread, 24 warps per SM, no spills), 8
// blocks of 4 warps for the 16-bit stores (64 registers, 32 warps), whose
// kernels are instruction-issue-bound and gain more from warps than they lose
// to a few spilled registers (measured on the 16384 x 4096 MRT step with
// 8-warp blocks: FP32 0.784 vs 0.805 ms at 3 vs 4 blocks; FP16 0.735 vs
// 0.699 ms).
__host__ __device__ constexpr int min_blocks_per_sm(int storage) {
  return storage == kF16 || storage == kBF16 ? 8 : 3;
}
__host__ __device__ constexpr int npt(int storage) { return storage == kF64 ? 2 : 4; }
__host__ __device__ constexpr int tile_x(int storage) { return kLanes * npt(storage); }

// Block shape of the per-node kernels (initialisation, moments, import/export).
constexpr int kBlockX = 64;
constexpr int kBlockY = 4;
constexpr int kGroup = 256;             // tiles per first-level reduction group
constexpr int kMeBlocks = 304;          // fixed grid of the momentum-exchange reduction (2 per SM)
constexpr uint8_t kStaticSolid = 255;   // mask value of a node solid through the static mask

// State of one rigid body at the time of a step.
struct BodyState {
  double cx, cy, vx, vy, omega;
};

// Collision and forcing constants in the arithmetic type of the kernel (the
// FP32 kernels read float copies: converting FP64 parameters per thread would
// run at the FP64 rate).
template <class T>
struct Consts {
  T s_e, s_eps, s_qx, s_qy, s_pxx, s_pxy;  // MRT rates
  // two-rate form, s+ (even moments) and s- (odd moments), c+- = 1 - s+-/2:
  T t_hsp, t_hsm;   // s+/2, s-/2
  T t_1msp, t_sp;   // 1 - s+, s+
  T t_c3p;          // 3 c+
  T t_a[2], t_b[2];    // w 4.5 s+ and w 9 c+ for w = 1/9, 1/36
  T t_am[2], t_bm[2];  // w 3 s- and w 3 c-
  T a_s, kappa_s;                         // 1/(2 eta) and (1/eta)/(1 + 1/(2 eta))
  T gx, gy;                               // body force per unit mass
  T heq_in[9];                            // inlet ghost f_eq(1, u_in) - w
  T h_ref[9];                             // 16-bit stores: elements hold h - h_ref
  // h_ref[a] - h_ref[b] for the opposite pairs (1,3), (2,4), (5,7), (6,8):
  // the fused step's two-rate collision decodes pair differences of stored
  // elements with them (h_ref is odd in xi: pair sums need no decoding)
  T r_d[4];
  T u_conv, conv_inv;                     // convective outlet: U_c and 1/(1 + U_c)
  T body[kMaxBodies][5];                  // cx, cy, vx, vy, omega of each body
};

// Everything one fused step of one solver needs (passed by value as a
// __grid_constant__ kernel parameter, or from a device array when grouped).
struct StepParams {
  const void* src;          // f*(t), storage element type, [9][ny][pitch]
  void* dst;                // f*(t+1)
  const uint8_t* mask;      // [ny][pitch]: 0 fluid, 1..kMaxBodies body, 255 static solid
  const void* us;           // static solid velocity, float2/double2 [ny][pitch], or null
  const void* ghost_src;    // convective outlet state g^{t-1}: [3][ny] of the arithmetic
  void* ghost_dst;          // type (offsets, rows alpha = 3, 6, 7); g^t goes to ghost_dst
  int mode;                 // kModeAB | kModeAAPush | kModeAALocal
  void* z;                  // AA, open outlet: stored f*(nx-1) of alpha = 3, 6, 7 ([3][ny])
  void* lost;               // AA, open x sides: values a push step sends out of the grid,
                            // [2][3][ny]: x = nx-1 alpha = 1, 5, 8; x = 0 alpha = 3, 6, 7
  int nx, ny, pitch;
  int bc_x, bc_y;
  int tiles_x, n_tiles;
  int tile_y, rows_per_warp;  // tile height (8, 16 or 32) and tile_y / warps_per_block
  int n_bodies;
  long long plane;          // pitch * ny
  Consts<double> cd;        // constants for the FP64 kernels
  Consts<float> cf;         // the same, rounded, for the FP32 kernels
  double* partials;         // [n_tiles][3]
  double* group_partials;   // [n_groups][3]
  unsigned* counters;       // [n_groups + 1], zero between steps
  double* ring;             // [ring_len][3]: F_x, F_y, sum rho per step
  int* flag;                // set to 1 on divergence
  long long t;              // index of this step
  int ring_len;
  int reduce_mass;
  int stochastic;           // 16-bit stores: 1 = stochastic rounding, 0 = nearest even
  int collision;            // kTrt | kMrt (read by the grouped kernel)
  int force_free;           // 1: no body force (g = 0), so fluid nodes feel no force
  unsigned round_key;       // stochastic rounding: key of the seed, mixed with the step
};

__host__ __device__ constexpr int elem_bytes(int storage) {
  return storage == kF64 ? 8 : (storage == kF32 ? 4 : 2);
}

template <class T> __host__ __device__ inline const Consts<T>& consts(const StepParams& p);
template <> __host__ __device__ inline const Consts<double>& consts<double>(const StepParams& p) { return p.cd; }
template <> __host__ __device__ inline const Consts<float>& consts<float>(const StepParams& p) { return p.cf; }

struct GroupTile {
  int solver;
  int tile;
};

// Arguments of the momentum-exchange reduction: a box of candidate solid
// nodes (inclusive bounds; empty when x1 < x0), united on the device with the
// box of the static solid layer, and the reduction's scratch and output.
struct MeArgs {
  int x0, y0, x1, y1;
  const int* static_box;  // device {x0, y0, x1, y1} of the static layer
  double* partials;       // [kMeBlocks][2]
  unsigned* counter;      // zero on entry, left zero
  double* out;            // F_x, F_y
};

}  // namespace vplbm
