/*
 * vplbm — C ABI of the GB300 (sm_103a) volume-penalization lattice Boltzmann
 * solver (Benamour, Liberge, Beghein, arXiv 1812.05401).
 *
 * One solver holds one D2Q9 grid on one GPU. Each time step is one fused CUDA
 * kernel that, for every node (fluid and solid alike, Section 2.2), pulls the
 * nine populations, forms the density (Eq. density) and the implicit penalized
 * velocity (Eq. vitesse_fluide_penalisation_1), evaluates the penalization
 * force f = -rho (chi/eta)(u - u_s) (Eq. 17), collides with SRT + Guo
 * forcing (Eqs. LatticeBoltz, Guo1) or MRT + Lu forcing (Eqs. equa_lbl_mrt,
 * Guo2), writes the post-collision populations, and reduces in FP64 the force
 * on the solids and the total mass. Moving rigid bodies get their staircase
 * mask and solid velocity rewritten by a second kernel before each step.
 *
 * Conventions shared by every entry point:
 *  - Node (i, j) sits at (x, y) = (i, j); lattice spacing and time step are 1.
 *  - Host arrays are row-major doubles: fields [ny][nx], vectors [2][ny][nx]
 *    (component, then row, then column), populations [9][ny][nx] with the
 *    velocity order of Eq. vecteurs_D2Q9: 0 rest, 1..4 = E, N, W, S,
 *    5..8 = NE, NW, SW, SE.
 *  - The solver owns its device memory (taken from the caller's allocator when
 *    the configuration sets the device memory hook); the caller owns every
 *    pointer it passes and every output buffer. Nothing is retained after a
 *    call returns.
 *  - Calls are asynchronous on the solver's stream unless stated; a call that
 *    returns data to the host synchronizes that stream.
 *  - No C++ exception crosses the ABI. A failing call returns a status and
 *    leaves a message for vplbm_last_error. VPLBM_ERR_CUDA is sticky: the
 *    handle then only accepts vplbm_destroy.
 *  - A handle is used by one host thread at a time.
 *  - Before any call, an earlier call's kernels on the same stream have been
 *    ordered: no extra synchronization is needed between calls.
 */
#ifndef VPLBM_H
#define VPLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VPLBM_OK = 0,
  VPLBM_ERR_INVALID = 1,  /* bad argument or configuration */
  VPLBM_ERR_NOMEM = 2,    /* device allocation failed or budget exceeded */
  VPLBM_ERR_CUDA = 3,     /* CUDA runtime error (sticky) */
  VPLBM_ERR_DIVERGED = 4, /* a step produced rho <= 0 or a non-finite velocity */
  VPLBM_ERR_TIMEOUT = 5,  /* reserved: no kernel of this library waits on the device */
  VPLBM_ERR_STATE = 6     /* call not valid in the handle's current state */
} vplbm_status;

/* Collision operator. */
enum { VPLBM_SRT = 0, /* BGK, Eq. LatticeBoltz with Guo forcing, Eq. Guo1 */
       VPLBM_MRT = 1  /* Eq. equa_lbl_mrt with Lu forcing, Eq. Guo2 */ };

/* Population storage. Arithmetic is FP64 for VPLBM_F64 and FP32 otherwise.
 * VPLBM_F64 stores f_alpha; VPLBM_F32 stores f_alpha - w_alpha in 32 bits
 * (the same bytes, a finer rounding step); the *_OFFSET forms store, in 16
 * bits, f_alpha - r_alpha, rounded as vplbm_config.rounding says
 * (stochastically by default). The reference r is w (the rest state), and for
 * a flow with an inlet (bc_x INLET_*) r = w + (3/2) w xi_x u_in,x, half of the
 * inlet equilibrium's momentum term along x, rounded to multiples of 2^-28:
 * a channel's populations lie between the stagnant wake and the free stream,
 * within about half the stream's offsets of r everywhere, which halves the
 * largest elements and their rounding steps. r is odd in xi (it adds nothing
 * to density or to sums of opposite populations) and even in xi_y (a
 * population and its mirror image at a free-slip wall share it). */
enum { VPLBM_F64 = 0, VPLBM_F32 = 1, VPLBM_F16_OFFSET = 2, VPLBM_BF16_OFFSET = 3 };

/* Rounding of the 16-bit stores. NEAREST: round to nearest even.
 * STOCHASTIC (the default): round up or down with probabilities given by the
 * distance to the two neighbouring 16-bit values, from counter-based random
 * bits (a hash of the node, the direction and the step), so rounding errors
 * average out instead of acting as a systematic forcing. Ignored for
 * FP64/FP32 storage. */
enum { VPLBM_ROUND_NEAREST = 0, VPLBM_ROUND_STOCHASTIC = 1 };

/* Boundary conditions, applied inside the pull (streaming) of each step.
 * x: PERIODIC, or INLET_OUTLET: a ghost column x = -1 held at f_eq(1, u_in)
 *    (uniform velocity inlet) and a ghost column x = nx that repeats column
 *    nx - 1 (zero-gradient outlet), or INLET_CONVECTIVE: the same inlet and
 *    the convective outlet of Section 3.3 (after Yang): the ghost column
 *    x = nx of the three entering directions (3, 6, 7) keeps a state g,
 *    advanced each step by the implicit upwind step of dg/dt + U_c dg/dx = 0,
 *    g^t = (g^{t-1} + U_c f*(nx - 1; t)) / (1 + U_c), with U_c = u_conv;
 *    it starts as a copy of the last column whenever the populations are set
 *    (initial velocity, perturbation, vplbm_set_populations) and is part of
 *    the checkpoint.
 * y: PERIODIC, or FREE_SLIP: specular reflection off walls half-way beyond
 *    rows 0 and ny - 1 (the symmetry planes of Section 3.3). */
enum { VPLBM_BC_PERIODIC = 0, VPLBM_BC_INLET_OUTLET = 1, VPLBM_BC_FREE_SLIP = 2,
       VPLBM_BC_INLET_CONVECTIVE = 3 };

/* Streaming scheme. AB: two population buffers, each step pulls from one and
 * writes the other. AA: in-place streaming on one buffer (the AA pattern),
 * half the population memory with the same bytes moved per node update; steps
 * alternate between a push step (each node pulls from the opposite slots of
 * its neighbours and writes to their own slots) and a local step (each node
 * reads its own slots and writes its opposite slots). The stored values are
 * rounded with the same bits as in AB, so the two schemes give bitwise the
 * same populations, forces and moments; all entry points behave alike, except
 * vplbm_step_noalloc, which takes AB buffers only. */
enum { VPLBM_STREAM_AB = 0, VPLBM_STREAM_AA = 1 };

/* Largest number of rigid bodies a solver tracks. */
#define VPLBM_MAX_BODIES 8

/* Rigid circular body (staircase mask: a node is solid when its position lies
 * in the closed disc, Section 3.2). Centre at step t:
 *   (cx, cy) + (amp_x, amp_y) sin(2 pi t / period)   (period <= 0: fixed).
 * Solid velocity u_s = d centre/dt + omega e_z x (x - centre).
 * outside = 1 makes the solid the region r >= radius (an enclosing wall). */
typedef struct {
  double cx, cy, radius;
  double amp_x, amp_y, period;
  double omega;
  int32_t outside;
  int32_t reserved;
} vplbm_body;

typedef struct {
  int32_t nx, ny;          /* nodes, each >= 1 */
  int32_t collision;       /* VPLBM_SRT | VPLBM_MRT */
  int32_t storage;         /* VPLBM_F64 | VPLBM_F32 | VPLBM_F16_OFFSET | VPLBM_BF16_OFFSET */
  int32_t bc_x, bc_y;      /* see the boundary enum above */
  int32_t use_rates;       /* MRT: 1 takes the nine rates from rates[] */
  int32_t reduce_mass;     /* 1: record the total density of every step */
  double tau;              /* relaxation time > 1/2; nu = (tau - 1/2)/3; MRT s_n = 1/tau */
  double lambda;           /* MRT: s_q from Lambda = (1/s_n - 1/2)(1/s_q - 1/2) */
  double eta;              /* penalization parameter, > 0 (paper: 1e-7) */
  double u_in[2];          /* inlet velocity (bc_x = INLET_OUTLET or INLET_CONVECTIVE) */
  double rho0;             /* initial density */
  double u0[2];            /* initial uniform velocity */
  double body_force[2];    /* uniform force per unit mass g (f_tot = f_pen + rho g) */
  double rates[9];         /* explicit MRT S diagonal when use_rates = 1 */
  int32_t force_ring_len;  /* steps of (F_x, F_y, mass) kept on the device; >= 1 */
  int32_t rounding;        /* VPLBM_ROUND_NEAREST | VPLBM_ROUND_STOCHASTIC (16-bit stores) */
  void* stream;            /* cudaStream_t to run on, or NULL for a private stream */
  double u_conv;           /* convective outlet velocity U_c >= 0 (bc_x = INLET_CONVECTIVE) */
  int32_t streaming;       /* VPLBM_STREAM_AB (default) | VPLBM_STREAM_AA */
  int32_t tile_rows;       /* rows of a fused-step tile: 8, 16 or 32, or 0 (default) for
                              the tallest that gives the GPU's 152 SMs four waves of tiles;
                              the tiles fix the order of the force and mass sums */
  /* Device memory hook (optional): both set, or both NULL (the default:
   * stream-ordered allocation from the CUDA memory pool on the solver's
   * stream). When set, every device buffer the solver owns comes from
   * dev_alloc(bytes, alloc_ctx) and goes back through dev_free(ptr,
   * alloc_ctx): the populations, mask, reduction scratch and rings at
   * vplbm_create, the solid-velocity and momentum-exchange buffers when first
   * needed, and the staging buffers of host transfers. dev_alloc returns
   * memory on the current device, aligned to 256 bytes and ready for work
   * queued afterwards on the solver's stream (PyTorch's caching allocator on
   * that stream qualifies), or NULL when it has none: the call then fails
   * with VPLBM_ERR_NOMEM. A pointer that is not 256-byte aligned goes back
   * through dev_free and the call fails with VPLBM_ERR_INVALID. The library
   * waits for the solver's stream before every dev_free, so the allocator may
   * hand the block out again at once; calls that stage through a temporary
   * buffer therefore return after their device work. Both functions are
   * called on the thread that makes the library call. vplbm_group_step's
   * small per-call launch tables and vplbm_step_noalloc (which allocates
   * nothing) do not use the hook. */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  /* Seed of the stochastic rounding of the 16-bit stores (default 0): each
   * seed gives another realization of the rounding errors, for ensembles
   * that separate rounding noise from its systematic effect. */
  uint32_t rounding_seed;
  uint32_t reserved; /* 0 */
} vplbm_config;

typedef struct vplbm_solver vplbm_solver;

/* Fills cfg with defaults: SRT, FP32, periodic, tau 0.8, Lambda 3/16,
 * eta 1e-7, rho0 1, mass reduction on, ring of 4096 steps, stochastic
 * rounding of 16-bit stores. nx = ny = 0. */
void vplbm_config_init(vplbm_config* cfg);

/* Relaxation time for a reference speed u_ref, length l_ref and Reynolds
 * number re: nu = u_ref l_ref / re, tau = 3 nu + 1/2 (Section 2.1.1). */
double vplbm_tau_from_reynolds(double u_ref, double l_ref, double re);

/* Device bytes a solver with this configuration allocates at creation
 * (admission). Buffers taken later come on top when used: the static
 * solid-velocity field, the momentum-exchange records, the staging buffers
 * of host transfers. 0 for an invalid configuration. */
size_t vplbm_footprint_bytes(const vplbm_config* cfg);

/* Allocates the solver and sets the store to f*(0) = f_eq(rho0, u0) with an
 * all-fluid mask. INVALID for nx or ny < 1, tau <= 1/2, eta <= 0, a negative
 * or non-finite u_conv with the convective outlet, unknown enums, or only one
 * of dev_alloc and dev_free set; NOMEM if the device allocation fails. *out
 * is NULL on failure, and every buffer already taken has been released. */
vplbm_status vplbm_create(const vplbm_config* cfg, vplbm_solver** out);

/* Restarts from f*(0) = f_eq(rho0, u(x)) with u a host [2][ny][nx] array
 * (NULL: the uniform u0). Resets the step counter and the force record. */
vplbm_status vplbm_set_initial_velocity(vplbm_solver* s, const double* u);

/* Restarts like vplbm_set_initial_velocity with the seeded field
 * u = (u0x, u0y) + amp (2 r - 1), r in [0, 1) drawn on the device by SplitMix64
 * (Steele, Lea, Flood 2014) from `seed`: output number i + 1 for
 * i = (y nx + x) 2 + component, scaled by its top 53 bits. Bit-identical to
 * the same generator on the host, and needs no host-to-device copy of a field
 * (for admitting many solves quickly). */
vplbm_status vplbm_set_initial_perturbation(vplbm_solver* s, double u0x, double u0y, double amp,
                                            uint64_t seed);

/* Static mask and solid velocity (Section 2.2, Eq. 17): chi [ny][nx] bytes,
 * nonzero = solid; us [2][ny][nx] doubles or NULL (u_s = 0). on_device = 1:
 * both are device pointers. Replaces any earlier static mask; bodies set with
 * vplbm_set_bodies stay, and a static solid node takes precedence. */
vplbm_status vplbm_set_mask_and_solid_velocity(vplbm_solver* s, const uint8_t* chi,
                                               const double* us, int32_t on_device);

/* Rigid bodies (host array of n <= VPLBM_MAX_BODIES; n = 0 removes them).
 * The mask is rebuilt now and, when a body moves, over the region it sweeps
 * before every step. Where bodies overlap the lower index wins. */
vplbm_status vplbm_set_bodies(vplbm_solver* s, const vplbm_body* bodies, int32_t n);

/* Advances n >= 0 time steps (asynchronous). Step t maps f*(t) to f*(t+1)
 * with the mask and solid velocity of time t. */
vplbm_status vplbm_step(vplbm_solver* s, int64_t n);

/* Waits for the solver's stream and reports VPLBM_ERR_DIVERGED if any step
 * since the last check produced rho <= 0 or a non-finite velocity. */
vplbm_status vplbm_synchronize(vplbm_solver* s);

/* Steps taken since creation or the last restart. */
int64_t vplbm_step_count(const vplbm_solver* s);

/* Density and implicit velocity that the next step computes (pulled
 * populations of step t = vplbm_step_count). Outputs [ny][nx] doubles, host
 * (on_device = 0, synchronizes) or device (on_device = 1) pointers. */
vplbm_status vplbm_moments(vplbm_solver* s, double* rho, double* ux, double* uy,
                           int32_t on_device);

/* Post-collision store f*(t) as doubles [9][ny][nx] (host or device). */
vplbm_status vplbm_populations(vplbm_solver* s, double* f, int32_t on_device);

/* Replaces the store with f [9][ny][nx] (rounded to the storage type), keeping
 * the step counter: loads a checkpoint or a test state. */
vplbm_status vplbm_set_populations(vplbm_solver* s, const double* f, int32_t on_device);

/* Mask the next step uses: [ny][nx] bytes, 0 fluid, nonzero solid (host). */
vplbm_status vplbm_mask(vplbm_solver* s, uint8_t* chi);

/* Checkpoint and restart. vplbm_state_bytes: size of a saved state.
 * vplbm_save_state writes into the caller's host buffer (synchronizes) the
 * store f*(t) exactly as stored, the mask, the static solid-velocity field if
 * one is set, the convective outlet state, the in-place scheme's phase and
 * side arrays, and the step counter t. vplbm_load_state restores them into a
 * solver created with the same grid, storage, outlet and streaming scheme
 * (and the same bodies, whose motion depends on t): stepping on from a loaded
 * state is bitwise identical to never having stopped. INVALID if the state
 * does not match the solver. `bytes` is the size of buf: save refuses a
 * buffer shorter than vplbm_state_bytes, load one shorter than the state its
 * header describes (INVALID), so neither call reads or writes past it. */
size_t vplbm_state_bytes(const vplbm_solver* s);
vplbm_status vplbm_save_state(vplbm_solver* s, void* buf, size_t bytes);
vplbm_status vplbm_load_state(vplbm_solver* s, const void* buf, size_t bytes);

/* Per-step record since the previous call (synchronizes): F_x, F_y, the force
 * the fluid exerts on all solid nodes (minus the sum of Eq. 17 over them,
 * reduced in FP64), and the total density (0 if reduce_mass = 0). Returns up
 * to cap entries, oldest first, in *count; if more than force_ring_len steps
 * went unread the oldest were overwritten. Any pointer may be NULL. */
vplbm_status vplbm_forces(vplbm_solver* s, double* fx, double* fy, double* mass,
                          int64_t cap, int64_t* count);

/* As vplbm_forces, but without synchronizing: enqueues on the solver's
 * stream the copy of the records since the previous read into records
 * ([count][3]: F_x, F_y, mass; host memory, page-locked for the copy to be
 * asynchronous), returns their number in *count at once, and the data is
 * valid once the stream has reached this point (an event or a sync). */
vplbm_status vplbm_forces_async(vplbm_solver* s, double* records, int64_t cap, int64_t* count);

/* Momentum-exchange force on the solids (the force measure of Section 3.3,
 * after Ladd), a second measure beside the penalization-force records of
 * vplbm_forces. Over every link from a fluid node x_f to a solid node
 * x_s = x_f + xi_a (mask nonzero), the momentum xi_a [f*_a(x_f) + f*_abar(x_s)]
 * of the post-collision store f*(t) crosses into the solid; the force is the
 * sum over links, in lattice units, summed in FP64 in a fixed order (results
 * are bitwise reproducible). Links that would start outside a non-periodic
 * side of the grid are not counted. The reduction covers the bounding box of
 * the bodies at t and of the static mask layer, so its cost scales with the
 * solids, not with the grid.
 *
 * vplbm_momentum_exchange computes it once at the current state (step index
 * vplbm_step_count, the mask of that step) and synchronizes; fx, fy receive
 * the two components (either may be NULL).
 *
 * vplbm_enable_momentum_exchange(s, 1) makes every later vplbm_step record
 * it for its own step index t (from f*(t), before the step), one extra launch
 * per step, into a ring of force_ring_len records; 0 stops recording. Solvers
 * that record are stepped one by one inside vplbm_group_step.
 * vplbm_momentum_exchange_forces returns the records of the steps since the
 * previous read (or since recording began, up to where it stopped) like
 * vplbm_forces: at most cap entries, oldest first, count in *count;
 * VPLBM_ERR_STATE if recording was never enabled. */
vplbm_status vplbm_momentum_exchange(vplbm_solver* s, double* fx, double* fy);
vplbm_status vplbm_enable_momentum_exchange(vplbm_solver* s, int32_t enable);
vplbm_status vplbm_momentum_exchange_forces(vplbm_solver* s, double* fx, double* fy,
                                            int64_t cap, int64_t* count);

/* Advances n solvers by steps[i] steps each, batching them into grouped
 * launches (one launch per time step per storage/collision class covering
 * every solver still running). All solvers must share one stream. Results
 * are bitwise identical to vplbm_step on each solver alone. */
vplbm_status vplbm_group_step(vplbm_solver* const* solvers, int32_t n,
                              const int64_t* steps);

/* Kernel launches this solver issued on its hot path (fused steps and mask
 * updates) since creation. */
int64_t vplbm_launch_count(const vplbm_solver* s);

/* Timing of the fused step kernel: enable = 1 brackets each fused launch with
 * CUDA events on the solver's stream. vplbm_fused_timing synchronizes and
 * returns the summed device time (ms) and the number of timed launches since
 * the last read. */
vplbm_status vplbm_enable_timing(vplbm_solver* s, int32_t enable);
vplbm_status vplbm_fused_timing(vplbm_solver* s, double* total_ms, int64_t* launches);

/* One fused time step that allocates nothing (the paper has no counterpart:
 * this is a service for callers that cannot allocate device memory when they
 * step, such as code being captured into a CUDA graph, a host callback, a
 * real-time loop with a fixed memory budget, or a framework that owns every
 * allocation itself). The caller owns all the state; the library only runs
 * the fused kernel of vplbm_step on it.
 *
 *  cfg       the solver's configuration (nx, ny, collision, storage, boundary
 *            conditions, tau, lambda, eta, u_in, body_force, rates,
 *            reduce_mass, rounding, stream); rho0, u0 and force_ring_len are
 *            not read (a config filled by hand may leave them zero). stream
 *            must belong to the current device (NULL: its default stream).
 *  bodies    host array of n_bodies <= VPLBM_MAX_BODIES rigid bodies, evaluated
 *            at step t, or NULL with n_bodies = 0.
 *  f_src     device populations f*(t) in the storage type, [9][ny][pitch]
 *            (f for FP64, f - w for FP32, f - r for the 16-bit forms with r
 *            the reference of the storage enum's comment, in FP32:
 *            r = w + (f_eq(1, u_in) - w) / 2 for a flow with an inlet),
 *            16-byte aligned.
 *  f_dst     device output f*(t+1), same layout; must not alias f_src.
 *  mask      device [ny][pitch] bytes: 0 fluid, k = 1..n_bodies solid of body
 *            k (solid velocity from its motion), 255 solid with the velocity
 *            from us; any other nonzero value is a solid at rest (u_s = 0).
 *  us        device solid velocity, float2 (double2 for VPLBM_F64 storage)
 *            [ny][pitch], read at mask = 255 nodes, or NULL for u_s = 0.
 *  pitch     row length in elements: >= nx and a multiple of 8.
 *  t         step index (body positions and the record's meaning).
 *  record    device output of 3 doubles: F_x, F_y on the solids and the total
 *            density (0 if reduce_mass = 0), as in vplbm_forces.
 *  flag      device int set to 1 if the step produced rho <= 0 or a
 *            non-finite velocity (never cleared here), or NULL.
 *
 * Scratch: the per-tile and per-group reduction sums live in a fixed 1 MiB
 * device array inside the library, which every GPU that loads the library
 * holds until the process exits. It holds at most 43,491 tiles of the fused
 * step: with tiles of 128 x 32 nodes (FP32 and 16-bit storage) about 178.1M
 * nodes, with tiles of 64 x 32 (FP64) about 89.1M. Larger grids are rejected
 * with VPLBM_ERR_INVALID and a message; use vplbm_create/vplbm_step for them.
 * The first call on a device looks up the array's device address (done once
 * per device, with that device current) and keeps it for the rest of the
 * process: make that first call before any stream capture, and call nothing
 * here after a cudaDeviceReset of that device (the kept address belongs to
 * the context the reset destroyed). Each call clears the array's counters on cfg->stream
 * before launching. All calls share the one array, so calls whose kernels
 * can overlap on the GPU (different streams without ordering) race and give
 * wrong results: order them on one stream. Asynchronous on cfg->stream;
 * returns VPLBM_ERR_INVALID for bad arguments (including the convective
 * outlet, whose state lives in a solver, and AA streaming) and VPLBM_ERR_CUDA
 * if a CUDA call fails. Calls no allocating routine. */
vplbm_status vplbm_step_noalloc(const vplbm_config* cfg, const vplbm_body* bodies,
                                int32_t n_bodies, const void* f_src, void* f_dst,
                                const uint8_t* mask, const void* us, int32_t pitch,
                                int64_t t, double* record, int* flag);

/* Message for the last failing call on this handle (never NULL). */
const char* vplbm_last_error(const vplbm_solver* s);

/* Why the calling thread's last vplbm_create failed ("" after a success;
 * never NULL): a failed creation leaves no handle to carry the message.
 * Valid until the thread's next vplbm_create. */
const char* vplbm_create_error(void);
const char* vplbm_status_string(vplbm_status st);

/* Frees everything the solver owns, stream-ordered: the memory returns once
 * the work already queued on the solver's stream completes; the host does not
 * wait. NULL is a no-op. Does not destroy a caller-supplied stream. */
void vplbm_destroy(vplbm_solver* s);

#ifdef __cplusplus
}
#endif
#endif /* VPLBM_H */
