// Host runtime of the VP-LBM solver: the C ABI of include/vplbm.h.
//
// A solver owns two population buffers (A/B ping-pong, [9][ny][pitch] in the
// storage type, rows padded to 128 bytes), the mask ([ny][pitch] bytes), an
// optional static solid-velocity field, the reduction scratch of the fused
// step and a ring of per-step (F_x, F_y, sum rho) records. Each time step is
// one launch of the fused kernel, preceded, when a body moves, by one launch
// of the mask update over the region the bodies sweep.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vplbm.h"
#include "vplbm_launch.h"
#include "vplbm_params.h"

using namespace vplbm;

namespace {

constexpr double kPi = 3.14159265358979323846;

struct BodyGeom {
  double cx, cy, r2;
  int outside;
};
struct BodyGeomSet {
  BodyGeom b[kMaxBodies];
  int n;
};

// Staircase mask of the rigid bodies over the box [x0, x0+w) x [y0, y0+h):
// a node takes the index (1-based) of the first body containing it, 0 if none;
// static solid nodes (255) are left alone. The in-disc test is evaluated with
// explicitly rounded FP64 operations (no contraction), so that the integer
// outcome is reproducible.
__global__ void mask_update_kernel(uint8_t* mask, int pitch, int x0, int y0, int w, int h,
                                   const __grid_constant__ BodyGeomSet g) {
  const int x = x0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= x0 + w || y >= y0 + h) return;
  const long long i = (long long)y * pitch + x;
  const uint8_t m = mask[i];
  if (m == kStaticSolid) return;
  uint8_t v = 0;
  for (int b = 0; b < g.n; ++b) {
    const double dx = __dsub_rn(double(x), g.b[b].cx);
    const double dy = __dsub_rn(double(y), g.b[b].cy);
    const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    const bool in = g.b[b].outside ? (r2 >= g.b[b].r2) : (r2 <= g.b[b].r2);
    if (in) {
      v = uint8_t(b + 1);
      break;
    }
  }
  if (v != m) mask[i] = v;
}

// Static mask import: chi != 0 -> 255; a node that was statically solid and is
// no longer becomes fluid (body nodes are then rebuilt by mask_update_kernel).
// Bounding box of the nonzero mask nodes, into box {x0, y0, x1, y1} (which
// holds {INT_MAX, INT_MAX, -1, -1} on entry).
__global__ void solid_box_kernel(const uint8_t* mask, int pitch, int nx, int ny, int* box) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const bool solid = x < nx && y < ny && mask[(long long)y * pitch + x] != 0;
  const unsigned any = __ballot_sync(0xffffffffu, solid);
  if (!any) return;
  const int lo_x = __reduce_min_sync(0xffffffffu, solid ? x : INT_MAX);
  const int lo_y = __reduce_min_sync(0xffffffffu, solid ? y : INT_MAX);
  const int hi_x = __reduce_max_sync(0xffffffffu, solid ? x : -1);
  const int hi_y = __reduce_max_sync(0xffffffffu, solid ? y : -1);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(box + 0, lo_x);
    atomicMin(box + 1, lo_y);
    atomicMax(box + 2, hi_x);
    atomicMax(box + 3, hi_y);
  }
}

__global__ void mask_import_kernel(uint8_t* mask, int pitch, int nx, int ny, const uint8_t* chi) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const long long i = (long long)y * pitch + x;
  const uint8_t c = chi[(long long)y * nx + x];
  const uint8_t m = mask[i];
  mask[i] = c ? kStaticSolid : (m == kStaticSolid ? uint8_t(0) : m);
}

__global__ void mask_export_kernel(const uint8_t* mask, int pitch, int nx, int ny, uint8_t* chi) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  chi[(long long)y * nx + x] = mask[(long long)y * pitch + x] ? 1 : 0;
}

// Static solid velocity [2][ny][nx] doubles -> {float2|double2}[ny][pitch].
template <class T2>
__global__ void us_import_kernel(T2* us, int pitch, int nx, int ny, const double* src) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const long long o = (long long)y * nx + x;
  const long long nn = (long long)nx * ny;
  T2 v;
  v.x = src[o];
  v.y = src[nn + o];
  us[(long long)y * pitch + x] = v;
}

// Seeded initial velocity: u = u0 + amp (2 r - 1) per node and component, r
// the SplitMix64 (Steele, Lea, Flood 2014) output number i + 1 of the seed
// (i = (y nx + x) 2 + component) scaled to [0, 1) by its top 53 bits. The
// operations are explicitly rounded, so the field is bit-identical to the
// same generator evaluated on the host.
__global__ void perturbation_kernel(double* u, int nx, int ny, double u0x, double u0y, double amp,
                                    unsigned long long seed) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nn = (long long)nx * ny;
  if (node >= nn) return;
  double r2[2];
  for (int c = 0; c < 2; ++c) {
    const unsigned long long i = (unsigned long long)node * 2ull + (unsigned long long)c + 1ull;
    unsigned long long z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double r = __dmul_rn(double(z >> 11), 1.0 / 9007199254740992.0);
    r2[c] = __dmul_rn(amp, __dsub_rn(__dmul_rn(2.0, r), 1.0));
  }
  u[node] = amp > 0.0 ? __dadd_rn(u0x, r2[0]) : u0x;
  u[nn + node] = amp > 0.0 ? __dadd_rn(u0y, r2[1]) : u0y;
}

dim3 grid2d(int w, int h, dim3 blk) {
  return dim3((w + blk.x - 1) / blk.x, (h + blk.y - 1) / blk.y);
}

// Element of the convective outlet state: the arithmetic type.
size_t ghost_elem(int storage) { return storage == kF64 ? sizeof(double) : sizeof(float); }

size_t element_size(int storage) {
  switch (storage) {
    case kF64: return 8;
    case kF32: return 4;
    default: return 2;
  }
}

int row_pitch(int nx, int storage) {
  const int per128 = int(128 / element_size(storage));
  return ((nx + per128 - 1) / per128) * per128;
}

}  // namespace

struct vplbm_solver {
  vplbm_config cfg{};
  int pitch = 0;
  long long plane = 0;
  size_t esize = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;

  void* f[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding f*(t)
  uint8_t* mask = nullptr;
  void* us = nullptr;
  double* partials = nullptr;
  double* group_partials = nullptr;
  unsigned* counters = nullptr;
  double* ring = nullptr;
  int* flag = nullptr;
  int* static_box = nullptr;  // device box {x0, y0, x1, y1} of the static solid layer
  void* ghost[2] = {nullptr, nullptr};  // convective outlet state of f[0], f[1] ([3][ny])
  // In-place (AA) streaming: one population buffer (f[1] aliases f[0]) and cur
  // is the phase (0: the next step is a push step, 1: a local step).
  bool aa = false;
  void* z = nullptr;     // AA, open outlet: stored f*(nx - 1) of alpha = 3, 6, 7
  void* lost = nullptr;  // AA, open x sides: values pushed out of the grid

  // Momentum-exchange force (Section 3.3): records per step when enabled.
  bool me_on = false;
  double* me_ring = nullptr;     // [force_ring_len][2]
  double* me_scratch = nullptr;  // [kMeBlocks][2] partials, then one on-demand result
  unsigned* me_counter = nullptr;
  int64_t me_read = 0;  // first step not yet returned by vplbm_momentum_exchange_forces
  int64_t me_stop = 0;  // step at which recording last stopped

  int tiles_x = 0, tiles_y = 0, n_tiles = 0, n_groups = 0;
  StepParams base{};  // constants; src/dst/t/bodies filled per step

  int64_t t = 0;
  int64_t ring_read = 0;  // first step not yet returned by vplbm_forces
  std::vector<vplbm_body> bodies;
  bool moving = false;
  int64_t mask_t = -1;  // time the moving bodies' mask reflects (-1: none)

  int64_t launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  double timed_ms = 0.0;
  int64_t timed_count = 0;

  std::string err;
  bool sticky = false;
};

namespace {

vplbm_status fail(vplbm_solver* s, vplbm_status st, const std::string& msg) {
  if (s) {
    s->err = msg;
    if (st == VPLBM_ERR_CUDA) s->sticky = true;
  }
  return st;
}

vplbm_status cuda_fail(vplbm_solver* s, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky in the runtime
    return fail(s, VPLBM_ERR_NOMEM, m);
  }
  return fail(s, VPLBM_ERR_CUDA, m);
}

#define VP_CUDA(s, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
  } while (0)

// Why the calling thread's last vplbm_create failed (no handle exists to
// carry the message).
thread_local std::string g_create_error;

// A named NVTX range over one library call, so that a profiler's timeline
// shows which launches a step or a grouped round made; without a profiler
// attached the calls do nothing.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

#define VP_OK(call)                          \
  do {                                       \
    vplbm_status st_ = (call);               \
    if (st_ != VPLBM_OK) return st_;         \
  } while (0)

// Device memory of a solver: from the caller's allocator when the
// configuration sets dev_alloc / dev_free, else stream-ordered from the CUDA
// memory pool on the solver's stream (neither allocation nor release
// synchronizes the device, so solvers can come and go while others run).
constexpr uintptr_t kAllocAlign = 256;

vplbm_status mem_get(vplbm_solver* s, void** p, size_t bytes) {
  *p = nullptr;
  if (!s->cfg.dev_alloc) {
    cudaError_t e = cudaMallocAsync(p, bytes, s->stream);
    return e == cudaSuccess ? VPLBM_OK : cuda_fail(s, e, "cudaMallocAsync");
  }
  void* q = s->cfg.dev_alloc(bytes, s->cfg.alloc_ctx);
  if (!q)
    return fail(s, VPLBM_ERR_NOMEM, "dev_alloc returned NULL for " + std::to_string(bytes) + " bytes");
  if (reinterpret_cast<uintptr_t>(q) % kAllocAlign != 0) {
    s->cfg.dev_free(q, s->cfg.alloc_ctx);
    return fail(s, VPLBM_ERR_INVALID, "dev_alloc returned a pointer not aligned to 256 bytes");
  }
  *p = q;
  return VPLBM_OK;
}

template <class T>
vplbm_status mem_get(vplbm_solver* s, T** p, size_t bytes) {
  void* q = nullptr;
  const vplbm_status st = mem_get(s, &q, bytes);
  *p = static_cast<T*>(q);
  return st;
}

// Releases a solver buffer. The caller's allocator may hand the block out
// again at once, so the work already queued on the stream finishes first.
void mem_put(vplbm_solver* s, void* p) {
  if (!p) return;
  if (!s->cfg.dev_free) {
    cudaFreeAsync(p, s->stream);
    return;
  }
  cudaStreamSynchronize(s->stream);
  s->cfg.dev_free(p, s->cfg.alloc_ctx);
}

// A staging buffer of one call, released when the call returns on any path.
template <class T>
struct Staging {
  vplbm_solver* s;
  T* p = nullptr;
  explicit Staging(vplbm_solver* solver) : s(solver) {}
  Staging(const Staging&) = delete;
  Staging& operator=(const Staging&) = delete;
  ~Staging() { mem_put(s, p); }
  vplbm_status get(size_t n) { return mem_get(s, &p, n * sizeof(T)); }
};

void body_state(const vplbm_body& b, int64_t t, BodyState* st) {
  // centre(t) = c + amp sin(2 pi t / period), velocity = its time derivative
  if (b.period > 0.0) {
    const double ph = 2.0 * kPi * (double)t / b.period;
    const double sn = std::sin(ph), co = std::cos(ph);
    const double rate = 2.0 * kPi / b.period;
    st->cx = b.cx + b.amp_x * sn;
    st->cy = b.cy + b.amp_y * sn;
    st->vx = b.amp_x * rate * co;
    st->vy = b.amp_y * rate * co;
  } else {
    st->cx = b.cx;
    st->cy = b.cy;
    st->vx = 0.0;
    st->vy = 0.0;
  }
  st->omega = b.omega;
}

struct Box {
  int x0, y0, x1, y1;  // inclusive
  bool empty() const { return x1 < x0 || y1 < y0; }
};

Box body_box(const vplbm_solver* s, const vplbm_body& b, int64_t t) {
  if (b.outside) return Box{0, 0, s->cfg.nx - 1, s->cfg.ny - 1};
  BodyState st;
  body_state(b, t, &st);
  Box r;
  r.x0 = std::max(0, int(std::floor(st.cx - b.radius)) - 1);
  r.x1 = std::min(s->cfg.nx - 1, int(std::ceil(st.cx + b.radius)) + 1);
  r.y0 = std::max(0, int(std::floor(st.cy - b.radius)) - 1);
  r.y1 = std::min(s->cfg.ny - 1, int(std::ceil(st.cy + b.radius)) + 1);
  return r;
}

Box unite(Box a, Box b) {
  if (a.empty()) return b;
  if (b.empty()) return a;
  return Box{std::min(a.x0, b.x0), std::min(a.y0, b.y0), std::max(a.x1, b.x1), std::max(a.y1, b.y1)};
}

vplbm_status launch_mask_update(vplbm_solver* s, Box box, int64_t t) {
  if (box.empty()) return VPLBM_OK;
  BodyGeomSet g{};
  g.n = int(s->bodies.size());
  for (int b = 0; b < g.n; ++b) {
    BodyState st;
    body_state(s->bodies[b], t, &st);
    g.b[b].cx = st.cx;
    g.b[b].cy = st.cy;
    g.b[b].r2 = s->bodies[b].radius * s->bodies[b].radius;
    g.b[b].outside = s->bodies[b].outside;
  }
  const dim3 blk(64, 4);
  const int w = box.x1 - box.x0 + 1, h = box.y1 - box.y0 + 1;
  mask_update_kernel<<<grid2d(w, h, blk), blk, 0, s->stream>>>(s->mask, s->pitch, box.x0, box.y0, w,
                                                               h, g);
  VP_CUDA(s, cudaGetLastError());
  s->launches++;
  return VPLBM_OK;
}

// Brings the mask of the moving bodies to time t (only the swept region).
vplbm_status ensure_mask(vplbm_solver* s, int64_t t) {
  if (!s->moving || s->mask_t == t) return VPLBM_OK;
  Box box{0, 0, -1, -1};
  for (const auto& b : s->bodies) {
    if (b.period <= 0.0) continue;
    box = unite(box, body_box(s, b, t));
    if (s->mask_t >= 0) box = unite(box, body_box(s, b, s->mask_t));
  }
  if (s->mask_t < 0) box = Box{0, 0, s->cfg.nx - 1, s->cfg.ny - 1};
  vplbm_status st = launch_mask_update(s, box, t);
  if (st != VPLBM_OK) return st;
  s->mask_t = t;
  return VPLBM_OK;
}

// Resets the static solid layer's box to empty and recomputes it from the
// mask as it stands (a superset is harmless: the reduction checks each node).
const int kEmptyBox[4] = {INT_MAX, INT_MAX, -1, -1};
vplbm_status update_static_box(vplbm_solver* s) {
  VP_CUDA(s, cudaMemcpyAsync(s->static_box, kEmptyBox, sizeof(kEmptyBox), cudaMemcpyHostToDevice,
                             s->stream));
  const dim3 blk(64, 4);
  solid_box_kernel<<<grid2d(s->cfg.nx, s->cfg.ny, blk), blk, 0, s->stream>>>(
      s->mask, s->pitch, s->cfg.nx, s->cfg.ny, s->static_box);
  VP_CUDA(s, cudaGetLastError());
  return VPLBM_OK;
}

vplbm_status ensure_me_buffers(vplbm_solver* s) {
  if (s->me_scratch) return VPLBM_OK;
  const size_t L = size_t(s->cfg.force_ring_len);
  if (!s->me_ring) VP_OK(mem_get(s, &s->me_ring, 2 * sizeof(double) * L));
  if (!s->me_counter) VP_OK(mem_get(s, &s->me_counter, sizeof(unsigned)));
  VP_OK(mem_get(s, &s->me_scratch, 2 * sizeof(double) * (kMeBlocks + 1)));
  VP_CUDA(s, cudaMemsetAsync(s->me_ring, 0, 2 * sizeof(double) * L, s->stream));
  VP_CUDA(s, cudaMemsetAsync(s->me_counter, 0, sizeof(unsigned), s->stream));
  return VPLBM_OK;
}

void fill_bodies(const vplbm_solver* s, int64_t t, StepParams* p) {
  p->n_bodies = int(s->bodies.size());
  for (int b = 0; b < p->n_bodies; ++b) {
    BodyState st;
    body_state(s->bodies[b], t, &st);
    const double v[5] = {st.cx, st.cy, st.vx, st.vy, st.omega};
    for (int k = 0; k < 5; ++k) {
      p->cd.body[b][k] = v[k];
      p->cf.body[b][k] = float(v[k]);
    }
  }
}

// Equilibrium offset f_eq(rho, u) - w in FP64 (host; inlet ghost column).
void heq_host(double rho, double ux, double uy, double out[9]) {
  static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  static const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  const double uu = ux * ux + uy * uy;
  for (int a = 0; a < 9; ++a) {
    const double xu = ex[a] * ux + ey[a] * uy;
    out[a] = w[a] * ((rho - 1.0) + rho * (3.0 * xu + 4.5 * xu * xu - 1.5 * uu));
  }
}

// Pair differences of a store's reference (zero without one), from the
// reference as the kernels hold it (odd in xi, so its pair sums are zero).
template <class T>
void ref_sums(Consts<T>& c) {
  static const int pa[4] = {1, 2, 5, 6}, pb[4] = {3, 4, 7, 8};
  for (int k = 0; k < 4; ++k) c.r_d[k] = T(double(c.h_ref[pa[k]]) - double(c.h_ref[pb[k]]));
}

// Float copies of the FP64 constants.
void round_consts(StepParams* p) {
  Consts<double>& d = p->cd;
  Consts<float>& f = p->cf;
  f.s_e = float(d.s_e);
  f.s_eps = float(d.s_eps);
  f.s_qx = float(d.s_qx);
  f.s_qy = float(d.s_qy);
  f.s_pxx = float(d.s_pxx);
  f.s_pxy = float(d.s_pxy);
  f.a_s = float(d.a_s);
  f.kappa_s = float(d.kappa_s);
  f.gx = float(d.gx);
  f.gy = float(d.gy);
  for (int a = 0; a < 9; ++a) f.heq_in[a] = float(d.heq_in[a]);
  for (int a = 0; a < 9; ++a) f.h_ref[a] = float(d.h_ref[a]);
  f.u_conv = float(d.u_conv);
  f.conv_inv = float(d.conv_inv);
  f.t_hsp = float(d.t_hsp);
  f.t_hsm = float(d.t_hsm);
  f.t_1msp = float(d.t_1msp);
  f.t_sp = float(d.t_sp);
  f.t_c3p = float(d.t_c3p);
  for (int k = 0; k < 2; ++k) {
    f.t_a[k] = float(d.t_a[k]);
    f.t_b[k] = float(d.t_b[k]);
    f.t_am[k] = float(d.t_am[k]);
    f.t_bm[k] = float(d.t_bm[k]);
  }
  ref_sums(f);
}

// Collision and forcing constants of a configuration (FP64, then their float
// copies), and the collision kernel that applies them: the two-rate form for
// SRT and for MRT whose even moments share one rate and whose two heat-flux
// moments share another (the printed S), the full moment-space form for any
// other rates.
void physics_consts(const vplbm_config* cfg, StepParams* p) {
  Consts<double>& cd = p->cd;
  if (cfg->use_rates) {
    cd.s_e = cfg->rates[1];
    cd.s_eps = cfg->rates[2];
    cd.s_qx = cfg->rates[4];
    cd.s_qy = cfg->rates[6];
    cd.s_pxx = cfg->rates[7];
    cd.s_pxy = cfg->rates[8];
  } else {
    // S = diag(0, s_n, s_n, 0, s_q, 0, s_q, s_n, s_n), s_n = 1/tau,
    // Lambda = (1/s_n - 1/2)(1/s_q - 1/2)
    const double sn = 1.0 / cfg->tau;
    const double sq = 1.0 / (0.5 + cfg->lambda / (1.0 / sn - 0.5));
    cd.s_e = cd.s_eps = cd.s_pxx = cd.s_pxy = sn;
    cd.s_qx = cd.s_qy = sq;
  }
  double sp, sm;  // rates of the even and odd moments in the two-rate form
  if (cfg->collision == VPLBM_SRT) {
    sp = sm = 1.0 / cfg->tau;
    p->collision = kTrt;
  } else {
    sp = cd.s_e;
    sm = cd.s_qx;
    const bool two_rate = cd.s_eps == sp && cd.s_pxx == sp && cd.s_pxy == sp && cd.s_qy == sm;
    p->collision = two_rate ? kTrt : kMrt;
  }
  const double cp = 1.0 - 0.5 * sp, cm = 1.0 - 0.5 * sm;
  cd.t_hsp = 0.5 * sp;
  cd.t_hsm = 0.5 * sm;
  cd.t_1msp = 1.0 - sp;
  cd.t_sp = sp;
  cd.t_c3p = 3.0 * cp;
  cd.t_a[0] = 4.5 * sp / 9.0;
  cd.t_a[1] = 4.5 * sp / 36.0;
  cd.t_b[0] = 9.0 * cp / 9.0;
  cd.t_b[1] = 9.0 * cp / 36.0;
  cd.t_am[0] = 3.0 * sm / 9.0;
  cd.t_am[1] = 3.0 * sm / 36.0;
  cd.t_bm[0] = 3.0 * cm / 9.0;
  cd.t_bm[1] = 3.0 * cm / 36.0;
  cd.a_s = 0.5 / cfg->eta;
  cd.kappa_s = (1.0 / cfg->eta) / (1.0 + 0.5 / cfg->eta);
  cd.gx = cfg->body_force[0];
  cd.gy = cfg->body_force[1];
  p->force_free = cfg->body_force[0] == 0.0 && cfg->body_force[1] == 0.0 ? 1 : 0;
  p->round_key = 0x9e3779b9u ^ (cfg->rounding_seed * 0x85ebca6bu);
  heq_host(1.0, cfg->u_in[0], cfg->u_in[1], cd.heq_in);
  // 16-bit stores of a channel keep offsets from a reference halfway towards
  // the inlet's equilibrium: r = w + (3/2) w xi_x u_in,x, half of the part of
  // f_eq(1, u_in) - w that is odd in xi and even in xi_y (its momentum term
  // along x). The populations of the stagnant wake and of the free stream
  // then both lie within about half the stream's offsets of r, which halves
  // the largest elements and their rounding steps (offsets from the inlet's
  // equilibrium itself would make the wake's elements the largest). Being odd
  // in xi, r adds nothing to the density or to the pair sums of opposite
  // populations; being even in xi_y, a population and its mirror image at a
  // free-slip wall share it. Other flows and storages keep offsets from w.
  static const double ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  const bool sixteen = cfg->storage == VPLBM_F16_OFFSET || cfg->storage == VPLBM_BF16_OFFSET;
  const bool inlet = cfg->bc_x == VPLBM_BC_INLET_OUTLET || cfg->bc_x == VPLBM_BC_INLET_CONVECTIVE;
  for (int a = 0; a < 9; ++a) cd.h_ref[a] = sixteen && inlet ? 1.5 * w[a] * ex[a] * cfg->u_in[0] : 0.0;
  // The reference is rounded to multiples of 2^-28 (of 2^-21 of its largest
  // magnitude, for references above 2^-7), so that it, its pair differences,
  // and element + reference for every FP16 element (a multiple
  // of 2^-24) whose sum stays below 2^-4 are exact in FP32: the kernels decode
  // stored elements without rounding, and no rounding error of a constant
  // repeats at every node and step (stochastic rounding carries such a
  // repeated error forward, like a small body force, instead of absorbing it).
  double rmax = 0.0;
  for (int a = 0; a < 9; ++a) rmax = std::max(rmax, std::fabs(cd.h_ref[a]));
  if (rmax > 0.0) {
    int e2;
    std::frexp(rmax, &e2);  // rmax < 2^e2
    const double grid = std::ldexp(1.0, std::max(-28, e2 - 21));
    for (int a = 0; a < 9; ++a) cd.h_ref[a] = std::nearbyint(cd.h_ref[a] / grid) * grid;
  }
  ref_sums(cd);
  cd.u_conv = cfg->u_conv;
  cd.conv_inv = 1.0 / (1.0 + cfg->u_conv);
  round_consts(p);
}

StepParams step_params(const vplbm_solver* s, int64_t t, int parity) {
  StepParams p = s->base;
  const int c = s->cur ^ parity;
  p.src = s->f[c];
  p.dst = s->f[c ^ 1];
  p.ghost_src = s->ghost[c];
  p.ghost_dst = s->ghost[c ^ 1];
  p.mode = s->aa ? (c == 0 ? kModeAAPush : kModeAALocal) : kModeAB;
  p.t = t;
  fill_bodies(s, t, &p);
  return p;
}

cudaError_t launch_fused(const vplbm_solver* s, const StepParams& p) {
  const int coll = p.collision;
  switch (s->cfg.storage) {
    case kF64: return launch_fused_f64(coll, p, s->stream);
    case kF32: return launch_fused_f32(coll, p, s->stream);
    case kF16: return launch_fused_f16(coll, p, s->stream);
    default: return launch_fused_bf16(coll, p, s->stream);
  }
}

cudaError_t launch_group(int storage, const StepParams* dp, const GroupTile* dt, int nb, long long k,
                         int mode, cudaStream_t st) {
  switch (storage) {
    case kF64: return launch_group_f64(dp, dt, nb, k, mode, st);
    case kF32: return launch_group_f32(dp, dt, nb, k, mode, st);
    case kF16: return launch_group_f16(dp, dt, nb, k, mode, st);
    default: return launch_group_bf16(dp, dt, nb, k, mode, st);
  }
}

// Momentum exchange at step index t from the store f*(t) (p.src) into out:
// the candidate box is the bodies' boxes at t, united on the device with the
// static layer's box.
cudaError_t launch_momentum_exchange(const vplbm_solver* s, const StepParams& p, double* out) {
  Box box{0, 0, -1, -1};
  for (const auto& b : s->bodies) box = unite(box, body_box(s, b, p.t));
  MeArgs m{box.x0, box.y0, box.x1, box.y1, s->static_box, s->me_scratch, s->me_counter, out};
  switch (s->cfg.storage) {
    case kF64: return launch_momentum_exchange_f64(p, m, s->stream);
    case kF32: return launch_momentum_exchange_f32(p, m, s->stream);
    case kF16: return launch_momentum_exchange_f16(p, m, s->stream);
    default: return launch_momentum_exchange_bf16(p, m, s->stream);
  }
}

cudaError_t launch_moments(const vplbm_solver* s, const StepParams& p, double* r, double* ux, double* uy) {
  switch (s->cfg.storage) {
    case kF64: return launch_moments_f64(p, r, ux, uy, s->stream);
    case kF32: return launch_moments_f32(p, r, ux, uy, s->stream);
    case kF16: return launch_moments_f16(p, r, ux, uy, s->stream);
    default: return launch_moments_bf16(p, r, ux, uy, s->stream);
  }
}

cudaError_t launch_init(const vplbm_solver* s, const StepParams& p, void* dst, const double* u) {
  const double r0 = s->cfg.rho0, ux = s->cfg.u0[0], uy = s->cfg.u0[1];
  switch (s->cfg.storage) {
    case kF64: return launch_init_f64(p, dst, u, r0, ux, uy, s->stream);
    case kF32: return launch_init_f32(p, dst, u, r0, ux, uy, s->stream);
    case kF16: return launch_init_f16(p, dst, u, r0, ux, uy, s->stream);
    default: return launch_init_bf16(p, dst, u, r0, ux, uy, s->stream);
  }
}

cudaError_t launch_ghost_init(const vplbm_solver* s, const StepParams& p, const void* src, void* g,
                              void* z) {
  switch (s->cfg.storage) {
    case kF64: return launch_ghost_init_f64(p, src, g, z, s->stream);
    case kF32: return launch_ghost_init_f32(p, src, g, z, s->stream);
    case kF16: return launch_ghost_init_f16(p, src, g, z, s->stream);
    default: return launch_ghost_init_bf16(p, src, g, z, s->stream);
  }
}

// Outlet state once the populations were set (cur: the new store's buffer,
// or phase in place): the convective state and, in place, the side copy of
// the last column start as copies of the store's last column.
vplbm_status init_outlet_state(vplbm_solver* s) {
  if (!s->ghost[0] && !s->z) return VPLBM_OK;
  VP_CUDA(s, launch_ghost_init(s, step_params(s, s->t, 0), s->f[s->cur], s->ghost[s->cur], s->z));
  return VPLBM_OK;
}

cudaError_t launch_export(const vplbm_solver* s, const StepParams& p, const void* src, double* f) {
  switch (s->cfg.storage) {
    case kF64: return launch_export_f64(p, src, f, s->stream);
    case kF32: return launch_export_f32(p, src, f, s->stream);
    case kF16: return launch_export_f16(p, src, f, s->stream);
    default: return launch_export_bf16(p, src, f, s->stream);
  }
}

cudaError_t launch_import(const vplbm_solver* s, const StepParams& p, void* dst, const double* f) {
  switch (s->cfg.storage) {
    case kF64: return launch_import_f64(p, dst, f, s->stream);
    case kF32: return launch_import_f32(p, dst, f, s->stream);
    case kF16: return launch_import_f16(p, dst, f, s->stream);
    default: return launch_import_bf16(p, dst, f, s->stream);
  }
}

vplbm_status validate(const vplbm_config* c, std::string* why) {
  if (!c) return *why = "config is NULL", VPLBM_ERR_INVALID;
  if (c->nx < 1 || c->ny < 1) return *why = "nx and ny must be >= 1", VPLBM_ERR_INVALID;
  if ((long long)c->nx * c->ny > (1ll << 34)) return *why = "grid too large", VPLBM_ERR_INVALID;
  if (c->collision != VPLBM_SRT && c->collision != VPLBM_MRT)
    return *why = "unknown collision", VPLBM_ERR_INVALID;
  if (c->storage < VPLBM_F64 || c->storage > VPLBM_BF16_OFFSET)
    return *why = "unknown storage", VPLBM_ERR_INVALID;
  if (c->bc_x != VPLBM_BC_PERIODIC && c->bc_x != VPLBM_BC_INLET_OUTLET &&
      c->bc_x != VPLBM_BC_INLET_CONVECTIVE)
    return *why = "bc_x must be PERIODIC, INLET_OUTLET or INLET_CONVECTIVE", VPLBM_ERR_INVALID;
  if (c->bc_x == VPLBM_BC_INLET_CONVECTIVE && !(c->u_conv >= 0.0 && std::isfinite(c->u_conv)))
    return *why = "u_conv must be finite and >= 0", VPLBM_ERR_INVALID;
  if (c->streaming != VPLBM_STREAM_AB && c->streaming != VPLBM_STREAM_AA)
    return *why = "streaming must be AB or AA", VPLBM_ERR_INVALID;
  if (c->bc_y != VPLBM_BC_PERIODIC && c->bc_y != VPLBM_BC_FREE_SLIP)
    return *why = "bc_y must be PERIODIC or FREE_SLIP", VPLBM_ERR_INVALID;
  if (!(c->tau > 0.5) || !std::isfinite(c->tau)) return *why = "tau must be > 1/2", VPLBM_ERR_INVALID;
  if (!(c->eta > 0.0)) return *why = "eta must be > 0", VPLBM_ERR_INVALID;
  if (c->collision == VPLBM_MRT && !c->use_rates && !(c->lambda > 0.0))
    return *why = "lambda must be > 0", VPLBM_ERR_INVALID;
  if (!(c->rho0 > 0.0)) return *why = "rho0 must be > 0", VPLBM_ERR_INVALID;
  if (c->force_ring_len < 1) return *why = "force_ring_len must be >= 1", VPLBM_ERR_INVALID;
  if (c->rounding != VPLBM_ROUND_NEAREST && c->rounding != VPLBM_ROUND_STOCHASTIC)
    return *why = "unknown rounding", VPLBM_ERR_INVALID;
  if (!c->dev_alloc != !c->dev_free)
    return *why = "dev_alloc and dev_free must both be set or both be NULL", VPLBM_ERR_INVALID;
  if (c->tile_rows != 0 && c->tile_rows != 8 && c->tile_rows != 16 && c->tile_rows != 32)
    return *why = "tile_rows must be 0 (automatic), 8, 16 or 32", VPLBM_ERR_INVALID;
  return VPLBM_OK;
}

// Tile height of a configuration: the requested one, or (tile_rows = 0) the
// tallest of 32, 16 and 8 rows that still gives four waves of blocks on the
// GPU's 152 SMs (fewer, shorter waves leave SMs idle in the last one, which
// small grids cannot hide). A fixed rule, so a configuration has one tile
// decomposition (and one reduction order) on any device.
constexpr long long kSmCount = 152;
int tile_rows_of(const vplbm_config* c) {
  if (c->tile_rows) return c->tile_rows;
  const long long tx = (c->nx + tile_x(c->storage) - 1) / tile_x(c->storage);
  const long long want = 4 * kSmCount * min_blocks_per_sm(c->storage);
  int rows = kTileRowsMax;
  while (rows > kTileRowsMin && tx * ((c->ny + rows - 1) / rows) < want) rows /= 2;
  return rows;
}

void tiles_of(const vplbm_config* c, int* tx, int* ty, int* nt, int* ng) {
  const int tw = tile_x(c->storage);
  const int rows = tile_rows_of(c);
  *tx = (c->nx + tw - 1) / tw;
  *ty = (c->ny + rows - 1) / rows;
  *nt = *tx * *ty;
  *ng = (*nt + kGroup - 1) / kGroup;
}

vplbm_status check_usable(vplbm_solver* s) {
  if (!s) return VPLBM_ERR_INVALID;
  if (s->sticky) return VPLBM_ERR_CUDA;
  return VPLBM_OK;
}

vplbm_status drain_timing(vplbm_solver* s) {
  for (auto& pr : s->ev_pending) {
    float ms = 0.f;
    VP_CUDA(s, cudaEventSynchronize(pr.second));
    VP_CUDA(s, cudaEventElapsedTime(&ms, pr.first, pr.second));
    s->timed_ms += ms;
    s->timed_count++;
    s->ev_pool.push_back(pr.first);
    s->ev_pool.push_back(pr.second);
  }
  s->ev_pending.clear();
  return VPLBM_OK;
}

vplbm_status get_event(vplbm_solver* s, cudaEvent_t* e) {
  if (!s->ev_pool.empty()) {
    *e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return VPLBM_OK;
  }
  VP_CUDA(s, cudaEventCreate(e));
  return VPLBM_OK;
}

}  // namespace

extern "C" {

void vplbm_config_init(vplbm_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->collision = VPLBM_SRT;
  c->storage = VPLBM_F32;
  c->bc_x = VPLBM_BC_PERIODIC;
  c->bc_y = VPLBM_BC_PERIODIC;
  c->reduce_mass = 1;
  c->tau = 0.8;
  c->lambda = 3.0 / 16.0;
  c->eta = 1e-7;
  c->rho0 = 1.0;
  c->force_ring_len = 4096;
  c->rounding = VPLBM_ROUND_STOCHASTIC;
  c->u_conv = 0.0;
}

double vplbm_tau_from_reynolds(double u_ref, double l_ref, double re) {
  const double nu = u_ref * l_ref / re;  // kinematic viscosity
  return 3.0 * nu + 0.5;                 // nu = c_s^2 (tau - 1/2), c_s^2 = 1/3
}

size_t vplbm_footprint_bytes(const vplbm_config* c) {
  std::string why;
  if (validate(c, &why) != VPLBM_OK) return 0;
  int tx, ty, nt, ng;
  tiles_of(c, &tx, &ty, &nt, &ng);
  const size_t pitch = size_t(row_pitch(c->nx, c->storage));
  const size_t plane = pitch * size_t(c->ny);
  const bool aa = c->streaming == VPLBM_STREAM_AA;
  size_t b = (aa ? 1 : 2) * 9 * plane * element_size(c->storage);  // A/B or in-place populations
  if (aa && c->bc_x != VPLBM_BC_PERIODIC) b += 9 * size_t(c->ny) * element_size(c->storage);
  b += plane;                                            // mask
  b += 3 * sizeof(double) * (size_t(nt) + size_t(ng));   // reduction partials
  b += sizeof(unsigned) * (size_t(ng) + 1);
  b += 3 * sizeof(double) * size_t(c->force_ring_len);
  b += sizeof(int) + sizeof(kEmptyBox);                  // error flag, static solid box
  if (c->bc_x == VPLBM_BC_INLET_CONVECTIVE) b += 2 * 3 * size_t(c->ny) * ghost_elem(c->storage);
  return b;
}

vplbm_status vplbm_create(const vplbm_config* cfg, vplbm_solver** out) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return VPLBM_ERR_INVALID;
  }
  *out = nullptr;
  std::string why;
  vplbm_status v = validate(cfg, &why);
  if (v != VPLBM_OK) {
    std::fprintf(stderr, "vplbm_create: %s\n", why.c_str());
    g_create_error = why;
    return v;
  }
  vplbm_solver* s = new (std::nothrow) vplbm_solver();
  if (!s) {
    g_create_error = "host allocation of the solver failed";
    return VPLBM_ERR_NOMEM;
  }
  s->cfg = *cfg;
  s->esize = element_size(cfg->storage);
  s->pitch = row_pitch(cfg->nx, cfg->storage);
  s->plane = (long long)s->pitch * cfg->ny;
  tiles_of(cfg, &s->tiles_x, &s->tiles_y, &s->n_tiles, &s->n_groups);

  auto bail = [&](vplbm_status st) {
    std::fprintf(stderr, "vplbm_create: %s\n", s->err.c_str());
    g_create_error = s->err;
    vplbm_destroy(s);
    return st;
  };
  vplbm_status st = VPLBM_OK;
  if (cfg->stream) {
    s->stream = static_cast<cudaStream_t>(cfg->stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(s, e, "cudaStreamCreate"));
    s->own_stream = true;
  }
  const size_t pop = size_t(9) * size_t(s->plane) * s->esize;
  cudaError_t e = cudaSuccess;
  cudaStream_t st0 = s->stream;
  s->aa = cfg->streaming == VPLBM_STREAM_AA;
  if ((st = mem_get(s, &s->f[0], pop)) != VPLBM_OK ||
      (!s->aa && (st = mem_get(s, &s->f[1], pop)) != VPLBM_OK) ||
      (st = mem_get(s, &s->mask, size_t(s->plane))) != VPLBM_OK ||
      (st = mem_get(s, &s->partials, 3 * sizeof(double) * s->n_tiles)) != VPLBM_OK ||
      (st = mem_get(s, &s->group_partials, 3 * sizeof(double) * s->n_groups)) != VPLBM_OK ||
      (st = mem_get(s, &s->counters, sizeof(unsigned) * (s->n_groups + 1))) != VPLBM_OK ||
      (st = mem_get(s, &s->ring, 3 * sizeof(double) * cfg->force_ring_len)) != VPLBM_OK ||
      (st = mem_get(s, &s->flag, sizeof(int))) != VPLBM_OK ||
      (st = mem_get(s, &s->static_box, sizeof(kEmptyBox))) != VPLBM_OK) {
    return bail(st);
  }
  if ((e = cudaMemsetAsync(s->mask, 0, size_t(s->plane), s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->counters, 0, sizeof(unsigned) * (s->n_groups + 1), s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->ring, 0, 3 * sizeof(double) * cfg->force_ring_len, s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(s->static_box, kEmptyBox, sizeof(kEmptyBox), cudaMemcpyHostToDevice,
                           s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->f[0], 0, pop, s->stream)) != cudaSuccess ||
      (!s->aa && (e = cudaMemsetAsync(s->f[1], 0, pop, s->stream)) != cudaSuccess)) {
    return bail(cuda_fail(s, e, "cudaMemsetAsync"));
  }
  if (s->aa) {
    s->f[1] = s->f[0];
    if (cfg->bc_x != VPLBM_BC_PERIODIC) {
      if ((st = mem_get(s, &s->z, 3 * size_t(cfg->ny) * s->esize)) != VPLBM_OK ||
          (st = mem_get(s, &s->lost, 6 * size_t(cfg->ny) * s->esize)) != VPLBM_OK)
        return bail(st);
      if ((e = cudaMemsetAsync(s->lost, 0, 6 * size_t(cfg->ny) * s->esize, st0)) != cudaSuccess)
        return bail(cuda_fail(s, e, "cudaMemsetAsync"));
    }
  }
  if (cfg->bc_x == VPLBM_BC_INLET_CONVECTIVE) {
    const size_t gb = 3 * size_t(cfg->ny) * ghost_elem(cfg->storage);
    if ((st = mem_get(s, &s->ghost[0], gb)) != VPLBM_OK ||
        (st = mem_get(s, &s->ghost[1], gb)) != VPLBM_OK)
      return bail(st);
  }

  StepParams& p = s->base;
  std::memset(&p, 0, sizeof(p));
  p.mask = s->mask;
  p.us = nullptr;
  p.nx = cfg->nx;
  p.ny = cfg->ny;
  p.pitch = s->pitch;
  p.plane = s->plane;
  p.bc_x = cfg->bc_x;
  p.bc_y = cfg->bc_y;
  p.tiles_x = s->tiles_x;
  p.n_tiles = s->n_tiles;
  p.tile_y = tile_rows_of(cfg);
  p.rows_per_warp = p.tile_y / warps_per_block(cfg->storage);
  p.mode = s->aa ? kModeAAPush : kModeAB;
  p.z = s->z;
  p.lost = s->lost;
  physics_consts(cfg, &p);
  p.partials = s->partials;
  p.group_partials = s->group_partials;
  p.counters = s->counters;
  p.ring = s->ring;
  p.flag = s->flag;
  p.ring_len = cfg->force_ring_len;
  p.reduce_mass = cfg->reduce_mass ? 1 : 0;
  p.stochastic = cfg->rounding == VPLBM_ROUND_STOCHASTIC ? 1 : 0;

  if ((st = vplbm_set_initial_velocity(s, nullptr)) != VPLBM_OK) return bail(st);
  *out = s;
  return VPLBM_OK;
}

vplbm_status vplbm_set_initial_velocity(vplbm_solver* s, const double* u) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  Staging<double> du(s);
  const size_t n = size_t(s->cfg.nx) * size_t(s->cfg.ny);
  if (u) {
    VP_OK(du.get(2 * n));
    VP_CUDA(s, cudaMemcpyAsync(du.p, u, 2 * n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  }
  s->cur = 0;
  VP_CUDA(s, launch_init(s, s->base, s->f[0], du.p));
  if ((st = init_outlet_state(s)) != VPLBM_OK) return st;
  s->t = 0;
  s->ring_read = 0;
  s->me_read = 0;
  s->me_stop = 0;
  VP_CUDA(s, cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream));
  VP_CUDA(s, cudaMemsetAsync(s->ring, 0, 3 * sizeof(double) * s->cfg.force_ring_len, s->stream));
  if (s->moving) s->mask_t = -1;
  return VPLBM_OK;
}

vplbm_status vplbm_set_mask_and_solid_velocity(vplbm_solver* s, const uint8_t* chi, const double* us,
                                               int32_t on_device) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!chi) return fail(s, VPLBM_ERR_INVALID, "chi is NULL");
  const int nx = s->cfg.nx, ny = s->cfg.ny;
  const size_t n = size_t(nx) * ny;
  const uint8_t* dchi = chi;
  const double* dus = us;
  Staging<uint8_t> tchi(s);
  Staging<double> tus(s);
  if (!on_device) {
    VP_OK(tchi.get(n));
    VP_CUDA(s, cudaMemcpyAsync(tchi.p, chi, n, cudaMemcpyHostToDevice, s->stream));
    dchi = tchi.p;
    if (us) {
      VP_OK(tus.get(2 * n));
      VP_CUDA(s, cudaMemcpyAsync(tus.p, us, 2 * n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      dus = tus.p;
    }
  }
  const dim3 blk(64, 4);
  mask_import_kernel<<<grid2d(nx, ny, blk), blk, 0, s->stream>>>(s->mask, s->pitch, nx, ny, dchi);
  VP_CUDA(s, cudaGetLastError());
  if ((st = update_static_box(s)) != VPLBM_OK) return st;
  if (dus) {
    const size_t vs = s->cfg.storage == kF64 ? sizeof(double2) : sizeof(float2);
    if (!s->us) VP_OK(mem_get(s, &s->us, vs * size_t(s->plane)));
    if (s->cfg.storage == kF64)
      us_import_kernel<double2><<<grid2d(nx, ny, blk), blk, 0, s->stream>>>(
          static_cast<double2*>(s->us), s->pitch, nx, ny, dus);
    else
      us_import_kernel<float2><<<grid2d(nx, ny, blk), blk, 0, s->stream>>>(
          static_cast<float2*>(s->us), s->pitch, nx, ny, dus);
    VP_CUDA(s, cudaGetLastError());
    s->base.us = s->us;
  } else {
    s->base.us = nullptr;
  }
  // Rebuild the bodies where the static layer changed.
  if (!s->bodies.empty()) {
    st = launch_mask_update(s, Box{0, 0, nx - 1, ny - 1}, s->t);
    if (st != VPLBM_OK) return st;
    s->mask_t = s->moving ? s->t : -1;
  }
  return VPLBM_OK;
}

vplbm_status vplbm_set_bodies(vplbm_solver* s, const vplbm_body* bodies, int32_t n) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (n < 0 || n > kMaxBodies || (n > 0 && !bodies))
    return fail(s, VPLBM_ERR_INVALID, "need 0 <= n <= VPLBM_MAX_BODIES bodies");
  for (int i = 0; i < n; ++i)
    if (!(bodies[i].radius >= 0.0) || !std::isfinite(bodies[i].cx) || !std::isfinite(bodies[i].cy))
      return fail(s, VPLBM_ERR_INVALID, "body radius must be >= 0 and centre finite");
  s->bodies.assign(bodies, bodies + n);
  s->moving = false;
  for (const auto& b : s->bodies)
    if (b.period > 0.0 && (b.amp_x != 0.0 || b.amp_y != 0.0)) s->moving = true;
  // Full rebuild at the current time (also clears removed bodies).
  st = launch_mask_update(s, Box{0, 0, s->cfg.nx - 1, s->cfg.ny - 1}, s->t);
  if (st != VPLBM_OK) return st;
  s->mask_t = s->moving ? s->t : -1;
  return VPLBM_OK;
}

vplbm_status vplbm_step(vplbm_solver* s, int64_t n) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (n < 0) return fail(s, VPLBM_ERR_INVALID, "n must be >= 0");
  TraceRange trace("vplbm_step");
  for (int64_t k = 0; k < n; ++k) {
    if ((st = ensure_mask(s, s->t)) != VPLBM_OK) return st;
    const StepParams p = step_params(s, s->t, 0);
    if (s->me_on) {
      VP_CUDA(s, launch_momentum_exchange(s, p, s->me_ring + 2 * (s->t % s->cfg.force_ring_len)));
      s->launches++;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s->timing) {
      if ((st = get_event(s, &e0)) != VPLBM_OK) return st;
      if ((st = get_event(s, &e1)) != VPLBM_OK) return st;
      VP_CUDA(s, cudaEventRecord(e0, s->stream));
    }
    VP_CUDA(s, launch_fused(s, p));
    if (s->timing) {
      VP_CUDA(s, cudaEventRecord(e1, s->stream));
      s->ev_pending.emplace_back(e0, e1);
    }
    s->launches++;
    s->cur ^= 1;
    s->t++;
  }
  return VPLBM_OK;
}

vplbm_status vplbm_synchronize(vplbm_solver* s) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  int flag = 0;
  VP_CUDA(s, cudaMemcpyAsync(&flag, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  if (flag) {
    VP_CUDA(s, cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream));
    return fail(s, VPLBM_ERR_DIVERGED, "a step produced rho <= 0 or a non-finite velocity");
  }
  return VPLBM_OK;
}

int64_t vplbm_step_count(const vplbm_solver* s) { return s ? s->t : -1; }

vplbm_status vplbm_moments(vplbm_solver* s, double* rho, double* ux, double* uy, int32_t on_device) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!rho || !ux || !uy) return fail(s, VPLBM_ERR_INVALID, "output pointer is NULL");
  if ((st = ensure_mask(s, s->t)) != VPLBM_OK) return st;
  const size_t n = size_t(s->cfg.nx) * s->cfg.ny;
  StepParams p = step_params(s, s->t, 0);
  if (on_device) {
    VP_CUDA(s, launch_moments(s, p, rho, ux, uy));
    return VPLBM_OK;
  }
  Staging<double> d(s);
  VP_OK(d.get(3 * n));
  VP_CUDA(s, launch_moments(s, p, d.p, d.p + n, d.p + 2 * n));
  VP_CUDA(s, cudaMemcpyAsync(rho, d.p, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaMemcpyAsync(ux, d.p + n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaMemcpyAsync(uy, d.p + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_populations(vplbm_solver* s, double* f, int32_t on_device) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!f) return fail(s, VPLBM_ERR_INVALID, "output pointer is NULL");
  const size_t n = size_t(s->cfg.nx) * s->cfg.ny;
  if (on_device) {
    VP_CUDA(s, launch_export(s, step_params(s, s->t, 0), s->f[s->cur], f));
    return VPLBM_OK;
  }
  Staging<double> d(s);
  VP_OK(d.get(9 * n));
  VP_CUDA(s, launch_export(s, step_params(s, s->t, 0), s->f[s->cur], d.p));
  VP_CUDA(s, cudaMemcpyAsync(f, d.p, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_set_populations(vplbm_solver* s, const double* f, int32_t on_device) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!f) return fail(s, VPLBM_ERR_INVALID, "input pointer is NULL");
  const size_t n = size_t(s->cfg.nx) * s->cfg.ny;
  if (s->aa) s->cur = 0;  // in place: the store restarts before a push step
  if (on_device) {
    VP_CUDA(s, launch_import(s, s->base, s->f[s->cur], f));
  } else {
    Staging<double> d(s);
    VP_OK(d.get(9 * n));
    VP_CUDA(s, cudaMemcpyAsync(d.p, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    VP_CUDA(s, launch_import(s, s->base, s->f[s->cur], d.p));
  }
  // the convective outlet restarts from a zero-gradient copy of the new store
  return init_outlet_state(s);
}

vplbm_status vplbm_mask(vplbm_solver* s, uint8_t* chi) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!chi) return fail(s, VPLBM_ERR_INVALID, "output pointer is NULL");
  if ((st = ensure_mask(s, s->t)) != VPLBM_OK) return st;
  const int nx = s->cfg.nx, ny = s->cfg.ny;
  const size_t n = size_t(nx) * ny;
  Staging<uint8_t> d(s);
  VP_OK(d.get(n));
  const dim3 blk(64, 4);
  mask_export_kernel<<<grid2d(nx, ny, blk), blk, 0, s->stream>>>(s->mask, s->pitch, nx, ny, d.p);
  VP_CUDA(s, cudaGetLastError());
  VP_CUDA(s, cudaMemcpyAsync(chi, d.p, n, cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_forces(vplbm_solver* s, double* fx, double* fy, double* mass, int64_t cap,
                          int64_t* count) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (count) *count = 0;
  if (cap < 0) return fail(s, VPLBM_ERR_INVALID, "cap must be >= 0");
  const int64_t L = s->cfg.force_ring_len;
  const int64_t k = std::min(std::min(s->t - s->ring_read, L), cap);
  std::vector<double> host(3 * size_t(std::max<int64_t>(k, 1)));
  // records of steps t-k .. t-1, at ring slots (step % L): at most two runs
  int64_t done = 0;
  while (done < k) {
    const int64_t step = s->t - k + done;
    const int64_t slot = step % L;
    const int64_t run = std::min(k - done, L - slot);
    VP_CUDA(s, cudaMemcpyAsync(host.data() + 3 * done, s->ring + 3 * slot, 3 * sizeof(double) * run,
                               cudaMemcpyDeviceToHost, s->stream));
    done += run;
  }
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  for (int64_t i = 0; i < k; ++i) {
    if (fx) fx[i] = host[3 * i + 0];
    if (fy) fy[i] = host[3 * i + 1];
    if (mass) mass[i] = host[3 * i + 2];
  }
  if (count) *count = k;
  s->ring_read = s->t;
  return VPLBM_OK;
}

namespace {
// Checkpoint layout: header, the post-collision store f*(t) as stored (raw
// elements, [9][ny][pitch]), the mask ([ny][pitch] bytes), and the static
// solid-velocity field when one is set.
struct StateHeader {
  uint64_t magic;
  int32_t nx, ny, pitch, storage, collision, has_us;
  int64_t t;
  uint64_t pop_bytes, mask_bytes, us_bytes;
  uint64_t ghost_bytes;  // convective outlet state, 0 for other outlets
  int32_t aa, phase;     // in-place streaming and its phase
  uint64_t side_bytes;   // in place, open x sides: the side copy z and the lost values
};
constexpr uint64_t kStateMagic = 0x56504c424d535433ull;  // "VPLBMST3"

size_t us_bytes(const vplbm_solver* s) {
  if (!s->us) return 0;
  return (s->cfg.storage == kF64 ? sizeof(double2) : sizeof(float2)) * size_t(s->plane);
}

size_t ghost_bytes(const vplbm_solver* s) {
  return s->ghost[0] ? 3 * size_t(s->cfg.ny) * ghost_elem(s->cfg.storage) : 0;
}

size_t side_bytes(const vplbm_solver* s) { return s->z ? 9 * size_t(s->cfg.ny) * s->esize : 0; }
}  // namespace

size_t vplbm_state_bytes(const vplbm_solver* s) {
  if (!s) return 0;
  return sizeof(StateHeader) + 9 * size_t(s->plane) * s->esize + size_t(s->plane) + us_bytes(s) +
         ghost_bytes(s) + side_bytes(s);
}

vplbm_status vplbm_save_state(vplbm_solver* s, void* buf, size_t bytes) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!buf) return fail(s, VPLBM_ERR_INVALID, "buffer is NULL");
  if (bytes < vplbm_state_bytes(s))
    return fail(s, VPLBM_ERR_INVALID, "buffer shorter than vplbm_state_bytes");
  if ((st = ensure_mask(s, s->t)) != VPLBM_OK) return st;
  StateHeader h{};
  h.magic = kStateMagic;
  h.nx = s->cfg.nx;
  h.ny = s->cfg.ny;
  h.pitch = s->pitch;
  h.storage = s->cfg.storage;
  h.collision = s->cfg.collision;
  h.has_us = s->us ? 1 : 0;
  h.t = s->t;
  h.pop_bytes = 9 * uint64_t(s->plane) * s->esize;
  h.mask_bytes = uint64_t(s->plane);
  h.us_bytes = us_bytes(s);
  h.ghost_bytes = ghost_bytes(s);
  h.aa = s->aa ? 1 : 0;
  h.phase = s->aa ? s->cur : 0;
  h.side_bytes = side_bytes(s);
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &h, sizeof(h));
  out += sizeof(h);
  VP_CUDA(s, cudaMemcpyAsync(out, s->f[s->cur], h.pop_bytes, cudaMemcpyDeviceToHost, s->stream));
  out += h.pop_bytes;
  VP_CUDA(s, cudaMemcpyAsync(out, s->mask, h.mask_bytes, cudaMemcpyDeviceToHost, s->stream));
  out += h.mask_bytes;
  if (h.us_bytes)
    VP_CUDA(s, cudaMemcpyAsync(out, s->us, h.us_bytes, cudaMemcpyDeviceToHost, s->stream));
  out += h.us_bytes;
  if (h.ghost_bytes)
    VP_CUDA(s, cudaMemcpyAsync(out, s->ghost[s->cur], h.ghost_bytes, cudaMemcpyDeviceToHost,
                               s->stream));
  out += h.ghost_bytes;
  if (h.side_bytes) {
    const size_t zb = 3 * size_t(s->cfg.ny) * s->esize;
    VP_CUDA(s, cudaMemcpyAsync(out, s->z, zb, cudaMemcpyDeviceToHost, s->stream));
    VP_CUDA(s, cudaMemcpyAsync(out + zb, s->lost, h.side_bytes - zb, cudaMemcpyDeviceToHost, s->stream));
  }
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_load_state(vplbm_solver* s, const void* buf, size_t bytes) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!buf) return fail(s, VPLBM_ERR_INVALID, "buffer is NULL");
  if (bytes < sizeof(StateHeader)) return fail(s, VPLBM_ERR_INVALID, "buffer shorter than a state");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  // every section the header announces must lie inside the buffer (each size
  // is checked against the buffer alone first, so the sum cannot wrap)
  const uint64_t avail = uint64_t(bytes) - sizeof(h);
  const uint64_t parts[5] = {h.pop_bytes, h.mask_bytes, h.has_us ? h.us_bytes : 0, h.ghost_bytes,
                             h.side_bytes};
  uint64_t total = 0;
  for (uint64_t b : parts) {
    if (b > avail || total + b > avail)
      return fail(s, VPLBM_ERR_INVALID, "buffer shorter than the state its header describes");
    total += b;
  }
  if (h.magic != kStateMagic || h.nx != s->cfg.nx || h.ny != s->cfg.ny || h.pitch != s->pitch ||
      h.storage != s->cfg.storage || h.pop_bytes != 9 * uint64_t(s->plane) * s->esize ||
      h.mask_bytes != uint64_t(s->plane) || h.t < 0 || h.ghost_bytes != ghost_bytes(s) ||
      h.aa != (s->aa ? 1 : 0) || h.side_bytes != side_bytes(s) || h.phase < 0 || h.phase > 1)
    return fail(s, VPLBM_ERR_INVALID, "state does not match this solver's grid and storage");
  const char* in = static_cast<const char*>(buf) + sizeof(h);
  VP_CUDA(s, cudaMemcpyAsync(s->f[s->cur], in, h.pop_bytes, cudaMemcpyHostToDevice, s->stream));
  in += h.pop_bytes;
  VP_CUDA(s, cudaMemcpyAsync(s->mask, in, h.mask_bytes, cudaMemcpyHostToDevice, s->stream));
  in += h.mask_bytes;
  if (h.has_us) {
    const size_t vs = s->cfg.storage == kF64 ? sizeof(double2) : sizeof(float2);
    if (h.us_bytes != vs * size_t(s->plane))
      return fail(s, VPLBM_ERR_INVALID, "state's solid-velocity field does not match");
    if (!s->us) VP_OK(mem_get(s, &s->us, h.us_bytes));
    VP_CUDA(s, cudaMemcpyAsync(s->us, in, h.us_bytes, cudaMemcpyHostToDevice, s->stream));
    s->base.us = s->us;
    in += h.us_bytes;
  }
  if (s->aa) s->cur = h.phase;  // before the state is placed: the ghost index is the phase
  if (h.ghost_bytes)
    VP_CUDA(s, cudaMemcpyAsync(s->ghost[s->cur], in, h.ghost_bytes, cudaMemcpyHostToDevice,
                               s->stream));
  in += h.ghost_bytes;
  if (h.side_bytes) {
    const size_t zb = 3 * size_t(s->cfg.ny) * s->esize;
    VP_CUDA(s, cudaMemcpyAsync(s->z, in, zb, cudaMemcpyHostToDevice, s->stream));
    VP_CUDA(s, cudaMemcpyAsync(s->lost, in + zb, h.side_bytes - zb, cudaMemcpyHostToDevice, s->stream));
  }
  // pageable host-to-device copies have been staged when they return
  s->t = h.t;
  s->ring_read = h.t;
  s->me_read = h.t;
  s->me_stop = h.t;
  s->mask_t = s->moving ? h.t : -1;
  if ((st = update_static_box(s)) != VPLBM_OK) return st;
  return VPLBM_OK;
}

vplbm_status vplbm_forces_async(vplbm_solver* s, double* records, int64_t cap, int64_t* count) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (count) *count = 0;
  if (cap < 0 || (cap > 0 && !records)) return fail(s, VPLBM_ERR_INVALID, "bad output buffer");
  const int64_t L = s->cfg.force_ring_len;
  const int64_t k = std::min(std::min(s->t - s->ring_read, L), cap);
  int64_t done = 0;
  while (done < k) {
    const int64_t step = s->t - k + done;
    const int64_t slot = step % L;
    const int64_t run = std::min(k - done, L - slot);
    VP_CUDA(s, cudaMemcpyAsync(records + 3 * done, s->ring + 3 * slot, 3 * sizeof(double) * run,
                               cudaMemcpyDeviceToHost, s->stream));
    done += run;
  }
  if (count) *count = k;
  s->ring_read = s->t;
  return VPLBM_OK;
}

vplbm_status vplbm_enable_momentum_exchange(vplbm_solver* s, int32_t enable) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (enable && !s->me_on) {
    if ((st = ensure_me_buffers(s)) != VPLBM_OK) return st;
    s->me_read = s->t;
  }
  if (!enable && s->me_on) s->me_stop = s->t;
  s->me_on = enable != 0;
  return VPLBM_OK;
}

vplbm_status vplbm_momentum_exchange(vplbm_solver* s, double* fx, double* fy) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if ((st = ensure_me_buffers(s)) != VPLBM_OK) return st;
  if ((st = ensure_mask(s, s->t)) != VPLBM_OK) return st;
  double* out = s->me_scratch + 2 * kMeBlocks;
  VP_CUDA(s, launch_momentum_exchange(s, step_params(s, s->t, 0), out));
  double host[2];
  VP_CUDA(s, cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, s->stream));
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  if (fx) *fx = host[0];
  if (fy) *fy = host[1];
  return VPLBM_OK;
}

vplbm_status vplbm_momentum_exchange_forces(vplbm_solver* s, double* fx, double* fy, int64_t cap,
                                            int64_t* count) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (count) *count = 0;
  if (cap < 0) return fail(s, VPLBM_ERR_INVALID, "cap must be >= 0");
  if (!s->me_ring) return fail(s, VPLBM_ERR_STATE, "momentum exchange was never enabled");
  const int64_t L = s->cfg.force_ring_len;
  const int64_t end = s->me_on ? s->t : std::max(s->me_stop, s->me_read);  // steps recorded
  const int64_t k = std::min(std::min(end - s->me_read, L), cap);
  std::vector<double> host(2 * size_t(std::max<int64_t>(k, 1)));
  int64_t done = 0;
  while (done < k) {
    const int64_t step = end - k + done;
    const int64_t slot = step % L;
    const int64_t run = std::min(k - done, L - slot);
    VP_CUDA(s, cudaMemcpyAsync(host.data() + 2 * done, s->me_ring + 2 * slot, 2 * sizeof(double) * run,
                               cudaMemcpyDeviceToHost, s->stream));
    done += run;
  }
  VP_CUDA(s, cudaStreamSynchronize(s->stream));
  for (int64_t i = 0; i < k; ++i) {
    if (fx) fx[i] = host[2 * i + 0];
    if (fy) fy[i] = host[2 * i + 1];
  }
  if (count) *count = k;
  s->me_read = end;
  return VPLBM_OK;
}

vplbm_status vplbm_set_initial_perturbation(vplbm_solver* s, double u0x, double u0y, double amp,
                                            uint64_t seed) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if (!(amp >= 0.0)) return fail(s, VPLBM_ERR_INVALID, "amp must be >= 0");
  const size_t n = size_t(s->cfg.nx) * s->cfg.ny;
  Staging<double> du(s);
  VP_OK(du.get(2 * n));
  const int threads = 256;
  const long long blocks = (long long)((n + threads - 1) / threads);
  perturbation_kernel<<<unsigned(blocks), threads, 0, s->stream>>>(du.p, s->cfg.nx, s->cfg.ny, u0x,
                                                                    u0y, amp, seed);
  VP_CUDA(s, cudaGetLastError());
  s->cur = 0;
  VP_CUDA(s, launch_init(s, s->base, s->f[0], du.p));
  if ((st = init_outlet_state(s)) != VPLBM_OK) return st;
  s->t = 0;
  s->ring_read = 0;
  s->me_read = 0;
  s->me_stop = 0;
  VP_CUDA(s, cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream));
  VP_CUDA(s, cudaMemsetAsync(s->ring, 0, 3 * sizeof(double) * s->cfg.force_ring_len, s->stream));
  if (s->moving) s->mask_t = -1;
  return VPLBM_OK;
}

vplbm_status vplbm_group_step(vplbm_solver* const* solvers, int32_t n, const int64_t* steps) {
  if (n < 0 || (n > 0 && (!solvers || !steps))) return VPLBM_ERR_INVALID;
  if (n == 0) return VPLBM_OK;
  if (!solvers[0]) return VPLBM_ERR_INVALID;
  cudaStream_t stream = solvers[0]->stream;
  int64_t max_steps = 0;
  for (int i = 0; i < n; ++i) {
    vplbm_solver* s = solvers[i];
    vplbm_status st = check_usable(s);
    if (st != VPLBM_OK) return st;
    if (s->stream != stream) return fail(s, VPLBM_ERR_INVALID, "group solvers must share a stream");
    if (steps[i] < 0) return fail(s, VPLBM_ERR_INVALID, "steps must be >= 0");
    for (int j = 0; j < i; ++j)
      if (solvers[j] == s) return fail(s, VPLBM_ERR_INVALID, "a solver appears twice in the group");
    max_steps = std::max(max_steps, steps[i]);
  }
  vplbm_solver* s0 = solvers[0];
  TraceRange trace("vplbm_group_step");
  // Solvers with moving bodies need a mask update between steps, and those
  // recording the momentum exchange a reduction before each step: step them
  // alone, interleaved with the grouped launches of the others.
  struct Member {
    int idx;
    int64_t steps;
  };
  // One grouped launch per step for each storage type and scheme class: A/B
  // (class 0), and in place by phase at the group's first step (classes 1, 2:
  // phase 0 or 1), whose launches alternate between push and local steps.
  std::vector<Member> classes[4][3];
  std::vector<int> moving;
  for (int i = 0; i < n; ++i) {
    if (solvers[i]->moving || solvers[i]->me_on) {
      moving.push_back(i);
      continue;
    }
    const vplbm_solver* s = solvers[i];
    classes[s->cfg.storage][s->aa ? 1 + s->cur : 0].push_back({i, steps[i]});
  }
  struct Plan {
    int storage = 0;
    int cls = 0;
    StepParams* d_params = nullptr;
    GroupTile* d_table = nullptr;
    std::vector<int64_t> prefix_steps;  // steps of the j-th member (descending)
    std::vector<int> prefix_tiles;      // tiles of members 0..j
  };
  // The launch tables live for this call only and go back to the memory pool
  // (stream-ordered, after the launches that read them) on every return path.
  struct Plans {
    std::vector<Plan> v;
    cudaStream_t stream;
    ~Plans() {
      for (auto& pl : v) {
        if (pl.d_params) cudaFreeAsync(pl.d_params, stream);
        if (pl.d_table) cudaFreeAsync(pl.d_table, stream);
      }
    }
  } owned{{}, stream};
  std::vector<Plan>& plans = owned.v;
  for (int sg = 0; sg < 4; ++sg) {
    for (int cls = 0; cls < 3; ++cls) {
      auto& mem = classes[sg][cls];
      if (mem.empty()) continue;
      std::stable_sort(mem.begin(), mem.end(),
                       [](const Member& a, const Member& b) { return a.steps > b.steps; });
      std::vector<StepParams> hp;
      std::vector<GroupTile> ht;
      plans.emplace_back();
      Plan& pl = plans.back();
      pl.storage = sg;
      pl.cls = cls;
      for (size_t j = 0; j < mem.size(); ++j) {
        vplbm_solver* s = solvers[mem[j].idx];
        hp.push_back(step_params(s, s->t, 0));
        hp.push_back(step_params(s, s->t, 1));
        for (int tile = 0; tile < s->n_tiles; ++tile) ht.push_back(GroupTile{int(j), tile});
        pl.prefix_steps.push_back(mem[j].steps);
        pl.prefix_tiles.push_back(int(ht.size()));
      }
      VP_CUDA(s0, cudaMallocAsync(reinterpret_cast<void**>(&pl.d_params), hp.size() * sizeof(StepParams), stream));
      VP_CUDA(s0, cudaMallocAsync(reinterpret_cast<void**>(&pl.d_table), ht.size() * sizeof(GroupTile), stream));
      VP_CUDA(s0, cudaMemcpyAsync(pl.d_params, hp.data(), hp.size() * sizeof(StepParams),
                                  cudaMemcpyHostToDevice, stream));
      VP_CUDA(s0, cudaMemcpyAsync(pl.d_table, ht.data(), ht.size() * sizeof(GroupTile),
                                  cudaMemcpyHostToDevice, stream));
    }
  }
  for (int64_t k = 0; k < max_steps; ++k) {
    for (auto& pl : plans) {
      // members are sorted by steps, so the ones still running are a prefix
      int active = 0;
      while (active < int(pl.prefix_steps.size()) && pl.prefix_steps[active] > k) ++active;
      if (active == 0) continue;
      const int nb = pl.prefix_tiles[active - 1];
      const int mode = pl.cls == 0 ? kModeAB
                                   : (((pl.cls - 1) ^ int(k & 1)) == 0 ? kModeAAPush : kModeAALocal);
      VP_CUDA(s0, launch_group(pl.storage, pl.d_params, pl.d_table, nb, k, mode, stream));
    }
    for (int i : moving) {
      if (steps[i] > k) {
        vplbm_status st = vplbm_step(solvers[i], 1);
        if (st != VPLBM_OK) return st;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    vplbm_solver* s = solvers[i];
    if (s->moving || s->me_on) continue;
    s->launches += steps[i];  // one grouped launch per step covers this solver
    s->cur ^= int(steps[i] & 1);
    s->t += steps[i];
  }
  return VPLBM_OK;
}

int64_t vplbm_launch_count(const vplbm_solver* s) { return s ? s->launches : -1; }

vplbm_status vplbm_enable_timing(vplbm_solver* s, int32_t enable) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  s->timing = enable != 0;
  return VPLBM_OK;
}

vplbm_status vplbm_fused_timing(vplbm_solver* s, double* total_ms, int64_t* launches) {
  vplbm_status st = check_usable(s);
  if (st != VPLBM_OK) return st;
  if ((st = drain_timing(s)) != VPLBM_OK) return st;
  if (total_ms) *total_ms = s->timed_ms;
  if (launches) *launches = s->timed_count;
  s->timed_ms = 0.0;
  s->timed_count = 0;
  return VPLBM_OK;
}

const char* vplbm_create_error(void) { return g_create_error.c_str(); }

const char* vplbm_last_error(const vplbm_solver* s) {
  if (!s) return "no solver";
  return s->err.c_str();
}

const char* vplbm_status_string(vplbm_status st) {
  switch (st) {
    case VPLBM_OK: return "ok";
    case VPLBM_ERR_INVALID: return "invalid argument";
    case VPLBM_ERR_NOMEM: return "out of device memory";
    case VPLBM_ERR_CUDA: return "CUDA error";
    case VPLBM_ERR_DIVERGED: return "diverged";
    case VPLBM_ERR_TIMEOUT: return "timeout";
    case VPLBM_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

void vplbm_destroy(vplbm_solver* s) {
  if (!s) return;
  // Stream-ordered release: the memory returns to the pool once the work
  // already queued on the stream is done; the host does not wait.
  for (auto& pr : s->ev_pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto e : s->ev_pool) cudaEventDestroy(e);
  if (s->stream) {
    void* bufs[] = {s->f[0], s->aa ? nullptr : s->f[1], s->mask, s->us, s->partials, s->group_partials,
                    s->counters, s->ring, s->flag, s->static_box, s->me_ring,
                    s->me_scratch, s->me_counter, s->ghost[0], s->ghost[1], s->z, s->lost};
    if (s->cfg.dev_free) cudaStreamSynchronize(s->stream);  // once, for all of them
    for (void* b : bufs) {
      if (!b) continue;
      if (s->cfg.dev_free)
        s->cfg.dev_free(b, s->cfg.alloc_ctx);
      else
        cudaFreeAsync(b, s->stream);
    }
    if (s->own_stream) cudaStreamDestroy(s->stream);
  }
  delete s;
}

}  // extern "C"

// ===========================================================================
// Allocation-free single step (vplbm_step_noalloc)
//
// For callers that cannot allocate device memory at the point where they
// step: code running inside a CUDA graph being built, a host callback, a
// real-time loop with a fixed memory budget, or a framework that owns every
// allocation itself. The reduction scratch of the fused step (per-tile and
// per-group partial sums and the arrival counters) lives in the fixed array
// below instead of per-solver cudaMalloc'd buffers. Every GPU that loads this
// library holds the array until the process exits.
// ===========================================================================

namespace {

// 1 MiB: 24 bytes per tile, 24 per group of 256 tiles, 4 per group counter
// (+1), 16-byte alignment and the 4-byte flag hold at most 43,491 tiles.
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;

// Shared by every call on a device; the last call's contents stay in it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Byte layout of the scratch for n_tiles tiles: partials, group partials,
// counters, divergence flag. Returns the bytes used.
size_t noalloc_layout(int n_tiles, size_t* off_group, size_t* off_counters, size_t* off_flag) {
  const int n_groups = (n_tiles + kGroup - 1) / kGroup;
  size_t off = 3 * sizeof(double) * size_t(n_tiles);
  *off_group = off;
  off += 3 * sizeof(double) * size_t(n_groups);
  *off_counters = off;
  off += sizeof(unsigned) * size_t(n_groups + 1);
  off = (off + 15) & ~size_t(15);
  *off_flag = off;
  off += sizeof(int);
  return off;
}

}  // namespace

extern "C" vplbm_status vplbm_step_noalloc(const vplbm_config* cfg, const vplbm_body* bodies,
                                           int32_t n_bodies, const void* f_src, void* f_dst,
                                           const uint8_t* mask, const void* us, int32_t pitch,
                                           int64_t t, double* record, int* flag) {
  std::string why;
  if (!cfg) {
    std::fprintf(stderr, "vplbm_step_noalloc: config is NULL\n");
    return VPLBM_ERR_INVALID;
  }
  {
    // rho0, u0 and force_ring_len belong to a solver's own state: not used here
    vplbm_config c = *cfg;
    c.rho0 = 1.0;
    c.force_ring_len = 1;
    if (validate(&c, &why) != VPLBM_OK) {
      std::fprintf(stderr, "vplbm_step_noalloc: %s\n", why.c_str());
      return VPLBM_ERR_INVALID;
    }
  }
  if (!f_src || !f_dst || !mask || !record || f_src == f_dst || t < 0 ||
      n_bodies < 0 || n_bodies > kMaxBodies || (n_bodies > 0 && !bodies)) {
    std::fprintf(stderr, "vplbm_step_noalloc: invalid pointer, step index or body count\n");
    return VPLBM_ERR_INVALID;
  }
  if (pitch < cfg->nx || pitch % 8 != 0) {
    std::fprintf(stderr, "vplbm_step_noalloc: pitch must be >= nx and a multiple of 8\n");
    return VPLBM_ERR_INVALID;
  }
  if (cfg->bc_x == VPLBM_BC_INLET_CONVECTIVE || cfg->streaming != VPLBM_STREAM_AB) {
    std::fprintf(stderr, "vplbm_step_noalloc: the convective outlet and in-place streaming keep "
                         "state between steps (use vplbm_create / vplbm_step)\n");
    return VPLBM_ERR_INVALID;
  }
  int tx, ty, nt, ng;
  tiles_of(cfg, &tx, &ty, &nt, &ng);
  size_t off_group, off_counters, off_flag;
  const size_t need = noalloc_layout(nt, &off_group, &off_counters, &off_flag);
  if (need > kNoAllocScratchBytes) {
    std::fprintf(stderr,
                 "vplbm_step_noalloc: grid of %d x %d needs %zu bytes of reduction scratch; the "
                 "fixed scratch holds %zu (use vplbm_create / vplbm_step for this size)\n",
                 cfg->nx, cfg->ny, need, kNoAllocScratchBytes);
    return VPLBM_ERR_INVALID;
  }

  // Set-up, once per device: the device address of the scratch array. The
  // array's name is only a host-side stand-in in this code.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    std::fprintf(stderr, "vplbm_step_noalloc: cudaGetDevice: %s\n", cudaGetErrorString(e));
    return VPLBM_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        std::fprintf(stderr, "vplbm_step_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
        return VPLBM_ERR_CUDA;
      }
      g_noalloc_addr[dev] = ptr;
    }
    base = g_noalloc_addr[dev];
  }
  unsigned char* sb = static_cast<unsigned char*>(base);
  cudaStream_t stream = static_cast<cudaStream_t>(cfg->stream);
  {
    // the scratch address is the current device's: the stream must be too
    int sdev = dev;
    if (stream && (e = cudaStreamGetDevice(stream, &sdev)) != cudaSuccess) {
      std::fprintf(stderr, "vplbm_step_noalloc: cudaStreamGetDevice: %s\n", cudaGetErrorString(e));
      return VPLBM_ERR_CUDA;
    }
    if (sdev != dev) {
      std::fprintf(stderr, "vplbm_step_noalloc: cfg->stream belongs to device %d, the current "
                           "device is %d\n", sdev, dev);
      return VPLBM_ERR_INVALID;
    }
  }

  // The arrival counters must start at zero (a failed earlier call could have
  // left them mid-count); the divergence slot too when the caller gives none.
  const size_t zero_bytes = off_flag + sizeof(int) - off_counters;
  if ((e = cudaMemsetAsync(sb + off_counters, 0, zero_bytes, stream)) != cudaSuccess) {
    std::fprintf(stderr, "vplbm_step_noalloc: cudaMemsetAsync: %s\n", cudaGetErrorString(e));
    return VPLBM_ERR_CUDA;
  }

  StepParams p;
  std::memset(&p, 0, sizeof(p));
  p.src = f_src;
  p.dst = f_dst;
  p.mask = mask;
  p.us = us;
  p.nx = cfg->nx;
  p.ny = cfg->ny;
  p.pitch = pitch;
  p.plane = (long long)pitch * cfg->ny;
  p.bc_x = cfg->bc_x;
  p.bc_y = cfg->bc_y;
  p.tiles_x = tx;
  p.n_tiles = nt;
  p.tile_y = tile_rows_of(cfg);
  p.rows_per_warp = p.tile_y / warps_per_block(cfg->storage);
  physics_consts(cfg, &p);
  p.n_bodies = n_bodies;
  for (int b = 0; b < n_bodies; ++b) {
    BodyState st;
    body_state(bodies[b], t, &st);
    const double v[5] = {st.cx, st.cy, st.vx, st.vy, st.omega};
    for (int k = 0; k < 5; ++k) {
      p.cd.body[b][k] = v[k];
      p.cf.body[b][k] = float(v[k]);
    }
  }
  p.partials = reinterpret_cast<double*>(sb);
  p.group_partials = reinterpret_cast<double*>(sb + off_group);
  p.counters = reinterpret_cast<unsigned*>(sb + off_counters);
  p.flag = flag ? flag : reinterpret_cast<int*>(sb + off_flag);
  p.ring = record;  // one record: ring of length 1
  p.ring_len = 1;
  p.reduce_mass = cfg->reduce_mass ? 1 : 0;
  p.stochastic = cfg->rounding == VPLBM_ROUND_STOCHASTIC ? 1 : 0;
  p.t = t;

  switch (cfg->storage) {
    case kF64: e = launch_fused_f64(p.collision, p, stream); break;
    case kF32: e = launch_fused_f32(p.collision, p, stream); break;
    case kF16: e = launch_fused_f16(p.collision, p, stream); break;
    default: e = launch_fused_bf16(p.collision, p, stream); break;
  }
  if (e != cudaSuccess) {
    std::fprintf(stderr, "vplbm_step_noalloc: launch: %s\n", cudaGetErrorString(e));
    return VPLBM_ERR_CUDA;
  }
  return VPLBM_OK;
}
