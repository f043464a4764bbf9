// Device side of the VP-LBM solver: storage traits, the fused
// stream-penalize-collide-reduce step, the mask update for moving bodies, and
// the initialisation / read-back kernels. Included by one translation unit per
// storage type (kernels_<storage>.cu).
//
// Arithmetic form. The kernel works on offsets h_alpha = f_alpha - w_alpha
// (w: the D2Q9 weights). Equilibrium, forcing and both collision operators are
// affine in f with the rest state w as a fixed point, so colliding h is the
// same operation, and it keeps the small deviations from the rest state out of
// the rounding of numbers near w. FP32 and the 16-bit storage forms store h
// itself; FP64 storage stores f.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "vplbm_params.h"

namespace vplbm {

// D2Q9 velocity set in the order of Eq. vecteurs_D2Q9.
__device__ __host__ constexpr int cx(int a) {
  return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__device__ __host__ constexpr int cy(int a) {
  return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
// Direction with the same x and opposite y velocity (free-slip reflection).
__device__ __host__ constexpr int mirror_y(int a) {
  return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}
// Direction with the opposite velocity.
__device__ __host__ constexpr int opposite(int a) {
  return a == 0 ? 0 : (a <= 4 ? (a + 1) % 4 + 1 : (a - 3) % 4 + 5);
}
// Weights, Eq. anex_eq19.
template <class T>
__device__ __forceinline__ constexpr T wgt(int a) {
  return a == 0 ? T(4.0 / 9.0) : (a <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}

// ---------------------------------------------------------------------------
// Storage traits: E is the element in HBM, T the arithmetic type, h = f - w
// the offset of a population. A 16-bit element holds h - ref, ref a
// per-direction reference (zero for the other stores, which hold h). The
// fused step works on the elements' values e = h - ref as they are (load_h,
// store_h, round_e, in_e: no reference), its collision taking ref through
// constant sums; in, out, to_f64 and from_f64 convert to and from h and f.
// ---------------------------------------------------------------------------
template <int S> struct Store;
template <> struct Store<kF64> {
  using E = double;
  using T = double;
  static constexpr bool kSixteen = false;
  static __device__ __forceinline__ T in(E e, int a, T) { return e - wgt<T>(a); }
  static __device__ __forceinline__ T in_e(E e, int a) { return e - wgt<T>(a); }
  static __device__ __forceinline__ E out(T h, int a, T) { return h + wgt<T>(a); }
  static __device__ __forceinline__ double to_f64(const E* p, int, T) { return *p; }
  static __device__ __forceinline__ void from_f64(E* p, double f, int, T) { *p = f; }
  // npt = 2 consecutive elements as one 16-byte access, as offsets h = f - w.
  // load_h_plain: a plain load, for a buffer the kernel also writes (the
  // in-place steps); load_h takes the read-only data path.
  static __device__ __forceinline__ void load_h_plain(const E* p, T h[2], int a) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    h[0] = v.x - wgt<T>(a);
    h[1] = v.y - wgt<T>(a);
  }
  static __device__ __forceinline__ void load_h(const E* p, T h[2], int a) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    h[0] = v.x - wgt<T>(a);
    h[1] = v.y - wgt<T>(a);
  }
  static __device__ __forceinline__ void store_h(E* p, const T h[2], int a, const unsigned*, bool) {
    *reinterpret_cast<double2*>(p) = make_double2(h[0] + wgt<T>(a), h[1] + wgt<T>(a));
  }
  // one element's raw bits, rounded as store_h rounds it (r: the word of the
  // element's node pair, k: the element's place in the lane's vector)
  using R = unsigned long long;
  static __device__ __forceinline__ R round_e(T h, int a, unsigned, int, bool) {
    return static_cast<R>(__double_as_longlong(h + wgt<T>(a)));
  }
};
template <> struct Store<kF32> {
  // FP32 elements hold the offsets h = f - w as well: the same bytes as f,
  // with the rounding step of |h| <~ 0.1 instead of that of f ~ w.
  using E = float;
  using T = float;
  static constexpr bool kSixteen = false;
  static __device__ __forceinline__ T in(E e, int, T) { return e; }
  static __device__ __forceinline__ T in_e(E e, int) { return e; }
  static __device__ __forceinline__ E out(T h, int, T) { return h; }
  static __device__ __forceinline__ double to_f64(const E* p, int a, T) {
    return wgt<double>(a) + double(*p);
  }
  static __device__ __forceinline__ void from_f64(E* p, double f, int a, T) {
    *p = float(f - wgt<double>(a));
  }
  // npt = 4 consecutive elements as one 16-byte access
  static __device__ __forceinline__ void load_h_plain(const E* p, T h[4], int) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    h[0] = v.x;
    h[1] = v.y;
    h[2] = v.z;
    h[3] = v.w;
  }
  static __device__ __forceinline__ void load_h(const E* p, T h[4], int) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    h[0] = v.x;
    h[1] = v.y;
    h[2] = v.z;
    h[3] = v.w;
  }
  static __device__ __forceinline__ void store_h(E* p, const T h[4], int, const unsigned*, bool) {
    *reinterpret_cast<float4*>(p) = make_float4(h[0], h[1], h[2], h[3]);
  }
  using R = unsigned;
  static __device__ __forceinline__ R round_e(T h, int, unsigned, int, bool) { return __float_as_uint(h); }
};
// 16-bit offset forms: npt = 4 elements as one 8-byte access.
// Multipliers deriving each direction's rounding bits from the node's word
// (distinct odd constants: a bijection of 32-bit words per direction).
__device__ __forceinline__ constexpr unsigned round_mul(int a) {
  return a == 0 ? 0x9e3779b1u : a == 1 ? 0x85ebca77u : a == 2 ? 0xc2b2ae3du : a == 3 ? 0x27d4eb2fu
       : a == 4 ? 0x165667b1u : a == 5 ? 0xd3a2646du : a == 6 ? 0xfd7046c5u : a == 7 ? 0xb55a4f09u
       : 0x68e31da5u;
}

// Packed conversion of two FP32 values to two 16-bit values in one register
// (lo in the low half, the lower address): round to nearest even.
__device__ __forceinline__ unsigned pack_f16_rn(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ unsigned pack_bf16_rn(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// Stochastic rounding of two FP32 values to two 16-bit values with the
// hardware conversion (cvt.rs): each result adds random bits below its kept
// significand bits and truncates, so the magnitude rounds up with probability
// equal to its distance from the lower neighbour. The low result takes its
// bits from the low half of rbits, the high result from the high half (the
// lowest 13 bits of each half for FP16, all 16 for BF16).
__device__ __forceinline__ unsigned pack_f16_rs(float lo, float hi, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
__device__ __forceinline__ unsigned pack_bf16_rs(float lo, float hi, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
// Rounding bits of direction a for a pair of nodes: their 32-bit pair word
// times the direction's odd constant; the low half goes to the first node,
// the high half to the second. The pair word is a full 32-bit hash, so the
// two halves are independent; each direction's bits are a different
// bijection of them.
__device__ __forceinline__ unsigned pair_bits(unsigned pair_word, int a) {
  return pair_word * round_mul(a);
}

// 16-bit offset forms: npt = 4 elements as one 8-byte access; an element
// holds h - ref (FP32 arithmetic on both sides of the conversion).
template <class H>
struct Store16 {
  using E = H;
  using T = float;
  static constexpr bool kSixteen = true;
};
template <> struct Store<kF16> : Store16<__half> {
  static __device__ __forceinline__ void load_h_plain(const E* p, T e[4], int) {
    unpack(*reinterpret_cast<const uint2*>(p), e);
  }
  static __device__ __forceinline__ void load_h(const E* p, T e[4], int) {
    unpack(__ldg(reinterpret_cast<const uint2*>(p)), e);
  }
  static __device__ __forceinline__ void unpack(const uint2 v, T e[4]) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    e[0] = a.x;
    e[1] = a.y;
    e[2] = b.x;
    e[3] = b.y;
  }
  // r[j]: the rounding word of node pair j (stochastic rounding only)
  static __device__ __forceinline__ void store_h(E* p, const T e[4], int a, const unsigned* r,
                                                 bool sr) {
    uint2 v;
    if (sr) {
      v.x = pack_f16_rs(e[0], e[1], pair_bits(r[0], a));
      v.y = pack_f16_rs(e[2], e[3], pair_bits(r[1], a));
    } else {
      v.x = pack_f16_rn(e[0], e[1]);
      v.y = pack_f16_rn(e[2], e[3]);
    }
    *reinterpret_cast<uint2*>(p) = v;
  }
  static __device__ __forceinline__ T in_e(E e, int) { return __half2float(e); }
  static __device__ __forceinline__ T in(E e, int, T ref) { return __half2float(e) + ref; }
  static __device__ __forceinline__ E out(T h, int, T ref) { return __float2half_rn(h - ref); }
  // one element as store_h rounds it (the packed conversions round each half alike)
  using R = unsigned short;
  static __device__ __forceinline__ R round_e(T e, int a, unsigned r, int k, bool sr) {
    return sr ? (unsigned short)(pack_f16_rs(e, 0.f, pair_bits(r, a) >> (16 * (k & 1))) & 0xffffu)
              : __half_as_ushort(__float2half_rn(e));
  }
  // f of a stored element: w + (element + ref), the offset as the kernel forms it
  static __device__ __forceinline__ double to_f64(const E* p, int a, T ref) {
    return wgt<double>(a) + double(__half2float(*p) + ref);
  }
  static __device__ __forceinline__ void from_f64(E* p, double f, int a, T ref) {
    *p = __double2half(f - wgt<double>(a) - double(ref));
  }
};
template <> struct Store<kBF16> : Store16<__nv_bfloat16> {
  static __device__ __forceinline__ void load_h_plain(const E* p, T e[4], int) {
    unpack(*reinterpret_cast<const uint2*>(p), e);
  }
  static __device__ __forceinline__ void load_h(const E* p, T e[4], int) {
    unpack(__ldg(reinterpret_cast<const uint2*>(p)), e);
  }
  // a bf16 is the upper half of an FP32: widening is a shift or a mask
  static __device__ __forceinline__ void unpack(const uint2 v, T e[4]) {
    e[0] = __uint_as_float(v.x << 16);
    e[1] = __uint_as_float(v.x & 0xffff0000u);
    e[2] = __uint_as_float(v.y << 16);
    e[3] = __uint_as_float(v.y & 0xffff0000u);
  }
  static __device__ __forceinline__ void store_h(E* p, const T e[4], int a, const unsigned* r,
                                                 bool sr) {
    uint2 v;
    if (sr) {
      v.x = pack_bf16_rs(e[0], e[1], pair_bits(r[0], a));
      v.y = pack_bf16_rs(e[2], e[3], pair_bits(r[1], a));
    } else {
      v.x = pack_bf16_rn(e[0], e[1]);
      v.y = pack_bf16_rn(e[2], e[3]);
    }
    *reinterpret_cast<uint2*>(p) = v;
  }
  static __device__ __forceinline__ T in_e(E e, int) { return __bfloat162float(e); }
  static __device__ __forceinline__ T in(E e, int, T ref) { return __bfloat162float(e) + ref; }
  static __device__ __forceinline__ E out(T h, int, T ref) { return __float2bfloat16_rn(h - ref); }
  using R = unsigned short;
  static __device__ __forceinline__ R round_e(T e, int a, unsigned r, int k, bool sr) {
    return sr ? (unsigned short)(pack_bf16_rs(e, 0.f, pair_bits(r, a) >> (16 * (k & 1))) & 0xffffu)
              : __bfloat16_as_ushort(__float2bfloat16_rn(e));
  }
  static __device__ __forceinline__ double to_f64(const E* p, int a, T ref) {
    return wgt<double>(a) + double(__bfloat162float(*p) + ref);
  }
  static __device__ __forceinline__ void from_f64(E* p, double f, int a, T ref) {
    *p = __double2bfloat16(f - wgt<double>(a) - double(ref));
  }
};

// The reference of direction a's stored elements (16-bit stores; 0 otherwise).
template <class S>
__device__ __forceinline__ typename S::T sref(const StepParams& p, int a) {
  if constexpr (S::kSixteen)
    return p.cf.h_ref[a];
  else
    return typename S::T(0);
}

// Scalar offset load/store of one population of direction a.
template <class S>
__device__ __forceinline__ typename S::T load_h(const StepParams& p, const typename S::E* ptr, int a) {
  return S::in(__ldg(ptr), a, sref<S>(p, a));
}
template <class S>
__device__ __forceinline__ void store_h(const StepParams& p, typename S::E* ptr, typename S::T h, int a) {
  *ptr = S::out(h, a, sref<S>(p, a));
}

// Random bits of the stochastic rounding: the MurmurHash3 32-bit finalizer
// (Appleby) of the node's index mixed with the step's key gives one uniform
// 32-bit word per node; direction alpha uses the word times a distinct odd
// constant (a bijection of 32-bit words, so each direction's bits are again
// uniform) and takes its top bits.
__device__ __forceinline__ unsigned round_bits(unsigned counter, unsigned key) {
  unsigned h = counter ^ key;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}



// Convective outlet (Section 3.3, after Yang): the ghost column x = nx of
// direction as (3, 6 or 7), row ys, advanced by the implicit upwind step of
// dg/dt + U_c dg/dx = 0 from the last column's f*(t):
// g^t = (g^{t-1} + U_c f*(nx - 1)) / (1 + U_c), in offsets (the weights cancel).
// The step's one reader of each entry writes g^t to ghost_dst (write = true).
template <class S>
__device__ __forceinline__ typename S::T outlet_ghost(const StepParams& p,
                                                      const typename S::E* src, int as, int ys,
                                                      bool write) {
  using T = typename S::T;
  const Consts<T>& c = consts<T>(p);
  const long long gi = (long long)(as == 3 ? 0 : (as == 6 ? 1 : 2)) * p.ny + ys;
  const T f_last = load_h<S>(p, src + (long long)as * p.plane + (long long)ys * p.pitch + (p.nx - 1), as);
  const T g = (static_cast<const T*>(p.ghost_src)[gi] + c.u_conv * f_last) * c.conv_inv;
  if (write) static_cast<T*>(p.ghost_dst)[gi] = g;
  return g;
}

// The same ghost value in the in-place (AA) push step, whose store no longer
// holds the last column intact (the neighbours' pushes overwrite it): the
// stored f*(nx - 1) comes from the side copy z that the local step wrote.
// ESP: the value as an element (offset minus the reference) instead of an
// offset; the convective state itself is always kept as offsets.
template <class S, bool ESP = false>
__device__ __forceinline__ typename S::T outlet_ghost_aa(const StepParams& p, int as, int ys,
                                                         bool write) {
  using T = typename S::T;
  const long long gi = (long long)(as == 3 ? 0 : (as == 6 ? 1 : 2)) * p.ny + ys;
  const typename S::E ze = static_cast<const typename S::E*>(p.z)[gi];
  if (p.bc_x != kBcInletConvective)  // zero gradient
    return ESP ? S::in_e(ze, as) : S::in(ze, as, sref<S>(p, as));
  const T f_last = S::in(ze, as, sref<S>(p, as));
  const Consts<T>& c = consts<T>(p);
  const T g = (static_cast<const T*>(p.ghost_src)[gi] + c.u_conv * f_last) * c.conv_inv;
  if (write && p.ghost_dst) static_cast<T*>(p.ghost_dst)[gi] = g;
  return ESP ? g - sref<S>(p, as) : g;
}

// ---------------------------------------------------------------------------
// Pull with boundary conditions (streaming, left-hand side of Eq. LatticeBoltz)
// ---------------------------------------------------------------------------
template <class S, int A>
__device__ __forceinline__ typename S::T pull_bc(const StepParams& p, const typename S::E* src,
                                                 int x, int y) {
  using T = typename S::T;
  int as = A;
  int xs = x - cx(A);
  int ys = y - cy(A);
  if (ys < 0 || ys >= p.ny) {
    if (p.bc_y == kBcPeriodic) {
      ys = ys < 0 ? ys + p.ny : ys - p.ny;
    } else {  // free slip: the mirror of the population that left this row
      as = mirror_y(A);
      ys = y;
    }
  }
  if (xs < 0 || xs >= p.nx) {
    if (p.bc_x == kBcPeriodic) {
      xs = xs < 0 ? xs + p.nx : xs - p.nx;
    } else if (xs < 0) {  // inlet ghost column at f_eq(1, u_in)
      const Consts<T>& c = consts<T>(p);
      return as == A ? c.heq_in[A] : c.heq_in[mirror_y(A)];
    } else if (p.bc_x == kBcInletConvective) {  // read only: the step writes the state
      return outlet_ghost<S>(p, src, as, ys, false);
    } else {  // zero-gradient outlet ghost column
      xs = p.nx - 1;
    }
  }
  return load_h<S>(p, src + (long long)as * p.plane + (long long)ys * p.pitch + xs, as);
}

// The nine pulled populations of node (x, y), one at a time with the boundary
// rules (the diagnostics' scalar pull; the fused step pulls whole vectors).
template <class S>
__device__ __forceinline__ void pull_node(const StepParams& p, const typename S::E* src, int x,
                                          int y, typename S::T h[9]) {
  h[0] = pull_bc<S, 0>(p, src, x, y);
  h[1] = pull_bc<S, 1>(p, src, x, y);
  h[2] = pull_bc<S, 2>(p, src, x, y);
  h[3] = pull_bc<S, 3>(p, src, x, y);
  h[4] = pull_bc<S, 4>(p, src, x, y);
  h[5] = pull_bc<S, 5>(p, src, x, y);
  h[6] = pull_bc<S, 6>(p, src, x, y);
  h[7] = pull_bc<S, 7>(p, src, x, y);
  h[8] = pull_bc<S, 8>(p, src, x, y);
}

// ---------------------------------------------------------------------------
// Density, implicit velocity and penalization force of one node
// (Eqs. density, velocity, 17 and 18).
//   d = j + rho g / 2 - rho u_s,  u = u_s + d / (rho (1 + a)),
//   f_pen = -kappa d,  a = chi/(2 eta),  kappa = (chi/eta)/(1 + a).
// This is Eq. 18 rewritten so that neither u - u_s nor a rho u_s appear:
// the 1/eta factor never multiplies a rounding error.
// ---------------------------------------------------------------------------
// Correctly rounded reciprocal.
__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip(double v) { return __drcp_rn(v); }

template <class T>
struct Macro {
  T drho, rho, ux, uy, fpx, fpy, Fx, Fy;
};

template <class T>
__device__ __forceinline__ void solid_velocity(const StepParams& p, uint8_t m, int x, int y,
                                               T& usx, T& usy) {
  if (m == kStaticSolid) {
    if (p.us) {
      const long long i = (long long)y * p.pitch + x;
      if (sizeof(T) == 8) {
        const double2 v = reinterpret_cast<const double2*>(p.us)[i];
        usx = T(v.x);
        usy = T(v.y);
      } else {
        const float2 v = reinterpret_cast<const float2*>(p.us)[i];
        usx = T(v.x);
        usy = T(v.y);
      }
    }
  } else if (m <= p.n_bodies) {
    const T* b = consts<T>(p).body[m - 1];
    const T dx = T(x) - b[0];
    const T dy = T(y) - b[1];
    usx = b[2] - b[4] * dy;
    usy = b[3] + b[4] * dx;
  }
  // any other label (only a caller-written mask can hold one) is solid at rest
}

// Sum and difference of the offsets of the opposite pair k ((1,3), (2,4),
// (5,7), (6,8)) whose values the kernel holds in ha, hb: offsets themselves,
// or (REF) the elements e = h - h_ref of a 16-bit store. h_ref is odd in xi,
// so the pair sum of the elements is that of the offsets, and the difference
// is decoded with the pair's reference difference (exact in FP32).
template <class T>
__device__ __forceinline__ T pair_s(T ha, T hb) {
  return ha + hb;
}
template <class T, bool REF>
__device__ __forceinline__ T pair_d(const Consts<T>& c, T ha, T hb, int k) {
  if constexpr (REF)
    return (ha - hb) + c.r_d[k];
  else
    return ha - hb;
}

// FREE: a fluid node (m = 0) without body force (g = 0), for which Eqs. 17
// and 18 reduce to f_pen = 0 and u = j / rho; the same values as the general
// form, which would compute them through zero terms.
// REF: h holds the elements e = h - h_ref of a 16-bit store.
template <class T, bool FREE = false, bool REF = false>
__device__ __forceinline__ Macro<T> macros(const StepParams& p, const T h[9], uint8_t m, int x,
                                           int y) {
  Macro<T> r;
  const Consts<T>& c = consts<T>(p);
  // sums and differences of opposite populations (the two-rate collision
  // reuses them)
  const T s13 = pair_s<T>(h[1], h[3]), s24 = pair_s<T>(h[2], h[4]);
  const T s57 = pair_s<T>(h[5], h[7]), s68 = pair_s<T>(h[6], h[8]);
  const T d13 = pair_d<T, REF>(c, h[1], h[3], 0), d24 = pair_d<T, REF>(c, h[2], h[4], 1);
  const T d57 = pair_d<T, REF>(c, h[5], h[7], 2), d68 = pair_d<T, REF>(c, h[6], h[8], 3);
  r.drho = h[0] + ((s13 + s24) + (s57 + s68));
  r.rho = T(1) + r.drho;
  const T jx = d13 + (d57 - d68);
  const T jy = d24 + (d57 + d68);
  if constexpr (FREE) {
    const T inv = recip(r.rho);
    r.ux = jx * inv;
    r.uy = jy * inv;
    r.fpx = r.fpy = r.Fx = r.Fy = T(0);
    return r;
  }
  T usx = T(0), usy = T(0), a = T(0), kap = T(0);
  if (m) {
    a = c.a_s;
    kap = c.kappa_s;
    solid_velocity<T>(p, m, x, y, usx, usy);
  }
  const T gx = c.gx, gy = c.gy;
  const T dx = jx + T(0.5) * r.rho * gx - r.rho * usx;
  const T dy = jy + T(0.5) * r.rho * gy - r.rho * usy;
  const T inv = recip(r.rho * (T(1) + a));
  r.ux = usx + dx * inv;
  r.uy = usy + dy * inv;
  r.fpx = -kap * dx;
  r.fpy = -kap * dy;
  r.Fx = r.fpx + r.rho * gx;
  r.Fy = r.fpy + r.rho * gy;
  return r;
}

// ---------------------------------------------------------------------------
// Collision on offsets, two-rate form.
// The printed S relaxes the even moments (e, eps, p_xx, p_xy: symmetric under
// xi -> -xi) at s+ = s_n and the odd ones (q_x, q_y) at s- = s_q; the rates of
// rho, j_x and j_y do not change the result (rho = rho_eq, and j* = j + F for
// any rate because m_eq uses the half-force velocity). Splitting each pair of
// opposite populations into its even and odd parts, h+- = (h_a +- h_abar)/2,
// Eq. equa_lbl_mrt with Eq. Guo2 is then, per pair,
//   h*_a    = h_a    + P + Q,   h*_abar = h_abar + P - Q,
//   P = -s+ (h+ - heq+) + (1 - s+/2) G+,   Q = -s- (h- - heq-) + (1 - s-/2) G-,
// with heq+ = w (drho - 1.5 rho u.u + 4.5 rho (xi.u)^2), heq- = 3 w rho xi.u,
// G+ = w (9 (xi.u)(xi.F) - 3 u.F), G- = 3 w xi.F (the even and odd parts of
// Eq. Guo2's F_a), and for the rest population h*_0 = (1 - s+) h_0 + w_0 K,
// K = s+ (drho - 1.5 rho u.u) - 3 (1 - s+/2) u.F. SRT with Eq. Guo1 is the
// same with s+ = s- = 1/tau. This is the moment-space operator rearranged,
// not an approximation of it.
// On the elements e = h - r of a 16-bit store (REF) the update is the same,
// e*_a = e_a + P + Q, with d decoded from the elements (pair_d); r is odd in
// xi, so s, e_0 = h_0 and the rest population's update need no decoding.
// ---------------------------------------------------------------------------
template <class T, bool FREE>
__device__ __forceinline__ void trt_pair(T& ha, T& hb, T s, T d, T xu, T xF, T kw, T aw, T bw,
                                         T amw, T bmw, T hsp, T hsm) {
  // w (s+ heq+ + c+ G+) and w (s- heq- + c- G-); without a force G+- = 0
  const T rp = FREE ? xu * (aw * xu) + kw : xu * (aw * xu + bw * xF) + kw;
  const T rm = FREE ? amw * xu : amw * xu + bmw * xF;
  const T P = rp - hsp * s;
  const T Q = rm - hsm * d;
  ha = ha + (P + Q);
  hb = hb + (P - Q);
}

template <class T, bool FREE = false, bool REF = false>
__device__ __forceinline__ void collide_trt(const StepParams& p, T h[9], const Macro<T>& q) {
  const Consts<T>& c = consts<T>(p);
  const T ux = q.ux, uy = q.uy, Fx = q.Fx, Fy = q.Fy, rho = q.rho;
  const T uu = ux * ux + uy * uy;
  const T K = FREE ? c.t_sp * (q.drho - T(1.5) * rho * uu)
                   : c.t_sp * (q.drho - T(1.5) * rho * uu) - c.t_c3p * (ux * Fx + uy * Fy);
  const T k9 = K * T(1.0 / 9.0), k36 = K * T(1.0 / 36.0);
  const T a9 = c.t_a[0] * rho, a36 = c.t_a[1] * rho;
  const T am9 = c.t_am[0] * rho, am36 = c.t_am[1] * rho;
  // the pair sums and differences as macros() formed them
  const T s13 = pair_s<T>(h[1], h[3]), s24 = pair_s<T>(h[2], h[4]);
  const T s57 = pair_s<T>(h[5], h[7]), s68 = pair_s<T>(h[6], h[8]);
  const T d13 = pair_d<T, REF>(c, h[1], h[3], 0), d24 = pair_d<T, REF>(c, h[2], h[4], 1);
  const T d57 = pair_d<T, REF>(c, h[5], h[7], 2), d68 = pair_d<T, REF>(c, h[6], h[8], 3);
  h[0] = c.t_1msp * h[0] + T(4.0 / 9.0) * K;
  trt_pair<T, FREE>(h[1], h[3], s13, d13, ux, Fx, k9, a9, c.t_b[0], am9, c.t_bm[0], c.t_hsp,
                    c.t_hsm);
  trt_pair<T, FREE>(h[2], h[4], s24, d24, uy, Fy, k9, a9, c.t_b[0], am9, c.t_bm[0], c.t_hsp,
                    c.t_hsm);
  trt_pair<T, FREE>(h[5], h[7], s57, d57, ux + uy, Fx + Fy, k36, a36, c.t_b[1], am36, c.t_bm[1],
                    c.t_hsp, c.t_hsm);
  trt_pair<T, FREE>(h[6], h[8], s68, d68, uy - ux, Fy - Fx, k36, a36, c.t_b[1], am36, c.t_bm[1],
                    c.t_hsp, c.t_hsm);
}

// MRT (Eq. equa_lbl_mrt with Lu forcing, Eq. Guo2), on the moments of h, for
// rates without the two-rate structure.
// m = M h with M of Eq. eq1.7; since M w = (1, -2, 1, 0, ...), the equilibrium
// moments of h are m_eq(rho, u) - M w. The forcing moments M F are
// (0, 6 u.F, -6 u.F, F_x, -F_x, F_y, -F_y, 2 (u F_x - v F_y), u F_y + v F_x).
// Rates of the conserved moments (rho, j_x, j_y) do not change the result
// (j* = j + F for any rate, because m_eq uses the half-force velocity).
// f* = M^-1 m* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
template <class T>
__device__ __forceinline__ void collide_mrt(const StepParams& p, T h[9], const Macro<T>& q) {
  const Consts<T>& c = consts<T>(p);
  const T s1 = c.s_e, s2 = c.s_eps, s4 = c.s_qx, s6 = c.s_qy, s7 = c.s_pxx, s8 = c.s_pxy;
  const T sum14 = (h[1] + h[2]) + (h[3] + h[4]);
  const T sum58 = (h[5] + h[6]) + (h[7] + h[8]);
  const T e = -T(4) * h[0] - sum14 + T(2) * sum58;
  const T eps = T(4) * h[0] - T(2) * sum14 + sum58;
  const T jx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
  const T qx = T(2) * (h[3] - h[1]) + (h[5] - h[6]) + (h[8] - h[7]);
  const T jy = (h[2] - h[4]) + (h[5] + h[6]) - (h[7] + h[8]);
  const T qy = T(2) * (h[4] - h[2]) + (h[5] + h[6]) - (h[7] + h[8]);
  const T pxx = (h[1] - h[2]) + (h[3] - h[4]);
  const T pxy = (h[5] - h[6]) + (h[7] - h[8]);

  const T rho = q.rho, ux = q.ux, uy = q.uy, Fx = q.Fx, Fy = q.Fy;
  const T uu = ux * ux + uy * uy;
  const T uF = ux * Fx + uy * Fy;
  const T e_eq = -T(2) * q.drho + T(3) * rho * uu;
  const T eps_eq = q.drho - T(3) * rho * uu;

  const T es = e - s1 * (e - e_eq) + (T(1) - T(0.5) * s1) * T(6) * uF;
  const T epss = eps - s2 * (eps - eps_eq) - (T(1) - T(0.5) * s2) * T(6) * uF;
  const T jxs = jx + Fx;
  const T jys = jy + Fy;
  const T qxs = qx - s4 * (qx + rho * ux) - (T(1) - T(0.5) * s4) * Fx;
  const T qys = qy - s6 * (qy + rho * uy) - (T(1) - T(0.5) * s6) * Fy;
  const T pxxs = pxx - s7 * (pxx - rho * (ux * ux - uy * uy)) +
                 (T(1) - T(0.5) * s7) * T(2) * (ux * Fx - uy * Fy);
  const T pxys = pxy - s8 * (pxy - rho * ux * uy) + (T(1) - T(0.5) * s8) * (ux * Fy + uy * Fx);

  const T a0 = q.drho * T(1.0 / 9.0);
  const T a1 = es * T(1.0 / 36.0);
  const T a2 = epss * T(1.0 / 36.0);
  const T a3 = jxs * T(1.0 / 6.0);
  const T a4 = qxs * T(1.0 / 12.0);
  const T a5 = jys * T(1.0 / 6.0);
  const T a6 = qys * T(1.0 / 12.0);
  const T a7 = pxxs * T(0.25);
  const T a8 = pxys * T(0.25);

  const T b14 = a0 - a1 - T(2) * a2;  // common part of directions 1..4
  const T b58 = a0 + T(2) * a1 + a2;  // common part of directions 5..8
  h[0] = a0 - T(4) * a1 + T(4) * a2;
  h[1] = b14 + (a3 - T(2) * a4) + a7;
  h[2] = b14 + (a5 - T(2) * a6) - a7;
  h[3] = b14 - (a3 - T(2) * a4) + a7;
  h[4] = b14 - (a5 - T(2) * a6) - a7;
  h[5] = b58 + (a3 + a4) + (a5 + a6) + a8;
  h[6] = b58 - (a3 + a4) + (a5 + a6) - a8;
  h[7] = b58 - (a3 + a4) - (a5 + a6) + a8;
  h[8] = b58 + (a3 + a4) - (a5 + a6) - a8;
}

// ---------------------------------------------------------------------------
// Deterministic block and grid reductions in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v[0..2] over the block of NT threads, fixed order; result valid in
// thread 0.
template <int NT = kThreads>
__device__ __forceinline__ void block_sum3(double v[3], double (*sm)[3]) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  constexpr int n_warps = NT / 32;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
    sm[warp][0] = v[0];
    sm[warp][1] = v[1];
    sm[warp][2] = v[2];
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int w = 0; w < n_warps; ++w) s += sm[w][k];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Finishes the per-step reduction once this tile's partial is written: the
// last tile of each group of kGroup tiles sums the group in tile order, and
// the last group to finish sums the groups in group order and writes the
// step's record (a grid of a single group writes its group sum directly).
// Both levels are fixed-order, so the result does not depend on which blocks
// ran when.
template <int NT>
__device__ __forceinline__ void finish_reduction(const StepParams& p, int tile, long long t,
                                                 const double tile_sum[3], double (*sm)[3]) {
  __shared__ int s_last;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  constexpr int n_threads = NT;
  const int group = tile / kGroup;
  const int n_groups = (p.n_tiles + kGroup - 1) / kGroup;
  if (tid == 0) {
    double* dst = p.partials + 3ll * tile;
    __stcg(dst + 0, tile_sum[0]);
    __stcg(dst + 1, tile_sum[1]);
    __stcg(dst + 2, tile_sum[2]);
    __threadfence();
    const int gsize = min(kGroup, p.n_tiles - group * kGroup);
    const unsigned prev = atomicAdd(p.counters + group, 1u);
    s_last = (prev == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  {
    double v[3] = {0.0, 0.0, 0.0};
    const int t0 = group * kGroup;
    const int gsize = min(kGroup, p.n_tiles - t0);
    // each thread adds its strided share of the group's tiles in increasing
    // order (one tile per thread for 8-warp blocks, two for 4-warp blocks)
    for (int i = tid; i < gsize; i += n_threads) {
      const double* src = p.partials + 3ll * (t0 + i);
      v[0] += __ldcg(src + 0);
      v[1] += __ldcg(src + 1);
      v[2] += __ldcg(src + 2);
    }
    block_sum3<NT>(v, sm);
    if (tid == 0) {
      p.counters[group] = 0u;  // ready for the next step
      if (n_groups == 1) {
        // one group (a small grid): its sum is the step's record
        double* r = p.ring + 3ll * (t % p.ring_len);
        r[0] = v[0];
        r[1] = v[1];
        r[2] = p.reduce_mass ? v[2] : 0.0;
        s_last = 0;
      } else {
        double* g = p.group_partials + 3ll * group;
        __stcg(g + 0, v[0]);
        __stcg(g + 1, v[1]);
        __stcg(g + 2, v[2]);
        __threadfence();
        const unsigned prev = atomicAdd(p.counters + n_groups, 1u);
        s_last = (prev == (unsigned)(n_groups - 1));
      }
    }
    __syncthreads();
  }
  if (!s_last) return;
  __threadfence();
  double v[3] = {0.0, 0.0, 0.0};
  for (int g = tid; g < n_groups; g += n_threads) {
    // each thread adds its strided share in increasing group order
    v[0] += __ldcg(p.group_partials + 3ll * g + 0);
    v[1] += __ldcg(p.group_partials + 3ll * g + 1);
    v[2] += __ldcg(p.group_partials + 3ll * g + 2);
  }
  block_sum3<NT>(v, sm);
  if (tid == 0) {
    double* r = p.ring + 3ll * (t % p.ring_len);
    r[0] = v[0];
    r[1] = v[1];
    r[2] = p.reduce_mass ? v[2] : 0.0;
    p.counters[n_groups] = 0u;
  }
}

// ---------------------------------------------------------------------------
// The fused time step of one tile: (32 N) x tile_y nodes, N = npt(STORE). Lane
// l of warp w takes nodes x0 + N l .. x0 + N l + N - 1 of rows y0 + w + W r,
// r = 0..rows_per_warp-1, W = warps_per_block(STORE).
//
// Every direction is pulled with one N-element vector load per lane: a
// direction with xi_x = +1 takes its first node's value from the lane to the
// left (warp shuffle), one with xi_x = -1 its last node's value from the lane
// to the right, and only the edge lanes 0 and 31 load that one value
// themselves. Interior tiles (no boundary within one node) do nothing else.
// Tiles touching a boundary (GEN) also remap: the source row of each direction
// (periodic wrap or free-slip mirror, uniform across the warp), the edge
// lanes' single values (periodic wrap, inlet ghost, outlet copy), and the value
// entering the domain's last column; lanes past the last column load and
// store nothing. The arithmetic per node is the same on both paths.
// ---------------------------------------------------------------------------
// AA: the push step reads f*_as(xs, ys) from the opposite slot of the source
// node (where the local step put it), with plain (coherent) loads, since the
// kernel also writes this buffer.
// ESP: the value as an element of direction A (offset minus the reference),
// as the fused step works on them; the reference is even in xi_y, so the
// mirrored source as of a free-slip wall has A's reference.
template <class S, int A, bool AA = false, bool ESP = false>
__device__ __forceinline__ typename S::T edge_pull(const StepParams& p, const typename S::E* src,
                                                   int as, int ys, int xs) {
  using T = typename S::T;
  if (xs < 0 || xs >= p.nx) {
    if (p.bc_x == kBcPeriodic) {
      xs %= p.nx;
      if (xs < 0) xs += p.nx;
    } else if (xs < 0) {  // inlet ghost column at f_eq(1, u_in)
      const Consts<T>& c = consts<T>(p);
      const T h = as == A ? c.heq_in[A] : c.heq_in[mirror_y(A)];
      return ESP ? h - sref<S>(p, A) : h;
    } else if (AA) {
      return outlet_ghost_aa<S, ESP>(p, as, ys, xs == p.nx);
    } else if (p.bc_x == kBcInletConvective) {
      // xs == nx: the last column's own pull (the entry's one reader); beyond
      // it, the unused edge value of a lane past the last column
      const T g = outlet_ghost<S>(p, src, as, ys, xs == p.nx);
      return ESP ? g - sref<S>(p, A) : g;
    } else {  // zero-gradient outlet ghost column
      xs = p.nx - 1;
    }
  }
  const typename S::E e = AA ? src[(long long)opposite(as) * p.plane + (long long)ys * p.pitch + xs]
                             : __ldg(src + (long long)as * p.plane + (long long)ys * p.pitch + xs);
  return ESP ? S::in_e(e, as) : S::in(e, as, sref<S>(p, as));
}

template <class S, int N, int A, bool GEN, bool AA = false>
__device__ __forceinline__ void pull_dir_vec(const StepParams& p, const typename S::E* src, int xb,
                                             int y, int lane, bool lane_active,
                                             typename S::T (&h)[N][9]) {
  using T = typename S::T;
  using E = typename S::E;
  int as = A;
  int ys = y - cy(A);
  if (GEN && (ys < 0 || ys >= p.ny)) {
    if (p.bc_y == kBcPeriodic) {
      ys = ys < 0 ? ys + p.ny : ys - p.ny;
    } else {  // free slip: the mirror of the population that left this row
      as = mirror_y(A);
      ys = y;
    }
  }
  const E* row = src + (long long)(AA ? opposite(as) : as) * p.plane + (long long)ys * p.pitch;
  T v[N];
  if (!GEN || lane_active) {
    if (AA)
      S::load_h_plain(row + xb, v, as);
    else
      S::load_h(row + xb, v, as);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = T(0);
  }
  if (cx(A) == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) h[k][A] = v[k];
  } else if (cx(A) == 1) {  // node k pulls from x - 1
    T left = __shfl_up_sync(0xffffffffu, v[N - 1], 1);
    // the edge lanes' extra value: through the x boundary rules only where
    // it lies outside the grid (the source row already carries the y rules)
    if (lane == 0)
      left = GEN && xb - 1 < 0 ? edge_pull<S, A, AA, true>(p, src, as, ys, xb - 1)
                               : S::in_e(AA ? row[xb - 1] : __ldg(row + xb - 1), as);
    h[0][A] = left;
#pragma unroll
    for (int k = 1; k < N; ++k) h[k][A] = v[k - 1];
  } else {  // node k pulls from x + 1
    T right = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == kLanes - 1)
      right = GEN && xb + N >= p.nx ? edge_pull<S, A, AA, true>(p, src, as, ys, xb + N)
                                    : S::in_e(AA ? row[xb + N] : __ldg(row + xb + N), as);
#pragma unroll
    for (int k = 0; k < N - 1; ++k) h[k][A] = v[k + 1];
    h[N - 1][A] = right;
    if (GEN && xb <= p.nx - 1 && xb + N > p.nx - 1) {
      // the domain's last column pulls from beyond it, through the x boundary
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (xb + k == p.nx - 1) h[k][A] = edge_pull<S, A, AA, true>(p, src, as, ys, p.nx);
    }
  }
}

// ---------------------------------------------------------------------------
// In-place (AA-pattern) streaming on one buffer. A push step reads each
// population from the opposite slot of its source node (where the previous
// local step put it), collides, and writes f*_a to slot a of the node it
// streams to; a local step reads a node's own slots, collides, and writes f*_a
// to the node's opposite slot. Every location a push step reads is written by
// the same node, after its read: in the vector layout both happen in the lane
// that owns the location's aligned vector (or the edge lane's extra element),
// so the buffer can be updated in place. Each value is rounded with the bits
// of its node, direction and step, as the A/B scheme rounds it, so the two
// schemes give bitwise the same populations.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void store_raw(typename S::E* p, typename S::R w) {
  *reinterpret_cast<typename S::R*>(p) = w;
}
// N raw elements to an aligned vector (16 bytes, or 8 for 16-bit storage)
template <class S, int N>
__device__ __forceinline__ void store_raw_vec(typename S::E* p, const typename S::R (&w)[N]) {
  if constexpr (sizeof(typename S::E) == 2) {
    uint2 v;
    v.x = unsigned(w[0]) | (unsigned(w[1 % N]) << 16);
    v.y = unsigned(w[2 % N]) | (unsigned(w[3 % N]) << 16);
    *reinterpret_cast<uint2*>(p) = v;
  } else if constexpr (sizeof(typename S::E) == 4) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1 % N], w[2 % N], w[3 % N]);
  } else {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(w[0], w[1 % N]);
  }
}
template <class R>
__device__ __forceinline__ R shfl_up_raw(R v) {
  if constexpr (sizeof(R) == 8)
    return __shfl_up_sync(0xffffffffu, v, 1);
  else
    return R(__shfl_up_sync(0xffffffffu, unsigned(v), 1));
}
template <class R>
__device__ __forceinline__ R shfl_down_raw(R v) {
  if constexpr (sizeof(R) == 8)
    return __shfl_down_sync(0xffffffffu, v, 1);
  else
    return R(__shfl_down_sync(0xffffffffu, unsigned(v), 1));
}

// Slot of the value that a push step sends out through an open x side:
// lost[side][k][y], side 0 = x = nx - 1 (alpha = 1, 5, 8), 1 = x = 0 (alpha = 3, 6, 7).
__device__ __forceinline__ long long lost_index(const StepParams& p, int a, int y, bool left) {
  const int k = left ? (a == 3 ? 0 : (a == 6 ? 1 : 2)) : (a == 1 ? 0 : (a == 5 ? 1 : 2));
  return (long long)((left ? 3 : 0) + k) * p.ny + y;
}

// Where a push step puts f*_a of node (x, y): the pull's boundary rules read
// backwards (periodic wrap; a free-slip wall returns it as mirror_y(a) in the
// same row at x + cx(a)). Returns false when it leaves through an open x side.
__device__ __forceinline__ bool push_target(const StepParams& p, int a, int x, int y, int* ap,
                                            int* xt, int* yt) {
  *ap = a;
  *xt = x + cx(a);
  *yt = y + cy(a);
  if (*yt < 0 || *yt >= p.ny) {
    if (p.bc_y == kBcPeriodic) {
      *yt = *yt < 0 ? *yt + p.ny : *yt - p.ny;
    } else {
      *ap = mirror_y(a);
      *yt = y;
    }
  }
  if (*xt < 0 || *xt >= p.nx) {
    if (p.bc_x != kBcPeriodic) return false;
    *xt = *xt < 0 ? *xt + p.nx : *xt - p.nx;
  }
  return true;
}

template <class S>
__device__ __forceinline__ void push_one(const StepParams& p, typename S::E* buf, int a, int x, int y,
                                         typename S::R e) {
  int ap, xt, yt;
  if (push_target(p, a, x, y, &ap, &xt, &yt))
    store_raw<S>(buf + (long long)ap * p.plane + (long long)yt * p.pitch + xt, e);
  else
    store_raw<S>(static_cast<typename S::E*>(p.lost) + lost_index(p, a, y, x + cx(a) < 0), e);
}

// The outlet's ghost column (a copy of the last column) streams its
// populations alpha = 3, 6, 7 into the last column: the push step writes them
// where the next local step reads them (that step turns them into the
// zero-gradient or convective ghost values).
template <class S>
__device__ __forceinline__ void push_outlet_copy(const StepParams& p, typename S::E* buf, int as,
                                                 int y, typename S::R e) {
  int ap = as, yt = y + cy(as);
  if (yt < 0 || yt >= p.ny) {
    if (p.bc_y == kBcPeriodic) {
      yt = yt < 0 ? yt + p.ny : yt - p.ny;
    } else {
      ap = mirror_y(as);
      yt = y;
    }
  }
  store_raw<S>(buf + (long long)ap * p.plane + (long long)yt * p.pitch + (p.nx - 1), e);
}

// Interior tiles: the push of direction a as one aligned vector store per
// lane (the x-shifted element from the neighbouring lane); the edge lanes
// write the element that crosses into the next tile, and leave the one the
// neighbouring tile writes.
template <class S, int N>
__device__ __forceinline__ void push_dir_vec(const StepParams& p, typename S::E* buf, int a, int xb,
                                             int y, int lane, const typename S::R (&e)[N]) {
  using R = typename S::R;
  typename S::E* row = buf + (long long)a * p.plane + (long long)(y + cy(a)) * p.pitch;
  if (cx(a) == 0) {
    store_raw_vec<S, N>(row + xb, e);
  } else if (cx(a) == 1) {  // element j of this lane's vector receives node xb + j - 1
    R w[N];
    w[0] = shfl_up_raw(e[N - 1]);
#pragma unroll
    for (int j = 1; j < N; ++j) w[j] = e[j - 1];
    if (lane == 0) {
#pragma unroll
      for (int j = 1; j < N; ++j) store_raw<S>(row + xb + j, w[j]);
    } else {
      store_raw_vec<S, N>(row + xb, w);
    }
    if (lane == kLanes - 1) store_raw<S>(row + xb + N, e[N - 1]);
  } else {  // element j receives node xb + j + 1
    R w[N];
#pragma unroll
    for (int j = 0; j < N - 1; ++j) w[j] = e[j + 1];
    w[N - 1] = shfl_down_raw(e[0]);
    if (lane == kLanes - 1) {
#pragma unroll
      for (int j = 0; j < N - 1; ++j) store_raw<S>(row + xb + j, w[j]);
    } else {
      store_raw_vec<S, N>(row + xb, w);
    }
    if (lane == 0) store_raw<S>(row + xb - 1, e[0]);
  }
}

// Local step at the open x sides: the values the A/B pull would take from the
// ghost columns. Inlet: f_eq(1, u_in) for the directions entering at x = 0.
// Outlet: h holds the ghost column's copy of f*(nx - 1) (pushed there by the
// previous push step); the convective outlet advances its state from it.
// ESP: h holds elements (offsets minus the reference) instead of offsets.
template <class S, bool ESP = false>
__device__ __forceinline__ void aa_local_boundary(const StepParams& p, typename S::T h[9], int x,
                                                  int y, bool write) {
  using T = typename S::T;
  if (p.bc_x == kBcPeriodic) return;
  const Consts<T>& c = consts<T>(p);
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if (!((cx(a) == 1 && x == 0) || (cx(a) == -1 && x == p.nx - 1))) continue;
    int as = a, ys = y - cy(a);
    if (ys < 0 || ys >= p.ny) {
      if (p.bc_y == kBcPeriodic) {
        ys = ys < 0 ? ys + p.ny : ys - p.ny;
      } else {
        as = mirror_y(a);
        ys = y;
      }
    }
    if (cx(a) == 1) {
      h[a] = ESP ? c.heq_in[as] - sref<S>(p, a) : c.heq_in[as];
    } else if (p.bc_x == kBcInletConvective) {
      const long long gi = (long long)(as == 3 ? 0 : (as == 6 ? 1 : 2)) * p.ny + ys;
      const T f_last = ESP ? h[a] + sref<S>(p, a) : h[a];
      const T g = (static_cast<const T*>(p.ghost_src)[gi] + c.u_conv * f_last) * c.conv_inv;
      if (write) static_cast<T*>(p.ghost_dst)[gi] = g;
      h[a] = ESP ? g - sref<S>(p, a) : g;
    }
  }
}

// f*_a(x, y) as stored, whatever the scheme and phase (for the diagnostics:
// export, momentum exchange, outlet state).
template <class S>
__device__ __forceinline__ typename S::E fstar_e(const StepParams& p, const typename S::E* buf, int a,
                                                 int x, int y) {
  if (p.mode == kModeAB) return buf[(long long)a * p.plane + (long long)y * p.pitch + x];
  if (p.mode == kModeAAPush)  // after a local step: the node's opposite slot
    return buf[(long long)opposite(a) * p.plane + (long long)y * p.pitch + x];
  int ap, xt, yt;  // after a push step: where it was pushed
  if (push_target(p, a, x, y, &ap, &xt, &yt))
    return buf[(long long)ap * p.plane + (long long)yt * p.pitch + xt];
  return static_cast<const typename S::E*>(p.lost)[lost_index(p, a, y, x + cx(a) < 0)];
}

// MODE: kModeAB (pull from p.src, store to p.dst), or one of the two in-place
// AA steps on the one buffer p.dst (== p.src).
template <int STORE, int COLL, int MODE = kModeAB>
__device__ __forceinline__ void step_tile(const StepParams& p, int tile, long long t) {
  using S = Store<STORE>;
  using T = typename S::T;
  using E = typename S::E;
  constexpr int N = npt(STORE);
  constexpr int TX = kLanes * N;
  constexpr int W = warps_per_block(STORE);
  __shared__ double sm[W][3];
  __shared__ T smass[W];

  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tx = tile % p.tiles_x;
  const int ty = tile / p.tiles_x;
  const int x0 = tx * TX, y0 = ty * p.tile_y;
  const int xb = x0 + lane * N;
  const bool interior = x0 >= 1 && x0 + TX <= p.nx - 1 && y0 >= 1 && y0 + p.tile_y <= p.ny - 1;
  const E* __restrict__ src = static_cast<const E*>(p.src);
  E* __restrict__ dst = static_cast<E*>(p.dst);
  E* buf = static_cast<E*>(p.dst);  // the in-place modes' one buffer (not restrict: read and written)

  T dm = T(0);           // sum of drho over this thread's nodes
  T tfx = T(0), tfy = T(0);  // force on this thread's solid nodes (<= 16, arithmetic type)
  bool any_solid = false;
  const unsigned key = round_bits(unsigned(t), p.round_key);

  auto finish_node = [&](const Macro<T>& q, uint8_t m) {
    // a NaN or infinite population makes rho NaN, infinite or non-positive
    if (!(q.rho > T(0) && q.rho < T(1e30))) atomicOr(p.flag, 1);
    dm += q.drho;
    if (m) {
      any_solid = true;
      tfx -= q.fpx;
      tfy -= q.fpy;
    }
  };

  // Collide and store one row of pulled populations (lane_active: the lane's
  // first node lies in the domain).
  auto process_row = [&](int y, auto& h, auto gen) {
    constexpr bool GEN = decltype(gen)::value;
    const long long i = (long long)y * p.pitch + xb;
    // the N mask bytes of this lane's nodes, byte k for node k (kept in one
    // register: the collision's registers are the kernel's tightest budget)
    const unsigned mw = N == 4 ? *reinterpret_cast<const unsigned*>(p.mask + i)
                               : unsigned(*reinterpret_cast<const unsigned short*>(p.mask + i));
    auto mk = [&](int k) -> uint8_t { return uint8_t(mw >> (8 * k)); };
    const bool sr = S::kSixteen && p.stochastic;
    constexpr bool REF = S::kSixteen;  // h holds elements e = h - h_ref
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (GEN && xb + k >= p.nx) continue;  // past the last column: padding, stored as pulled
      if (COLL == kTrt && !GEN && p.force_free && mk(k) == 0) {
        // a fluid node without body force: the force-free form of the step
        const Macro<T> q = macros<T, true, REF>(p, h[k], 0, xb + k, y);
        collide_trt<T, true, REF>(p, h[k], q);
        finish_node(q, 0);
      } else if (COLL == kTrt) {
        const Macro<T> q = macros<T, false, REF>(p, h[k], mk(k), xb + k, y);
        collide_trt<T, false, REF>(p, h[k], q);
        finish_node(q, mk(k));
      } else {
        // the moment-space form works on offsets
        if constexpr (REF) {
#pragma unroll
          for (int a = 0; a < 9; ++a) h[k][a] = h[k][a] + sref<S>(p, a);
        }
        const Macro<T> q = macros<T>(p, h[k], mk(k), xb + k, y);
        collide_mrt<T>(p, h[k], q);
        finish_node(q, mk(k));
        if constexpr (REF) {
#pragma unroll
          for (int a = 0; a < 9; ++a) h[k][a] = h[k][a] - sref<S>(p, a);
        }
      }
    }
    // the rounding word of each of the lane's node pairs (16-bit stores):
    // pairs (xb, xb + 1), (xb + 2, xb + 3) are numbered row by row
    unsigned nb[(N + 1) / 2];
#pragma unroll
    for (int j = 0; j < (N + 1) / 2; ++j)
      nb[j] = sr ? round_bits(unsigned((long long)y * ((p.nx + 1) >> 1) + (xb >> 1) + j), key) : 0u;
    if constexpr (MODE == kModeAB) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        T o[N];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = h[k][a];
        S::store_h(dst + (long long)a * p.plane + i, o, a, nb, sr);
      }
    } else if constexpr (MODE == kModeAALocal) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        T o[N];
#pragma unroll
        for (int k = 0; k < N; ++k) o[k] = h[k][a];
        S::store_h(buf + (long long)opposite(a) * p.plane + i, o, a, nb, sr);
      }
      if (GEN && p.bc_x != kBcPeriodic) {
        // the outlet column's stored f* of alpha = 3, 6, 7, for the next push step
#pragma unroll
        for (int k = 0; k < N; ++k) {
          if (xb + k != p.nx - 1) continue;
          typename S::R* z = static_cast<typename S::R*>(p.z);
          z[0 * p.ny + y] = S::round_e(h[k][3], 3, nb[k >> 1], k, sr);
          z[1 * p.ny + y] = S::round_e(h[k][6], 6, nb[k >> 1], k, sr);
          z[2 * p.ny + y] = S::round_e(h[k][7], 7, nb[k >> 1], k, sr);
        }
      }
    } else {  // push step
      // vector pushes wherever every target of the row lies in the grid: all
      // of an interior tile, and the rows of a boundary tile that touches
      // neither x side nor the first or last row (warp-uniform)
      const bool vec = !GEN || (x0 >= 1 && x0 + TX <= p.nx - 1 && y >= 1 && y <= p.ny - 2);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        typename S::R e[N];
#pragma unroll
        for (int k = 0; k < N; ++k) e[k] = S::round_e(h[k][a], a, nb[k >> 1], k, sr);
        if (vec) {
          push_dir_vec<S, N>(p, buf, a, xb, y, lane, e);
        } else {
#pragma unroll
          for (int k = 0; k < N; ++k)
            if (xb + k < p.nx) push_one<S>(p, buf, a, xb + k, y, e[k]);
        }
      }
      if (GEN && p.bc_x != kBcPeriodic) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
          if (xb + k != p.nx - 1) continue;
          push_outlet_copy<S>(p, buf, 3, y, S::round_e(h[k][3], 3, nb[k >> 1], k, sr));
          push_outlet_copy<S>(p, buf, 6, y, S::round_e(h[k][6], 6, nb[k >> 1], k, sr));
          push_outlet_copy<S>(p, buf, 7, y, S::round_e(h[k][7], 7, nb[k >> 1], k, sr));
        }
      }
    }
  };

  auto do_row = [&](int y, auto gen) {
    constexpr bool GEN = decltype(gen)::value;
    const bool lane_active = !GEN || xb < p.nx;
    T h[N][9];
    if constexpr (MODE == kModeAALocal) {
      if (!lane_active) return;
      const long long i = (long long)y * p.pitch + xb;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        T v[N];
        S::load_h_plain(buf + (long long)a * p.plane + i, v, a);
#pragma unroll
        for (int k = 0; k < N; ++k) h[k][a] = v[k];
      }
      if (GEN) {
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (xb + k < p.nx) aa_local_boundary<S, true>(p, h[k], xb + k, y, true);
      }
    } else {
      constexpr bool AA = MODE == kModeAAPush;
      const E* from = AA ? buf : src;
      pull_dir_vec<S, N, 0, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 1, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 2, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 3, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 4, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 5, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 6, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 7, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      pull_dir_vec<S, N, 8, GEN, AA>(p, from, xb, y, lane, lane_active, h);
      if (!lane_active) return;
    }
    process_row(y, h, gen);
  };

  if (interior) {
#pragma unroll 1
    for (int r = 0; r < p.rows_per_warp; ++r) do_row(y0 + warp + r * W, std::false_type());
  } else {
#pragma unroll 1
    for (int r = 0; r < p.rows_per_warp; ++r) {
      const int y = y0 + warp + r * W;
      if (y >= p.ny) break;  // warp-uniform: a warp is one row
      do_row(y, std::true_type());
    }
  }

  // Per-step record: the force on the solid nodes, summed per thread in the
  // arithmetic type (each thread holds at most 16 nodes) and in FP64 from the
  // thread up; the total density, in the arithmetic type within the block and
  // FP64 from the tile up. Warps and blocks without solid nodes skip the FP64
  // work (on GB300 FP64 runs at a small fraction of the FP32 rate).
  const int tid = lane + warp * kLanes;
  const bool warp_solid = __any_sync(0xffffffffu, any_solid);
  double bfx = 0.0, bfy = 0.0;
  if (warp_solid) {
    bfx = double(tfx);
    bfy = double(tfy);
  }
  if (p.reduce_mass) dm = warp_sum(dm);
  if (warp_solid) {
    bfx = warp_sum(bfx);
    bfy = warp_sum(bfy);
  }
  if (lane == 0) {
    smass[warp] = dm;
    sm[warp][0] = bfx;
    sm[warp][1] = bfy;
  }
  const int block_solid = __syncthreads_or(any_solid);
  double ts[3] = {0.0, 0.0, 0.0};
  if (tid == 0) {
    T msum = T(0);
#pragma unroll
    for (int w = 0; w < W; ++w) msum += smass[w];
    if (block_solid) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        ts[0] += sm[w][0];
        ts[1] += sm[w][1];
      }
    }
    if (p.reduce_mass) {
      // sum rho = active nodes + sum drho
      const int nact = min(TX, p.nx - x0) * min(p.tile_y, p.ny - y0);
      ts[2] = double(nact) + double(msum);
    }
  }
  __syncthreads();
  finish_reduction<threads_per_block(STORE)>(p, tile, t, ts, sm);
}

template <int STORE, int COLL, int MODE = kModeAB>
__global__ void __launch_bounds__(threads_per_block(STORE), min_blocks_per_sm(STORE))
    fused_step_kernel(const __grid_constant__ StepParams p) {
  step_tile<STORE, COLL, MODE>(p, blockIdx.x, p.t);
}

// Grouped launch for serving: block b runs tile table[b].tile of solver
// table[b].solver at that solver's k-th step of the batch. Each solver has two
// parameter sets in a device array, for even and odd k (source and destination
// buffers swapped); params[].t is the solver's step index at k = 0. The block
// copies its solver's parameters to shared memory first (they are read many
// times per node), and takes the collision operator from them, so one launch
// covers SRT and MRT solvers of one storage type. MODE: the streaming step of
// every solver in the launch (in-place solvers are grouped by phase).
template <int STORE, int MODE = kModeAB>
__global__ void __launch_bounds__(threads_per_block(STORE), min_blocks_per_sm(STORE))
    fused_group_kernel(const StepParams* __restrict__ params, const GroupTile* __restrict__ table,
                       long long k) {
  __shared__ StepParams sp;
  const GroupTile gt = table[blockIdx.x];
  const StepParams* g = params + 2 * gt.solver + int(k & 1);
  {
    static_assert(sizeof(StepParams) % sizeof(int) == 0, "StepParams is copied in 4-byte words");
    const int* from = reinterpret_cast<const int*>(g);
    int* to = reinterpret_cast<int*>(&sp);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    for (int w = tid; w < int(sizeof(StepParams) / sizeof(int)); w += threads_per_block(STORE))
      to[w] = __ldg(from + w);
  }
  __syncthreads();
  if (sp.collision == kTrt)
    step_tile<STORE, kTrt, MODE>(sp, gt.tile, sp.t + k);
  else
    step_tile<STORE, kMrt, MODE>(sp, gt.tile, sp.t + k);
}

// ---------------------------------------------------------------------------
// Moments: the density and implicit velocity the next step computes.
// ---------------------------------------------------------------------------
// The populations the next step pulls, in any scheme and phase (read only:
// the caller's parameters carry no ghost_dst).
template <class S, int A>
__device__ __forceinline__ typename S::T pull_aa(const StepParams& p, const typename S::E* buf, int x,
                                                 int y) {
  int as = A, ys = y - cy(A);
  if (ys < 0 || ys >= p.ny) {
    if (p.bc_y == kBcPeriodic) {
      ys = ys < 0 ? ys + p.ny : ys - p.ny;
    } else {
      as = mirror_y(A);
      ys = y;
    }
  }
  return edge_pull<S, A, true>(p, buf, as, ys, x - cx(A));
}
template <class S>
__device__ __forceinline__ void pull_node_any(const StepParams& p, int x, int y, typename S::T h[9]) {
  const typename S::E* buf = static_cast<const typename S::E*>(p.src);
  if (p.mode == kModeAB) {
    pull_node<S>(p, buf, x, y, h);
  } else if (p.mode == kModeAALocal) {
#pragma unroll
    for (int a = 0; a < 9; ++a)
      h[a] = S::in(buf[(long long)a * p.plane + (long long)y * p.pitch + x], a, sref<S>(p, a));
    aa_local_boundary<S>(p, h, x, y, false);
  } else {
    h[0] = pull_aa<S, 0>(p, buf, x, y);
    h[1] = pull_aa<S, 1>(p, buf, x, y);
    h[2] = pull_aa<S, 2>(p, buf, x, y);
    h[3] = pull_aa<S, 3>(p, buf, x, y);
    h[4] = pull_aa<S, 4>(p, buf, x, y);
    h[5] = pull_aa<S, 5>(p, buf, x, y);
    h[6] = pull_aa<S, 6>(p, buf, x, y);
    h[7] = pull_aa<S, 7>(p, buf, x, y);
    h[8] = pull_aa<S, 8>(p, buf, x, y);
  }
}

template <int STORE>
__global__ void moments_kernel(const __grid_constant__ StepParams p, double* rho, double* ux,
                               double* uy) {
  using S = Store<STORE>;
  using T = typename S::T;
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  T h[9];
  pull_node_any<S>(p, x, y, h);
  const uint8_t m = p.mask[(long long)y * p.pitch + x];
  const Macro<T> q = macros<T>(p, h, m, x, y);
  const long long o = (long long)y * p.nx + x;
  rho[o] = double(q.rho);
  ux[o] = double(q.ux);
  uy[o] = double(q.uy);
}

// ---------------------------------------------------------------------------
// Momentum exchange (Section 3.3, after Ladd). Over every link from a fluid
// node x_f to a solid node x_s = x_f + xi_a the momentum
// xi_a [f*_a(x_f) + f*_abar(x_s)] of the store f*(t) crosses into the solid.
// Threads take the solid nodes of the box and look back along each direction
// for a fluid node; a link whose start lies outside a non-periodic side does
// not exist. The grid is fixed (kMeBlocks) and each thread walks its nodes
// grid-stride, so the share of each thread depends on the box alone; sums are
// FP64 in fixed order (thread, warp, block, then the last block to finish
// adds the block partials in block order).
// ---------------------------------------------------------------------------
template <int STORE>
__global__ void __launch_bounds__(kThreads)
    momentum_exchange_kernel(const __grid_constant__ StepParams p, const MeArgs m) {
  using S = Store<STORE>;
  using E = typename S::E;
  __shared__ double sm[kThreads / 32][3];
  __shared__ int s_last;
  const E* src = static_cast<const E*>(p.src);
  int x0 = m.x0, y0 = m.y0, x1 = m.x1, y1 = m.y1;
  {
    const int sx0 = m.static_box[0], sy0 = m.static_box[1];
    const int sx1 = m.static_box[2], sy1 = m.static_box[3];
    if (sx1 >= sx0 && sy1 >= sy0) {
      if (x1 < x0 || y1 < y0) {
        x0 = sx0, y0 = sy0, x1 = sx1, y1 = sy1;
      } else {
        x0 = min(x0, sx0), y0 = min(y0, sy0), x1 = max(x1, sx1), y1 = max(y1, sy1);
      }
    }
  }
  double fx = 0.0, fy = 0.0;
  if (x1 >= x0 && y1 >= y0) {
    const int w = x1 - x0 + 1;
    const long long n = (long long)w * (y1 - y0 + 1);
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads) {
      const int x = x0 + int(i % w), y = y0 + int(i / w);
      if (p.mask[(long long)y * p.pitch + x] == 0) continue;
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        int xf = x - cx(a), yf = y - cy(a);
        if (xf < 0 || xf >= p.nx) {
          if (p.bc_x != kBcPeriodic) continue;
          xf = xf < 0 ? xf + p.nx : xf - p.nx;
        }
        if (yf < 0 || yf >= p.ny) {
          if (p.bc_y != kBcPeriodic) continue;
          yf = yf < 0 ? yf + p.ny : yf - p.ny;
        }
        if (p.mask[(long long)yf * p.pitch + xf] != 0) continue;
        const int o = opposite(a);
        const E ef = fstar_e<S>(p, src, a, xf, yf), es = fstar_e<S>(p, src, o, x, y);
        const double flow = S::to_f64(&ef, a, sref<S>(p, a)) + S::to_f64(&es, o, sref<S>(p, o));
        fx += double(cx(a)) * flow;
        fy += double(cy(a)) * flow;
      }
    }
  }
  double v[3] = {fx, fy, 0.0};
  block_sum3(v, sm);
  if (threadIdx.x == 0) {
    __stcg(m.partials + 2 * blockIdx.x + 0, v[0]);
    __stcg(m.partials + 2 * blockIdx.x + 1, v[1]);
    __threadfence();
    s_last = atomicAdd(m.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double u[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
    u[0] += __ldcg(m.partials + 2 * b + 0);
    u[1] += __ldcg(m.partials + 2 * b + 1);
  }
  block_sum3(u, sm);
  if (threadIdx.x == 0) {
    m.out[0] = u[0];
    m.out[1] = u[1];
    *m.counter = 0u;
  }
}

// f*(t) := f_eq(rho0, u(x)), u from a device [2][ny][nx] array or uniform.
template <int STORE>
__global__ void init_kernel(const __grid_constant__ StepParams p, void* dst, const double* u,
                            double rho0, double u0x, double u0y) {
  using S = Store<STORE>;
  using T = typename S::T;
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long o = (long long)y * p.nx + x;
  const long long nn = (long long)p.nx * p.ny;
  const T ux = T(u ? u[o] : u0x), uy = T(u ? u[nn + o] : u0y), rho = T(rho0);
  const T drho = rho - T(1);
  const T common = drho - T(1.5) * rho * (ux * ux + uy * uy);
  typename S::E* d = static_cast<typename S::E*>(dst);
  const long long i = (long long)y * p.pitch + x;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const T xu = T(cx(a)) * ux + T(cy(a)) * uy;
    const T heq = wgt<T>(a) * (common + rho * xu * (T(3) + T(4.5) * xu));
    // in place (AA), a state before a push step keeps f*_a in the opposite slot
    const int slot = p.mode == kModeAB ? a : opposite(a);
    store_h<S>(p, d + (long long)slot * p.plane + i, heq, a);
  }
}

// Convective outlet state g := the offsets of the last column of the store
// (a zero-gradient start), [3][ny] rows alpha = 3, 6, 7.
// In place (AA), also the side copy z of those stored values (either output
// may be null).
template <int STORE>
__global__ void ghost_init_kernel(const __grid_constant__ StepParams p, const void* srcv, void* ghostv,
                                  void* zv) {
  using S = Store<STORE>;
  using T = typename S::T;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * p.ny) return;
  const int k = i / p.ny, y = i - k * p.ny;
  const int a = k == 0 ? 3 : (k == 1 ? 6 : 7);
  const typename S::E e = fstar_e<S>(p, static_cast<const typename S::E*>(srcv), a, p.nx - 1, y);
  if (ghostv) static_cast<T*>(ghostv)[i] = S::in(e, a, sref<S>(p, a));
  if (zv) static_cast<typename S::E*>(zv)[i] = e;
}

// Store <-> dense FP64 [9][ny][nx].
template <int STORE>
__global__ void export_kernel(const __grid_constant__ StepParams p, const void* srcv, double* f) {
  using S = Store<STORE>;
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const typename S::E* src = static_cast<const typename S::E*>(srcv);
  const long long i = (long long)y * p.pitch + x;
  const long long o = (long long)y * p.nx + x;
  const long long nn = (long long)p.nx * p.ny;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const typename S::E e = fstar_e<S>(p, src, a, x, y);
    f[a * nn + o] = S::to_f64(&e, a, sref<S>(p, a));
  }
  (void)i;
}

template <int STORE>
__global__ void import_kernel(const __grid_constant__ StepParams p, void* dstv, const double* f) {
  using S = Store<STORE>;
  const int x = blockIdx.x * kBlockX + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  typename S::E* dst = static_cast<typename S::E*>(dstv);
  const long long i = (long long)y * p.pitch + x;
  const long long o = (long long)y * p.nx + x;
  const long long nn = (long long)p.nx * p.ny;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int slot = p.mode == kModeAB ? a : opposite(a);  // in place: before a push step
    S::from_f64(dst + slot * p.plane + i, f[a * nn + o], a, sref<S>(p, a));
  }
}

}  // namespace vplbm
