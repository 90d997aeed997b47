// lattice.cuh -- velocity sets, model weights and storage formats of the CUDA path.
//
// Coordinates inside the kernels are (a, b, m): a = x (contiguous in memory), b = y for D3Q19
// (absent for D2Q9), m = the axis the kernels march along (z for D3Q19, y for D2Q9).
//
// Weights (paper Sec. II.A defers them to Leclaire et al. 2017; standard values of that model):
//   W_i  isotropic lattice weights, c_s^2 = 1/3;
//   A_i + B_i alpha = phi_i(alpha), the rest state of a component with free parameter alpha
//                     (f_i^eq(rho, 0) = rho phi_i(abar), Eq. feq);
//   C_i  the constants of the perturbation operator, Eq. (perturb).
// Opposite directions are adjacent pairs (1,2), (3,4), ..., so opp(i) = i + 1 - 2 ((i-1) & 1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cgevap {

template <int Q>
struct Lattice;

template <>
struct Lattice<9> {
  static constexpr int Q = 9;
  static constexpr bool D3 = false;
  // (x, y) of D2Q9 mapped to (a, b, m) = (x, -, y)
  __host__ __device__ static constexpr int ca(int i) {
    constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int cb(int) { return 0; }
  __host__ __device__ static constexpr int cm(int i) {
    constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int speed2(int i) { return i == 0 ? 0 : (i < 5 ? 1 : 2); }
  __host__ __device__ static constexpr double W(int i) {
    return speed2(i) == 0 ? 4.0 / 9.0 : (speed2(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr double A(int i) {
    return speed2(i) == 0 ? 0.0 : (speed2(i) == 1 ? 1.0 / 5.0 : 1.0 / 20.0);
  }
  __host__ __device__ static constexpr double B(int i) {
    return speed2(i) == 0 ? 1.0 : (speed2(i) == 1 ? -1.0 / 5.0 : -1.0 / 20.0);
  }
  __host__ __device__ static constexpr double C(int i) {
    return speed2(i) == 0 ? -4.0 / 27.0 : (speed2(i) == 1 ? 2.0 / 27.0 : 5.0 / 108.0);
  }
};

template <>
struct Lattice<19> {
  static constexpr int Q = 19;
  static constexpr bool D3 = true;
  __host__ __device__ static constexpr int ca(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
  }
  __host__ __device__ static constexpr int cb(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int cm(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int speed2(int i) { return i == 0 ? 0 : (i < 7 ? 1 : 2); }
  __host__ __device__ static constexpr double W(int i) {
    return speed2(i) == 0 ? 1.0 / 3.0 : (speed2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr double A(int i) {
    return speed2(i) == 0 ? 0.0 : (speed2(i) == 1 ? 1.0 / 12.0 : 1.0 / 24.0);
  }
  __host__ __device__ static constexpr double B(int i) {
    return speed2(i) == 0 ? 1.0 : (speed2(i) == 1 ? -1.0 / 12.0 : -1.0 / 24.0);
  }
  __host__ __device__ static constexpr double C(int i) {
    return speed2(i) == 0 ? -1.0 / 3.0 : (speed2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// True when every odd direction i has its opposite at i + 1 (checked where code relies on it).
template <class L>
__host__ __device__ constexpr bool opposites_adjacent() {
  for (int i = 1; i + 1 < L::Q; i += 2)
    if (L::ca(i + 1) != -L::ca(i) || L::cb(i + 1) != -L::cb(i) || L::cm(i + 1) != -L::cm(i))
      return false;
  return (L::Q & 1) == 1;
}

// 1/|c_i| for the recoloring angle (0 for the rest direction, whose cos is defined as 0).
template <class L>
__host__ __device__ constexpr double inv_norm(int i) {
  return L::speed2(i) == 0 ? 0.0 : (L::speed2(i) == 1 ? 1.0 : 0.70710678118654752440);
}

// Bit masks of the directions whose pull source x - c_i lies on the low / high side of an axis.
template <class L>
__host__ __device__ constexpr uint32_t dirs_where(int axis, int sign) {
  uint32_t m = 0;
  for (int i = 0; i < L::Q; ++i) {
    int c = axis == 0 ? L::ca(i) : (axis == 1 ? L::cb(i) : L::cm(i));
    if (c == sign) m |= 1u << i;
  }
  return m;
}

// ---------------------------------------------------------------- storage formats ----------
//
// ST_F64 / ST_F32: vec2 pops[i][cell] = (f_i^r, f_i^b).  The two components of a direction share
//   one aligned 16- / 8-byte load, so a pull is Q vector loads per cell.
// ST_F16 / ST_BF16 ("deviation" storage): float2 rest[cell] = (f_0^r, f_0^b) in FP32 and, for
//   i >= 1, a packed pair dev[i-1][cell] = s (f_i^k - f_0^k kappa_i^k) in FP16 / BF16, where
//   kappa_i^k = phi_i(alpha_k) / phi_0(alpha_k) is the ratio of the rest state of component k,
//   so bulk cells at rest store deviations near 0; s is a power of two (FP16 only) that keeps
//   small deviations out of the subnormal range.  Decoding multiplies by 1/s exactly.
// ST_RC ("recolour on pull"): float pops[i][cell] = the colour-blind post-collision population
//   f_i, and one float4 rec[cell] = (w_r, V) after the Q planes, from which either colour of any
//   direction follows exactly as Eq. (recolor) forms it:
//     f_i^r = w_r f_i + s_|c_i| (c_i . V),   f_i^b = f_i - f_i^r,
//   w_r = rho_r / rho, V = beta (rho_r rho_b / rho) (1 - abar) F / |F| and s = A_s / |c| for the
//   speed class s (phi_i(abar) = A_s (1 - abar) for i >= 1), 0 for the rest direction.  Q + 4
//   floats per cell instead of 2Q.  Arbitrary population pairs (an initial state with noise,
//   an import) are not of this form: those are held as FP32 pairs and the first step reads them
//   with ST_RCI (pairs in, ST_RC out).
// ST_H16RC / ST_B16RC ("recolour on pull, 16-bit"): the colour-blind populations of ST_RC held as
//   FP16 / BF16 deviations from the lattice-weight rest state of the cell, with each colour's
//   mass carried exactly.  Per cell, in four arrays (offsets in Rc16Layout):
//     float2 rest[cell] = (f_0^r, f_0^b)        the rest populations of both colours (FP32),
//     float4 rec[cell]  = (w_r, V)              as ST_RC,
//     float  ref[cell]  = Rf                    the rest-state scale, Rf = A_1 rho (1 - abar),
//     P      dev[i-1][cell] = s (f_i - r_i Rf)  i >= 1, FP16 / BF16, r_i = A_i / A_1,
//   so f_i^eq(rho, 0) = rho phi_i(abar) = r_i Rf and a cell at rest stores deviations near 0.  A
//   reader decodes f_i = fl(r_i Rf + dev / s) (r_i is 1 or a power of two: one rounding) and
//   splits it as ST_RC does: f_i^r = fl(w_r f_i + s_|c| (c_i . V)), f_i^b = fl(f_i - f_i^r).  The
//   writer forms those same values and sets the rest pair to the exact colour masses minus what
//   the moving populations will deliver, so the mass of each colour a cell stores is its exact
//   post-exchange mass up to the rounding of the rest pair.  ST_H16RCI / ST_B16RCI: the same
//   step reading FP32 pairs (an imported state).
// ST_F32X: the FP32 pairs of ST_F32 with each colour's mass carried exactly through the step:
//   the pulled pairs are summed per colour with Fast2Sum, the exchange's rounding is kept by
//   TwoSum, and the rest pair is stored last as the exact post-exchange colour masses less the
//   stored moving pairs, so the mass of each colour a cell passes on equals its exact mass up
//   to one rounding of the rest pair (the FP32 arithmetic of the collision is otherwise that of
//   ST_F32).
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3, ST_RC = 4, ST_RCI = 5, ST_H16RC = 6,
       ST_B16RC = 7, ST_H16RCI = 8, ST_B16RCI = 9, ST_F32X = 10 };

// Traits of a storage code: dev = per-colour 16-bit deviations; rc = writes a recolour-on-pull
// layout; rc16 = that layout is the 16-bit one; rc_in = reads a recolour-on-pull layout (the
// pulls need the sources' records, staged in shared memory).
template <int S>
struct Storage;
template <>
struct Storage<ST_F64> {
  using real = double;
  using vec = double2;
  static constexpr bool dev = false, rc = false, rc16 = false, rc_in = false;
  static constexpr int bytes_per_pop = 8;
};
template <>
struct Storage<ST_F32> {
  using real = float;
  using vec = float2;
  static constexpr bool dev = false, rc = false, rc16 = false, rc_in = false;
  static constexpr int bytes_per_pop = 4;
};
template <>
struct Storage<ST_RC> {  // reads and writes the recolour-on-pull layout
  using real = float;
  using vec = float2;
  static constexpr bool dev = false, rc = true, rc16 = false, rc_in = true;
  static constexpr int bytes_per_pop = 4;
};
template <>
struct Storage<ST_RCI> {  // reads FP32 pairs, writes the recolour-on-pull layout
  using real = float;
  using vec = float2;
  static constexpr bool dev = false, rc = true, rc16 = false, rc_in = false;
  static constexpr int bytes_per_pop = 4;
};
template <>
struct Storage<ST_F16> {
  using real = float;
  using packed = __half2;
  static constexpr bool dev = true, rc = false, rc16 = false, rc_in = false;
  static constexpr int bytes_per_pop = 2;
  static __device__ __forceinline__ float2 unpack(packed p) { return __half22float2(p); }
  static __device__ __forceinline__ packed pack(float r, float b) { return __floats2half2_rn(r, b); }
};
template <>
struct Storage<ST_BF16> {
  using real = float;
  using packed = __nv_bfloat162;
  static constexpr bool dev = true, rc = false, rc16 = false, rc_in = false;
  static constexpr int bytes_per_pop = 2;
  static __device__ __forceinline__ float2 unpack(packed p) { return __bfloat1622float2(p); }
  static __device__ __forceinline__ packed pack(float r, float b) {
    return __floats2bfloat162_rn(r, b);
  }
};
// 16-bit recolour-on-pull: one 16-bit value per moving population
struct Half16 {
  using packed = __half;
  static __device__ __forceinline__ float unpack(packed p) { return __half2float(p); }
  static __device__ __forceinline__ packed pack(float v) { return __float2half_rn(v); }
  // the raw 16 bits, in and out of a register without going through memory
  static __device__ __forceinline__ float unpack_bits(unsigned short u) {
    return __half2float(__ushort_as_half(u));
  }
};
struct BHalf16 {
  using packed = __nv_bfloat16;
  static __device__ __forceinline__ float unpack(packed p) { return __bfloat162float(p); }
  static __device__ __forceinline__ packed pack(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float unpack_bits(unsigned short u) {
    return __bfloat162float(__ushort_as_bfloat16(u));
  }
};
template <class H, bool PAIRS_IN>
struct Rc16Storage {
  using real = float;
  using vec = float2;
  using half_t = H;
  static constexpr bool dev = false, rc = true, rc16 = true, rc_in = !PAIRS_IN;
  static constexpr int bytes_per_pop = 2;
};
template <>
struct Storage<ST_F32X> : Storage<ST_F32> {};
// Storages whose FP32 pairs carry each colour's mass exactly (ST_F32X).
template <int S>
struct ExactPairs {
  static constexpr bool value = false;
};
template <>
struct ExactPairs<ST_F32X> {
  static constexpr bool value = true;
};
template <>
struct Storage<ST_H16RC> : Rc16Storage<Half16, false> {};
template <>
struct Storage<ST_B16RC> : Rc16Storage<BHalf16, false> {};
template <>
struct Storage<ST_H16RCI> : Rc16Storage<Half16, true> {};
template <>
struct Storage<ST_B16RCI> : Rc16Storage<BHalf16, true> {};

// Byte offset of the deviation block inside one state buffer of a deviation storage.
__host__ __device__ inline size_t dev_block_offset(long long nstore) {
  return ((size_t)nstore * sizeof(float2) + 255) & ~(size_t)255;
}

// Padded storage of a lattice (see Geom in common.cuh): pitch, rows per plane, elements per
// population array.  kOx = stored elements before x = 0 in each row (the last two are ghosts);
// 16 puts x = 0 of FP32 / rest pairs on a 128-byte line boundary.
constexpr int kOx = 16;
struct StoreShape {
  int pitch, rows;
  long long nstore;
};
__host__ inline StoreShape store_shape(int q, int nx, int ny, int nz) {
  StoreShape s;
  s.pitch = (nx + kOx + 2 + 15) & ~15;
  s.rows = q == 19 ? ny + 4 : 1;
  const long long planes = q == 19 ? nz : ny;
  s.nstore = planes * s.rows * (long long)s.pitch;
  return s;
}

// Byte offset of the recolouring records inside an ST_RC state buffer.
__host__ __device__ inline size_t rc_record_offset(int q, long long nstore) {
  return (size_t)q * nstore * sizeof(float);
}

// Recolouring factor s_|c| = A_s / |c| of ST_RC for direction i (0 for the rest direction).
template <class L>
__host__ __device__ constexpr double rc_factor(int i) {
  return L::speed2(i) == 0 ? 0.0 : L::A(i) * inv_norm<L>(i);
}

// Byte offsets of the arrays of a 16-bit recolour-on-pull state buffer (each 256-byte aligned):
// rest pairs at 0, records at rec, rest-state scales at ref, deviations at dev; total bytes.
struct Rc16Layout {
  size_t rec, ref, dev, total;
};
__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
__host__ __device__ inline Rc16Layout rc16_layout(int q, long long nstore) {
  Rc16Layout l;
  l.rec = align256((size_t)nstore * 8);
  l.ref = align256(l.rec + (size_t)nstore * 16);
  l.dev = align256(l.ref + (size_t)nstore * 4);
  l.total = l.dev + (size_t)(q - 1) * nstore * 2;
  return l;
}

// Ratio r_i = A_i / A_1 of the rest state of direction i >= 1 to that of an axis direction:
// 1 or a power of two (D3Q19 1/2, D2Q9 1/4), so r_i Rf is exact.
template <class L>
__host__ __device__ constexpr double rc16_ratio(int i) {
  return L::A(i) / L::A(1);
}

__host__ inline size_t state_bytes(int storage, int q, long long nstore) {
  switch (storage) {
    case ST_F64: return (size_t)q * nstore * sizeof(double2);
    case ST_F32:
    case ST_F32X:
    case ST_RC:  // room for the FP32 pairs of an imported state
    case ST_RCI: return (size_t)q * nstore * sizeof(float2);
    case ST_H16RC:
    case ST_B16RC:
    case ST_H16RCI:
    case ST_B16RCI: {  // room for the FP32 pairs of an imported state as well
      const size_t pairs = (size_t)q * nstore * sizeof(float2);
      const size_t own = rc16_layout(q, nstore).total;
      return pairs > own ? pairs : own;
    }
    default: return dev_block_offset(nstore) + (size_t)(q - 1) * nstore * 4;
  }
}

}  // namespace cgevap
