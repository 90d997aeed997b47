// aux_kernels.cu -- initial equilibrium, population import/export, macroscopic readout, the
// gradient-rule sites of a given state, solid links, the health check and the heated-substrate
// flux field.  One thread per cell (per column for the flux field); none of these is on the
// timed path of the constant-flux step.
#include "launch.h"

namespace cgevap {

namespace {

constexpr int kThreads = 256;

inline dim3 grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 64) b = 152LL * 64;
  if (b < 1) b = 1;
  return dim3((unsigned)b);
}

struct Coord {
  int a, b, m;
};

__device__ __forceinline__ Coord coord_of(const Geom& g, int cell) {
  Coord c;
  c.a = cell % g.na;
  int t = cell / g.na;
  c.b = t % g.nb;
  c.m = t / g.nb;
  return c;
}

// Index of (a,b,m) + d, or -1 beyond a wall.
__device__ __forceinline__ int neighbour(const Geom& g, Coord c, int da, int db, int dm) {
  int a = step_coord(c.a, da, g.na, g.per_a);
  int b = step_coord(c.b, db, g.nb, g.per_b);
  int m = step_coord(c.m, dm, g.nm, g.per_m);
  if (a < 0 || b < 0 || m < 0) return -1;
  return (m * g.nb + b) * g.na + a;
}

__device__ __forceinline__ bool cell_solid(const Geom& g, int cell) {
  return g.links && (__ldg(g.links + cell) >> 31);
}

// Stores the populations of a cell (compact index) at its storage index and periodic images.
template <int Q, int S>
__device__ __forceinline__ void store_cell(void* state, const Geom& g, int cell, const double (&fr)[Q],
                                           const double (&fb)[Q], const Physics& ph) {
  using R = typename Storage<S>::real;
  const Coord c = coord_of(g, cell);
  const Images im = images_of(g, c.a, c.b, c.m);
  V2<R> f0{(R)fr[0], (R)fb[0]};
#pragma unroll
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < im.n; ++j)
      PopIO<S, Q>::store(state, g.nstore, i, im.s[j], (R)fr[i], (R)fb[i], f0, ph);
}

template <int Q, int S>
__device__ __forceinline__ void load_cell(const void* state, const Geom& g, int cell, double (&fr)[Q],
                                          double (&fb)[Q], const Physics& ph) {
  const Coord c = coord_of(g, cell);
  const int si = sidx(g, c.a, c.b, c.m);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    auto v = PopIO<S, Q>::load(state, g.nstore, i, i, si, ph);
    fr[i] = (double)v.r;
    fb[i] = (double)v.b;
  }
}

__device__ __forceinline__ double read_any(const void* p, int dtype, size_t i) {
  return dtype == 0 ? reinterpret_cast<const double*>(p)[i] : (double)reinterpret_cast<const float*>(p)[i];
}
__device__ __forceinline__ void write_any(void* p, int dtype, size_t i, double v) {
  if (dtype == 0) reinterpret_cast<double*>(p)[i] = v;
  else reinterpret_cast<float*>(p)[i] = (float)v;
}

// f_i^k = rho_k phi_i(alpha_k) + noise (Eq. feq at u = 0).
template <int Q, int S>
__global__ void k_init_eq(Geom g, Physics ph, double rri, double rbi, const double* rhoN0,
                          const void* noise, int ndt, void* state) {
  using L = Lattice<Q>;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    double fr[Q], fb[Q];
    const bool solid = cell_solid(g, cell);
    const double rn = rhoN0[cell];
    const double rr = rri * (1.0 + rn) / 2.0, rb = rbi * (1.0 - rn) / 2.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (solid) {
        fr[i] = fb[i] = 0.0;
        continue;
      }
      fr[i] = rr * (L::A(i) + L::B(i) * ph.alpha_r);
      fb[i] = rb * (L::A(i) + L::B(i) * ph.alpha_b);
      if (noise) {
        fr[i] += read_any(noise, ndt, (size_t)i * g.ncell + cell);
        fb[i] += read_any(noise, ndt, (size_t)(Q + i) * g.ncell + cell);
      }
    }
    store_cell<Q, S>(state, g, cell, fr, fb, ph);
  }
}

template <int Q, int S>
__global__ void k_set_pops(Geom g, Physics ph, const void* in, int dt, void* state) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    double fr[Q], fb[Q];
    const bool solid = cell_solid(g, cell);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      fr[i] = solid ? 0.0 : read_any(in, dt, (size_t)i * g.ncell + cell);
      fb[i] = solid ? 0.0 : read_any(in, dt, (size_t)(Q + i) * g.ncell + cell);
    }
    store_cell<Q, S>(state, g, cell, fr, fb, ph);
  }
}

template <int Q, int S>
__global__ void k_get_pops(Geom g, Physics ph, const void* state, void* out, int dt) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    double fr[Q], fb[Q];
    load_cell<Q, S>(state, g, cell, fr, fb, ph);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      write_any(out, dt, (size_t)i * g.ncell + cell, fr[i]);
      write_any(out, dt, (size_t)(Q + i) * g.ncell + cell, fb[i]);
    }
  }
}

// rho_k, u, rho^N of the state (local sums; Sec. II.A).  u is [3][N] in (x, y, z) order.
template <int Q, int S>
__global__ void k_macros(Geom g, Physics ph, const void* state, double* rr_out, double* rb_out,
                         double* u_out, double* rn_out) {
  using L = Lattice<Q>;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    double fr[Q], fb[Q];
    load_cell<Q, S>(state, g, cell, fr, fb, ph);
    double rr = 0, rb = 0, ja = 0, jb = 0, jm = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      rr += fr[i];
      rb += fb[i];
      const double f = fr[i] + fb[i];
      ja += L::ca(i) * f;
      jb += L::cb(i) * f;
      jm += L::cm(i) * f;
    }
    const double rho = rr + rb;
    const bool solid = cell_solid(g, cell) || !(rho > 0.0);
    if (rr_out) rr_out[cell] = solid ? 0.0 : rr;
    if (rb_out) rb_out[cell] = solid ? 0.0 : rb;
    if (rn_out) rn_out[cell] = solid ? 0.0 : (rr - rb) / rho;
    if (u_out) {
      // (a, b, m) -> (x, y, z): 3D (x, y, z); 2D (x, -, y)
      const double ux = solid ? 0.0 : ja / rho;
      const double uy = solid ? 0.0 : (L::D3 ? jb : jm) / rho;
      const double uz = solid ? 0.0 : (L::D3 ? jm : 0.0) / rho;
      u_out[cell] = ux;
      u_out[(size_t)g.ncell + cell] = uy;
      u_out[2 * (size_t)g.ncell + cell] = uz;
    }
  }
}

// |F| of a state from its local rho^N (Eq. cg): sets bits 1 and 3 of the site byte.
template <int Q>
__global__ void k_grad_sites(Geom g, double threshold, const double* rn, uint8_t* mask) {
  using L = Lattice<Q>;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    if (cell_solid(g, cell)) {
      mask[cell] = 0;
      continue;
    }
    const Coord c = coord_of(g, cell);
    const double own = rn[cell];
    double Fa = 0, Fb = 0, Fm = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      int nb = neighbour(g, c, L::ca(i), L::cb(i), L::cm(i));
      if (nb >= 0 && cell_solid(g, nb)) nb = -1;
      const double v = 3.0 * L::W(i) * (nb < 0 ? own : rn[nb]);
      Fa += L::ca(i) * v;
      Fb += L::cb(i) * v;
      Fm += L::cm(i) * v;
    }
    const double Fn = sqrt(Fa * Fa + Fb * Fb + Fm * Fm);
    const double d = Fn - threshold;
    mask[cell] = (uint8_t)((d > 0 ? 2u : 0u) | (fabs(d) < 1e-6 ? 8u : 0u));
  }
}

template <int Q, int S>
__global__ void k_local_rn(Geom g, Physics ph, const void* state, double* rn) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    double fr[Q], fb[Q];
    load_cell<Q, S>(state, g, cell, fr, fb, ph);
    double rr = 0, rb = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      rr += fr[i];
      rb += fb[i];
    }
    rn[cell] = (rr + rb > 0.0) ? (rr - rb) / (rr + rb) : 0.0;
  }
}

// bit i: pull source x - c_i is solid or beyond a wall; bit 31: the cell is solid.
template <int Q>
__global__ void k_links(Geom g, const uint8_t* solid, uint32_t* links) {
  using L = Lattice<Q>;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    const Coord c = coord_of(g, cell);
    uint32_t w = solid[cell] ? (1u << 31) : 0u;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int s = neighbour(g, c, -L::ca(i), -L::cb(i), -L::cm(i));
      if (s < 0 || solid[s]) w |= 1u << i;
    }
    links[cell] = w;
  }
}

template <int Q, int S>
__global__ void k_zero_solid(Geom g, Physics ph, void* state) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    if (!cell_solid(g, cell)) continue;
    double z[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) z[i] = 0.0;
    store_cell<Q, S>(state, g, cell, z, z, ph);
  }
}

template <int Q, int S>
__global__ void k_health(Geom g, Physics ph, const void* state, int* flag) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    if (cell_solid(g, cell)) continue;
    double fr[Q], fb[Q];
    load_cell<Q, S>(state, g, cell, fr, fb, ph);
    double rho = 0.0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bad |= !isfinite(fr[i]) || !isfinite(fb[i]);
      rho += fr[i] + fb[i];
    }
    if (bad || !(rho > 0.0)) atomicOr(flag, 1);
  }
}

// Copy every cell within two of a periodic x / y edge into its ghost images (raw storage bits).
template <int Q, int S>
__global__ void k_fill_ghosts(Geom g, void* state) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += gridDim.x * blockDim.x) {
    const Coord c = coord_of(g, cell);
    const Images im = images_of(g, c.a, c.b, c.m);
    if (im.n < 2) continue;
    if constexpr (Storage<S>::rc) {
      float* pop = reinterpret_cast<float*>(state);
      float4* rec = reinterpret_cast<float4*>(reinterpret_cast<char*>(state) + rc_record_offset(Q, g.nstore));
      for (int j = 1; j < im.n; ++j) {
        rec[im.s[j]] = rec[im.s[0]];
        for (int i = 0; i < Q; ++i) pop[(size_t)i * g.nstore + im.s[j]] = pop[(size_t)i * g.nstore + im.s[0]];
      }
    } else if (Storage<S>::dev) {
      float2* rest = reinterpret_cast<float2*>(state);
      uint32_t* dev = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(state) + dev_block_offset(g.nstore));
      for (int j = 1; j < im.n; ++j) {
        rest[im.s[j]] = rest[im.s[0]];
        for (int i = 1; i < Q; ++i)
          dev[(size_t)(i - 1) * g.nstore + im.s[j]] = dev[(size_t)(i - 1) * g.nstore + im.s[0]];
      }
    } else {
      using Vec = typename Storage<(S == ST_F64 ? ST_F64 : ST_F32)>::vec;
      Vec* p = reinterpret_cast<Vec*>(state);
      for (int j = 1; j < im.n; ++j)
        for (int i = 0; i < Q; ++i) p[(size_t)i * g.nstore + im.s[j]] = p[(size_t)i * g.nstore + im.s[0]];
    }
  }
}

// Heated-substrate flux (Sec. III.C, Eq. heated), first pass: the liquid fraction
// rho_r / (rho_r + rho_b) summed over the fluid cells of planes [y*cz, y*cz + cz) of every column
// (a, b) along the march axis m (the wall normal), into part[chunk][column].  Threads run along a,
// so every population plane is read coalesced.  The cell's densities are summed in the storage's
// arithmetic (FP32 for FP32 and 16-bit storage, as in the step), the column in FP64.
template <int Q, int S>
__global__ void k_column_liquid(Geom g, Physics ph, const void* state, int cz, double* part) {
  using R = typename Storage<S>::real;
  const int ncol = g.na * g.nb;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const int a = col % g.na, b = col / g.na;
  const int m0 = blockIdx.y * cz;
  const int m1 = min(g.nm, m0 + cz);
  double h = 0.0;
  for (int m = m0; m < m1; ++m) {
    if (cell_solid(g, m * ncol + col)) continue;
    const int si = sidx(g, a, b, m);
    R rr = 0, rb = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const auto v = PopIO<S, Q>::load(state, g.nstore, i, i, si, ph);
      rr += v.r;
      rb += v.b;
    }
    if (rr + rb > R(0)) h += (double)(rr / (rr + rb));
  }
  part[(size_t)blockIdx.y * ncol + col] = h;
}

// Second pass, per column: h = the chunk partials summed in chunk order (deterministic) and the
// column's flux phi_s / (K + h / length), into row nchunk of part.
__global__ void k_heated_column(Geom g, double* part, int nchunk, double phi_s, double K,
                                double inv_length) {
  const int ncol = g.na * g.nb;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  double h = 0.0;
  for (int c = 0; c < nchunk; ++c) h += part[(size_t)c * ncol + col];
  part[(size_t)nchunk * ncol + col] = phi_s / (K + h * inv_length);
}

// Third pass: every cell of planes [y*cz, y*cz + cz) of the column takes the column's flux.
__global__ void k_heated_field(Geom g, const double* part, int nchunk, int cz, void* field,
                               int field_double) {
  const int ncol = g.na * g.nb;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const double v = part[(size_t)nchunk * ncol + col];
  const int m0 = blockIdx.y * cz;
  const int m1 = min(g.nm, m0 + cz);
  for (int m = m0; m < m1; ++m) write_any(field, field_double ? 0 : 1, (size_t)m * ncol + col, v);
}

__global__ void k_convert(const void* in, int in_dt, void* out, int out_double, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    write_any(out, out_double ? 0 : 1, (size_t)i, read_any(in, in_dt, (size_t)i));
}

// Writes the blue half of the population pair of direction `dir` (>= 1) at storage index si,
// leaving the red half's stored bits as they are.
template <int S>
__device__ __forceinline__ void store_blue(void* state, const Geom& g, const Physics& ph, int dir,
                                           int si, double v) {
  if constexpr (Storage<S>::rc) {
    return;  // not launched for this layout (launch_outlets refuses it)
  } else if constexpr (Storage<S>::dev) {
    using P = typename Storage<S>::packed;
    const float f0b = reinterpret_cast<const float2*>(state)[si].y;
    P* d = reinterpret_cast<P*>(reinterpret_cast<char*>(state) + dev_block_offset(g.nstore)) +
           (size_t)(dir - 1) * g.nstore + si;
    const float dv = __fmul_rn(__fmaf_rn(-f0b, ph.kap_b[dir], (float)v), ph.scale);
    P w = *d;
    w.y = Storage<S>::pack(0.0f, dv).y;
    *d = w;
  } else {
    using Vec = typename Storage<S>::vec;
    reinterpret_cast<Vec*>(state)[(size_t)dir * g.nstore + si].y = (typename Storage<S>::real)v;
  }
}

// Blue pressure outlet (Sec. III.B.2, the boundary condition of Zou and He), run before a step on
// the first (inward normal +m) and last (-m) plane of the march axis where a density is given.
// The step pulls the populations entering through the plane from beyond the wall, i.e. by
// halfway bounce-back from the cell's own slots of the opposite (leaving) directions.  This
// kernel rebuilds the blue ones from the cell's pulled known populations -- blue density rho0,
// no blue velocity along the plane:
//   rho0 u_n = rho0 - (S_0 + 2 S_out)        (mass and normal momentum; S over c.n = 0 / -1),
//   g_i = g_opp(i) + 6 W_i rho0 u_n - sum_t c_it N_t,   N_t = 1/2 sum_{c.n = 0} g_j c_jt
// (non-equilibrium bounce-back: only the odd part of Eq. feq differs between i and opp(i)) --
// and stores them in those leaving slots, so the step's bounce-back delivers them.  Red keeps
// its bounce-back: the outlet is a wall for red.  Leaving slots of a plane are read by no other
// cell, so the plane's cells are independent.
template <int Q, int S>
__global__ void k_outlet(Geom g, Physics ph, void* state, double rho_lo, double rho_hi) {
  using L = Lattice<Q>;
  using R = typename Storage<S>::real;  // the storage's arithmetic, as in the step
  const int ncol = g.na * g.nb;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * ncol; t += gridDim.x * blockDim.x) {
    const int side = t / ncol;
    const R rho0 = (R)(side ? rho_hi : rho_lo);
    if (!(rho0 > R(0))) continue;
    const int col = t - side * ncol;
    const int a = col % g.na, b = col / g.na, m = side ? g.nm - 1 : 0;
    const int cell = m * ncol + col;
    const uint32_t links = g.links ? __ldg(g.links + cell) : 0u;
    if (links >> 31) continue;  // a solid cell
    const int inward = side ? -1 : 1;
    const int si = sidx(g, a, b, m);
    R gb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int sa = step_coord(a, -L::ca(i), g.na, g.per_a);
      const int sb = step_coord(b, -L::cb(i), g.nb, g.per_b);
      const int sm = step_coord(m, -L::cm(i), g.nm, g.per_m);
      const bool bounce = sa < 0 || sb < 0 || sm < 0 || ((links >> i) & 1u);
      gb[i] = bounce ? PopIO<S, Q>::load(state, g.nstore, i, opp(i), si, ph).b
                     : PopIO<S, Q>::load(state, g.nstore, i, i, sidx(g, sa, sb, sm), ph).b;
    }
    R s0 = R(0), sout = R(0), ta = R(0), tb = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cn = L::cm(i) * inward;
      if (cn == 0) {
        s0 += gb[i];
        ta += R(L::ca(i)) * gb[i];
        tb += R(L::cb(i)) * gb[i];
      } else if (cn < 0) {
        sout += gb[i];
      }
    }
    const R un = R(1) - (s0 + R(2) * sout) / rho0;
    const Images im = images_of(g, a, b, m);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      if (L::cm(i) * inward <= 0) continue;
      const R v = gb[opp(i)] + R(6.0 * L::W(i)) * rho0 * un -
                  (R(L::ca(i)) * R(0.5) * ta + R(L::cb(i)) * R(0.5) * tb);
      for (int j = 0; j < im.n; ++j) store_blue<S>(state, g, ph, opp(i), im.s[j], (double)v);
    }
  }
}

__global__ void k_fill(double* out, double v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = v;
}

}  // namespace

#define CGEVAP_DISPATCH(A, KERNEL, GRID, STREAM, ...)                                            \
  do {                                                                                            \
    switch ((A).q * 10 + (A).storage) {                                                           \
      case 90: KERNEL<9, ST_F64><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;              \
      case 91: KERNEL<9, ST_F32><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;              \
      case 92: KERNEL<9, ST_F16><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;              \
      case 93: KERNEL<9, ST_BF16><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;             \
      case 190: KERNEL<19, ST_F64><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;            \
      case 191: KERNEL<19, ST_F32><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;            \
      case 192: KERNEL<19, ST_F16><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;            \
      case 193: KERNEL<19, ST_BF16><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;           \
      case 94: KERNEL<9, ST_RC><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;               \
      case 194: KERNEL<19, ST_RC><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;             \
      case 96: KERNEL<9, ST_H16RC><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;            \
      case 97: KERNEL<9, ST_B16RC><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;            \
      case 196: KERNEL<19, ST_H16RC><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;          \
      case 197: KERNEL<19, ST_B16RC><<<GRID, kThreads, 0, STREAM>>>(__VA_ARGS__); break;          \
      default: return cudaErrorInvalidValue;                                                      \
    }                                                                                             \
  } while (0)

cudaError_t launch_init_equilibrium(const AuxArgs& a, const double* rhoN0, const void* noise,
                                    int noise_dtype, void* state, cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_init_eq, grid_for(a.g.ncell), s, a.g, a.ph, a.rho_r_in, a.rho_b_in, rhoN0,
                  noise, noise_dtype, state);
  return cudaGetLastError();
}

cudaError_t launch_set_populations(const AuxArgs& a, const void* in, int dtype, void* state,
                                   cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_set_pops, grid_for(a.g.ncell), s, a.g, a.ph, in, dtype, state);
  return cudaGetLastError();
}

cudaError_t launch_get_populations(const AuxArgs& a, const void* state, void* out, int dtype,
                                   cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_get_pops, grid_for(a.g.ncell), s, a.g, a.ph, state, out, dtype);
  return cudaGetLastError();
}

cudaError_t launch_macros(const AuxArgs& a, const void* state, double* rho_r, double* rho_b,
                          double* u, double* rhoN, cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_macros, grid_for(a.g.ncell), s, a.g, a.ph, state, rho_r, rho_b, u, rhoN);
  return cudaGetLastError();
}

cudaError_t launch_gradient_sites(const AuxArgs& a, const void* state, double* tmp_rn,
                                  uint8_t* mask, cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_local_rn, grid_for(a.g.ncell), s, a.g, a.ph, state, tmp_rn);
  if (a.q == 19)
    k_grad_sites<19><<<grid_for(a.g.ncell), kThreads, 0, s>>>(a.g, a.ph.threshold, tmp_rn, mask);
  else
    k_grad_sites<9><<<grid_for(a.g.ncell), kThreads, 0, s>>>(a.g, a.ph.threshold, tmp_rn, mask);
  return cudaGetLastError();
}

cudaError_t launch_links(const AuxArgs& a, const uint8_t* solid, uint32_t* links, cudaStream_t s) {
  if (a.q == 19)
    k_links<19><<<grid_for(a.g.ncell), kThreads, 0, s>>>(a.g, solid, links);
  else
    k_links<9><<<grid_for(a.g.ncell), kThreads, 0, s>>>(a.g, solid, links);
  return cudaGetLastError();
}

cudaError_t launch_zero_solid(const AuxArgs& a, void* state, cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_zero_solid, grid_for(a.g.ncell), s, a.g, a.ph, state);
  return cudaGetLastError();
}

cudaError_t launch_health(const AuxArgs& a, const void* state, int* flag, cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_health, grid_for(a.g.ncell), s, a.g, a.ph, state, flag);
  return cudaGetLastError();
}

cudaError_t launch_fill_ghosts(const AuxArgs& a, void* state, cudaStream_t s) {
  CGEVAP_DISPATCH(a, k_fill_ghosts, grid_for(a.g.ncell), s, a.g, state);
  return cudaGetLastError();
}

HeatedPlan heated_plan(const Geom& g) {  // part: nchunk rows of partials + one of fluxes
  HeatedPlan hp;
  const int ncol = g.na * g.nb;
  hp.col_blocks = (ncol + kThreads - 1) / kThreads;
  int want = (152 * 16 + hp.col_blocks - 1) / hp.col_blocks;  // >= 16 CTAs per SM in all
  if (want > g.nm) want = g.nm;
  if (want < 1) want = 1;
  hp.cz = (g.nm + want - 1) / want;
  hp.nchunk = (g.nm + hp.cz - 1) / hp.cz;
  return hp;
}

cudaError_t launch_heated_flux(const AuxArgs& a, const void* state, double* part, double phi_s,
                               double K, double length, void* field, int field_double, cudaStream_t s) {
  const HeatedPlan hp = heated_plan(a.g);
  const dim3 grid((unsigned)hp.col_blocks, (unsigned)hp.nchunk);
  CGEVAP_DISPATCH(a, k_column_liquid, grid, s, a.g, a.ph, state, hp.cz, part);
  k_heated_column<<<hp.col_blocks, kThreads, 0, s>>>(a.g, part, hp.nchunk, phi_s, K, 1.0 / length);
  k_heated_field<<<grid, kThreads, 0, s>>>(a.g, part, hp.nchunk, hp.cz, field, field_double);
  return cudaGetLastError();
}

cudaError_t launch_convert_field(const void* in, int in_dtype, void* out, int out_is_double,
                                 long long n, cudaStream_t s) {
  k_convert<<<grid_for(n), kThreads, 0, s>>>(in, in_dtype, out, out_is_double, n);
  return cudaGetLastError();
}

cudaError_t launch_outlets(const AuxArgs& a, void* state, double rho_lo, double rho_hi, cudaStream_t s) {
  // a colour-blind layout holds no blue half
  if (a.storage == ST_RC || a.storage == ST_H16RC || a.storage == ST_B16RC) return cudaErrorInvalidValue;
  CGEVAP_DISPATCH(a, k_outlet, grid_for(2LL * a.g.na * a.g.nb), s, a.g, a.ph, state, rho_lo, rho_hi);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* out, double v, long long n, cudaStream_t s) {
  k_fill<<<grid_for(n), kThreads, 0, s>>>(out, v, n);
  return cudaGetLastError();
}

}  // namespace cgevap
