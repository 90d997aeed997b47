// step_tma.cuh -- the fused timestep with a TMA pipeline through shared memory.
//
// Same arithmetic as cg_step_kernel (step_kernel.cuh), different data movement:
//   * one producer thread streams, for every plane the CTA pulls, Q "source boxes" into a
//     shared-memory stage with TMA tensor copies (cp.async.bulk.tensor, one per direction),
//     completing on an mbarrier; box i holds f_i at plane m - c_i,m over lattice rows
//     b0-1-c_i,b .. b0+TY-c_i,b and columns a0-2 .. a0+TX+1, so every cell of the tile and of its
//     one-cell ring finds its pulled population of direction i at (row, column) =
//     (e_b, e_a + 1 - c_i,a) of box i;
//   * the populations are stored with two ghost columns (and, in 3D, rows) holding periodic
//     images, so a box never wraps; parts of a box beyond the stored grid (ragged last tiles)
//     are zero-filled by the TMA unit and never read; planes beyond a z wall are not copied;
//     links into walls or solids bounce back and read the cell's own population from global
//     memory;
//   * NST stages are in flight; consumers release a stage (empty mbarrier, one arrival per
//     consumer warp) once the plane it holds has been collided;
//   * consumer warps compute rho^N of the tile plus ring into a 4-plane ring, synchronise on a
//     named barrier (the producer never joins it), then collide the previous plane.
// Every mbarrier wait is bounded (about two seconds of wall time); on timeout the thread sets
// the step's status word and carries on, so the launch always ends and the host reports
// CGEVAP_ERR_TIMEOUT.
#pragma once

#include <cuda.h>

#include "step_kernel.cuh"

namespace cgevap {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_arrive(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase with the given parity to complete; gives up after ~2 s and flags it.
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, int* status) {
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return;
    if ((it & 255u) == 0u) {
      const uint64_t t = global_ns();
      if (it == 0) {
        t0 = t;
      } else if (t - t0 > 2000000000ull) {
        if (status) atomicExch(status, 1);
        return;
      }
    }
  }
}

// TMA tensor load of one box: 3-D (x, plane, direction) for D2Q9, 4-D (x, row, plane,
// direction) for D3Q19.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <int Q, int S, int TX, int TY>
struct BoxShape {
  using L = Lattice<Q>;
  using Vec = typename Storage<S>::vec;
  static constexpr int EX = TX + 2;               // tile + ring, columns
  static constexpr int EY = L::D3 ? TY + 2 : 1;   // tile + ring, rows
  static constexpr int BW = TX + 4;               // box columns a0-2 .. a0+TX+1
  static constexpr int BR = EY;                   // box rows
  static constexpr int ROW_BYTES = BW * (int)sizeof(Vec);
  static constexpr int BOX_BYTES = BR * ROW_BYTES;
  static constexpr int BOX_SLOT = (BOX_BYTES + 127) / 128 * 128;  // TMA destinations: 128 B
  static constexpr int STAGE_BYTES = Q * BOX_SLOT;
  static constexpr int NC = TX * TY;              // consumer threads
  static_assert(ROW_BYTES % 16 == 0, "TMA box rows are multiples of 16 bytes");
  static_assert(BW <= 256 && BR <= 256, "TMA box dimensions are at most 256");
};

template <int Q, int S, int TX, int TY, int NST>
constexpr int tma_smem_bytes() {
  using B = BoxShape<Q, S, TX, TY>;
  using R = typename Storage<S>::real;
  return NST * B::STAGE_BYTES + 4 * B::EY * B::EX * (int)sizeof(R) + 2 * NST * 8 +
         (B::NC / 32) * 16 + 16;
}

template <int Q, int S, int TX, int TY, int NST>
__global__ void __launch_bounds__(TX* TY + 32, 1)
    cg_step_tma_kernel(const __grid_constant__ StepArgs A, const __grid_constant__ CUtensorMap tmap) {
  using L = Lattice<Q>;
  using R = typename Storage<S>::real;
  using Vec = typename Storage<S>::vec;
  using B = BoxShape<Q, S, TX, TY>;
  using IO = PopIO<S, Q>;
  constexpr int NC = B::NC;
  constexpr int EX = B::EX, EY = B::EY, OB = L::D3 ? 1 : 0;
  static_assert(!Storage<S>::dev, "deviation storages use another kernel");

  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stages = smem;
  R(*ring)[EY][EX] = reinterpret_cast<R(*)[EY][EX]>(smem + NST * B::STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NST * B::STAGE_BYTES + 4 * EY * EX * sizeof(R));
  double* red_d = reinterpret_cast<double*>(bars + 2 * NST);
  long long* red_n = reinterpret_cast<long long*>(red_d + NC / 32);
  int* is_last = reinterpret_cast<int*>(red_n + NC / 32);

  const Geom& G = A.g;
  const int tid = threadIdx.x;
  const int a0 = (blockIdx.x % A.ntx) * TX;
  const int b0 = (blockIdx.x / A.ntx) * TY;
  const int m0 = blockIdx.y * A.pc;
  const int m1 = min(m0 + A.pc, G.nm);
  const int NP = m1 - m0 + 2;  // planes pulled: m0-1 .. m1
  const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + NST);

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, NC / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  long long n_sites = 0;
  double removed = 0.0;

  if (tid >= NC) {
    // ------------------------------------------------------------------ producer thread ----
    if (tid == NC) {
      const uint32_t stage0 = smem_addr(stages);
      for (int k = 0; k < NP; ++k) {
        const int s = k % NST;
        if (k >= NST) mbar_wait(empty0 + 8 * s, (uint32_t)((k / NST) - 1) & 1u, A.red.status);
        const Plane pl = make_plane(G, m0 - 1 + k);
        int ms[Q];
        uint32_t bytes = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          ms[i] = pl.ok ? step_coord(pl.m, -L::cm(i), G.nm, G.per_m) : -1;
          if (ms[i] >= 0) bytes += B::BOX_BYTES;
        }
        mbar_expect_arrive(full0 + 8 * s, bytes);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (ms[i] < 0) continue;
          const uint32_t dst = stage0 + s * B::STAGE_BYTES + i * B::BOX_SLOT;
          if (L::D3)
            tma_load_4d(dst, &tmap, a0 + kOx - 2, b0 + 1 - L::cb(i), ms[i], i, full0 + 8 * s);
          else
            tma_load_3d(dst, &tmap, a0 + kOx - 2, ms[i], i, full0 + 8 * s);
        }
      }
    }
  } else {
    // ------------------------------------------------------------------ consumer warps -----
    const int lx = tid % TX, ly = tid / TX;
    const bool active = (a0 + lx < G.na) && (b0 + ly < G.nb);
    const Slot me = make_slot<L>(G, a0 + lx, b0 + ly);
    int dimg[3] = {0, 0, 0};
    const int nimg = active ? image_deltas(G, me.a, me.b, dimg) : 0;
    for (int k = 0; k < NP; ++k) {
      const int s = k % NST;
      mbar_wait(full0 + 8 * s, (uint32_t)(k / NST) & 1u, A.red.status);
      const unsigned char* st = stages + s * B::STAGE_BYTES;
      const Plane pl = make_plane(G, m0 - 1 + k);
      // rho^N after the exchange for the tile and its ring (Eq. cg needs it at x + c_i)
      for (int h = tid; h < EX * EY; h += NC) {
        const int ex = h % EX, ey = h / EX;
        const Slot sl = make_slot<L>(G, a0 - 1 + ex, b0 - OB + ey);
        const int cell = (pl.m * G.nb + sl.b) * G.na + sl.a;
        uint32_t bits = 0;
        R rn = R(0);
        if (solid_bits<L>(G, sl, pl, cell, bits)) {
          V2<R> g[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if ((bits >> i) & 1u) {
              g[i] = IO::load(A.pin, G.nstore, i, opp(i), sidx(G, sl.a, sl.b, pl.m), A.ph);
            } else {
              const Vec v = *reinterpret_cast<const Vec*>(
                  st + i * B::BOX_SLOT + ey * B::ROW_BYTES + (ex + 1 - L::ca(i)) * (int)sizeof(Vec));
              g[i] = {v.x, v.y};
            }
          }
          R rr, rb, e, irho;
          uint32_t fl;
          rn = site_exchange<Q, S>(A, cell, g, rr, rb, e, fl, irho);
        }
        ring[k & 3][ey][ex] = rn;
      }
      consumer_sync(NC);
      if (k >= 2) {
        // collide plane m0 + k - 2 from the stage that holds it
        const int kc = k - 1;
        const unsigned char* sc = stages + (kc % NST) * B::STAGE_BYTES;
        const Plane pc = make_plane(G, m0 - 1 + kc);
        const int cell = (pc.m * G.nb + me.b) * G.na + me.a;
        uint32_t bits = 0;
        if (active && solid_bits<L>(G, me, pc, cell, bits)) {
          V2<R> g[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            if ((bits >> i) & 1u) {
              g[i] = IO::load(A.pin, G.nstore, i, opp(i), sidx(G, me.a, me.b, pc.m), A.ph);
            } else {
              const Vec v = *reinterpret_cast<const Vec*>(
                  sc + i * B::BOX_SLOT + (ly + OB) * B::ROW_BYTES + (lx + 2 - L::ca(i)) * (int)sizeof(Vec));
              g[i] = {v.x, v.y};
            }
          }
          R rr, rb, e, irho;
          uint32_t fl;
          site_exchange<Q, S>(A, cell, g, rr, rb, e, fl, irho);
          const R own = ring[kc & 3][ly + OB][lx + 1];
          R rnb[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const bool solid_nb = (bits >> opp(i)) & 1u;
            rnb[i] = solid_nb ? own : ring[(kc + L::cm(i)) & 3][ly + OB + L::cb(i)][lx + 1 + L::ca(i)];
          }
          R Fn;
          collide_store<Q, S>(A, sidx(G, me.a, me.b, pc.m), nimg, dimg, g, rr, rb, irho, rnb, Fn);
          uint32_t mb = fl;
          if (A.ph.rule == 0) {
            const R d = Fn - PHYS(R, A.ph, threshold);
            mb |= (d > R(0) ? 2u : 0u) | (fabs(d) < R(1e-6) ? 8u : 0u);
          }
          A.mask_out[cell] = (uint8_t)mb;
          if (fl & 1u) {
            ++n_sites;
            removed += (double)e;
          }
        }
      }
      // release the stage that no consumer reads again
      const int kr = (k >= 2) ? k - 1 : (k == 1 ? 0 : -1);
      if (kr >= 0 && (kr + NST) < NP) {
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(empty0 + 8 * (kr % NST));
      }
    }
  }

  // ---- ledger: warp shuffle, block, last block folds all partials in order ----
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n_sites += __shfl_down_sync(0xffffffffu, n_sites, off);
    removed += __shfl_down_sync(0xffffffffu, removed, off);
  }
  if ((tid & 31) == 0 && tid < NC) {
    red_d[tid >> 5] = removed;
    red_n[tid >> 5] = n_sites;
  }
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y;
  if (tid == 0) {
    double s = 0.0;
    long long n = 0;
    for (int w = 0; w < NC / 32; ++w) {
      s += red_d[w];
      n += red_n[w];
    }
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    A.red.part_removed[bid] = s;
    A.red.part_sites[bid] = n;
    __threadfence();
    const unsigned prev = atomicAdd(A.red.done, 1u);
    *is_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (*is_last && tid < 32) {
    __threadfence();
    double s = 0.0;
    long long n = 0;
    for (unsigned j = tid; j < nblk; j += 32) {
      s += __ldcg(A.red.part_removed + j);
      n += __ldcg(A.red.part_sites + j);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, off);
      n += __shfl_down_sync(0xffffffffu, n, off);
    }
    if (tid == 0) {
      DevLedger* led = A.red.ledger;
      led->evaporated += s;
      led->last_removed = s;
      led->site_steps += n;
      led->last_sites = n;
      led->steps += 1;
      *A.red.done = 0u;
    }
  }
}

}  // namespace cgevap
