// adjoint_kernels.cu -- instantiations and launchers of the adjoint sweep and of the volume
// observable (adjoint.cuh).
#include "adjoint.cuh"
#include "launch.h"

namespace cgevap {

namespace {

template <int Q, int S, int TX, int TY>
KernelRef adj_ref() {
  // the tile's shared memory, then the prefetched lambda^{n+1} columns (Q vec per thread), then
  // the box of ab
  constexpr int smem = TileSmem<Q, S, TX, TY, 1>::BYTES +
                       Q * TX * TY * (int)sizeof(typename Storage<S>::vec) +
                       AdjointEpilogue<TX, TY>::template box_bytes<Q, S>();
  const void* fn = (const void*)cg_adjoint_local_kernel<Q, S, TX, TY>;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return {nullptr, 0};
    attr = true;
  }
  KernelRef k{fn, TX * TY};
  k.smem = smem;
  k.tx = TX;
  k.ty = TY;
  return k;
}

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

KernelRef adjoint_local_kernel(int q, int storage) {
  if (q == 19 && storage == ST_F64) return adj_ref<19, ST_F64, 32, 4>();
  if (q == 19 && storage == ST_F32) return adj_ref<19, ST_F32, 32, 4>();
  if (q == 9 && storage == ST_F64) return adj_ref<9, ST_F64, 128, 1>();
  if (q == 9 && storage == ST_F32) return adj_ref<9, ST_F32, 128, 1>();
  return {nullptr, 0};
}

cudaError_t launch_adjoint_stencil(const AuxArgs& a, const void* aux, const void* lam_g, void* ab,
                                   const uint8_t* mask, double* dphi, double inv_sbar,
                                   const double* dLdV, cudaStream_t s) {
  if (a.g.ncell <= 0) return cudaSuccess;
  const unsigned nb = blocks_for(a.g.ncell);
  if (a.q == 19 && a.storage == ST_F64)
    cg_adjoint_stencil_kernel<19, double><<<nb, kThreads, 0, s>>>(
        a.g, (const double*)aux, lam_g, ab, mask, dphi, inv_sbar, dLdV);
  else if (a.q == 19 && a.storage == ST_F32)
    cg_adjoint_stencil_kernel<19, float><<<nb, kThreads, 0, s>>>(
        a.g, (const float*)aux, lam_g, ab, mask, dphi, inv_sbar, dLdV);
  else if (a.q == 9 && a.storage == ST_F64)
    cg_adjoint_stencil_kernel<9, double><<<nb, kThreads, 0, s>>>(
        a.g, (const double*)aux, lam_g, ab, mask, dphi, inv_sbar, dLdV);
  else if (a.q == 9 && a.storage == ST_F32)
    cg_adjoint_stencil_kernel<9, float><<<nb, kThreads, 0, s>>>(
        a.g, (const float*)aux, lam_g, ab, mask, dphi, inv_sbar, dLdV);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_volume(const AuxArgs& a, const void* state, double* part, unsigned int* done,
                          double* out, cudaStream_t s) {
  long long nb = blocks_for(a.g.ncell);
  if (nb > kVolumeBlocks) nb = kVolumeBlocks;
  if (nb < 1) nb = 1;
  const dim3 grid((unsigned)nb);
#define CG_VOL(QQ, SS) cg_volume_kernel<QQ, SS><<<grid, kThreads, 0, s>>>(a.g, a.ph, state, part, done, out)
  switch (a.q * 10 + a.storage) {
    case 90: CG_VOL(9, ST_F64); break;
    case 91: CG_VOL(9, ST_F32); break;
    case 92: CG_VOL(9, ST_F16); break;
    case 93: CG_VOL(9, ST_BF16); break;
    case 190: CG_VOL(19, ST_F64); break;
    case 191: CG_VOL(19, ST_F32); break;
    case 192: CG_VOL(19, ST_F16); break;
    case 193: CG_VOL(19, ST_BF16); break;
    case 94: CG_VOL(9, ST_RC); break;
    case 194: CG_VOL(19, ST_RC); break;
    case 96: CG_VOL(9, ST_H16RC); break;
    case 97: CG_VOL(9, ST_B16RC); break;
    case 196: CG_VOL(19, ST_H16RC); break;
    case 197: CG_VOL(19, ST_B16RC); break;
    default: return cudaErrorInvalidValue;
  }
#undef CG_VOL
  return cudaGetLastError();
}

}  // namespace cgevap
