// step_f32.cu -- instantiations of the fused step for ST_F32 storage.
#include "launch.h"
#include "step_kernel.cuh"

namespace cgevap {

// Every FP32 variant issues its own cells' pulls one plane ahead (PF): 16.2 -> 18.7 GLUPS on the
// 192^3 drop at the same 128 registers.
template <int Q, int TX, int TY, int MINB, int CPT, int S = ST_F32>
static KernelRef reg_ref() {
  constexpr int smem = TileSmem<Q, S, TX, TY, CPT>::BYTES;
  const void* fn = (const void*)cg_step_kernel<Q, S, TX, TY, MINB, CPT, true>;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return {nullptr, 0};
    attr = true;
  }
  KernelRef k{fn, TX * TY};
  k.smem = smem;
  k.tx = TX;
  k.ty = TY * CPT;
  return k;
}

KernelRef step_kernel_f32(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return reg_ref<19, 32, 4, 4, 1>();  // 128 threads, four CTAs per SM
      case 1: return reg_ref<19, 16, 8, 4, 1>();
      case 2: return reg_ref<19, 16, 16, 2, 1>();
      case 3: return reg_ref<19, 16, 4, 8, 1>();  // 64 threads, eight CTAs per SM
      case 4: return reg_ref<19, 32, 8, 2, 1>();
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return reg_ref<9, 128, 1, 4, 1>();
      case 1: return reg_ref<9, 64, 1, 8, 1>();
    }
  }
  return {nullptr, 0};
}

// FP32 pairs with exact colour masses (ST_F32X): the same tiles.
KernelRef step_kernel_f32x(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return reg_ref<19, 32, 4, 4, 1, ST_F32X>();
      case 1: return reg_ref<19, 16, 8, 4, 1, ST_F32X>();
      case 2: return reg_ref<19, 16, 16, 2, 1, ST_F32X>();
      case 3: return reg_ref<19, 16, 4, 8, 1, ST_F32X>();
      case 4: return reg_ref<19, 32, 8, 2, 1, ST_F32X>();
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return reg_ref<9, 128, 1, 4, 1, ST_F32X>();
      case 1: return reg_ref<9, 64, 1, 8, 1, ST_F32X>();
    }
  }
  return {nullptr, 0};
}

}  // namespace cgevap
