// step_rc16.cu -- instantiations of the fused step for the 16-bit recolour-on-pull layouts
// (ST_H16RC: FP16 deviations, ST_B16RC: BF16), FP32 arithmetic; ST_H16RCI / ST_B16RCI are the
// same step reading an imported state held as FP32 pairs.
#include "launch.h"
#include "step_kernel.cuh"

namespace cgevap {

template <int Q, int S, int TX, int TY, int MINB, int CPT>
static KernelRef rc16_ref() {
  constexpr int smem = TileSmem<Q, S, TX, TY, CPT>::BYTES;
  const void* fn = (const void*)cg_step_kernel<Q, S, TX, TY, MINB, CPT>;
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

template <int S>
static KernelRef pick(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return rc16_ref<19, S, 16, 8, 4, 1>();
      case 1: return rc16_ref<19, S, 32, 4, 4, 1>();
      case 2: return rc16_ref<19, S, 16, 16, 2, 1>();  // 256 threads: a smaller ring per cell
      case 3: return rc16_ref<19, S, 16, 4, 8, 1>();
      case 4: return rc16_ref<19, S, 32, 8, 2, 1>();  // 256 threads: a smaller ring per cell
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return rc16_ref<9, S, 128, 1, 4, 1>();
      case 1: return rc16_ref<9, S, 64, 1, 8, 1>();
    }
  }
  return {nullptr, 0};
}

KernelRef step_kernel_rc16(int q, int storage, int variant, bool pairs_in) {
  if (storage == ST_H16RC) return pairs_in ? pick<ST_H16RCI>(q, variant) : pick<ST_H16RC>(q, variant);
  if (storage == ST_B16RC) return pairs_in ? pick<ST_B16RCI>(q, variant) : pick<ST_B16RC>(q, variant);
  return {nullptr, 0};
}

}  // namespace cgevap
