// step_bulk_f32.cu -- instantiations of the bulk-copy pipelined step for FP32 storage.
#include "launch.h"
#include "step_bulk.cuh"

namespace cgevap {

template <int Q, int TX, int TY, int NST>
static KernelRef bulk_ref() {
  constexpr int smem = bulk_smem_bytes<Q, ST_F32, TX, TY, NST>();
  const void* fn = (const void*)cg_step_bulk_kernel<Q, ST_F32, TX, TY, NST>;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return {nullptr, 0};
    attr = true;
  }
  KernelRef k{fn, TX * TY + 32};
  k.smem = smem;
  k.tx = TX;
  k.ty = TY;
  return k;
}

KernelRef step_bulk_f32(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return bulk_ref<19, 32, 8, 4>();
      case 1: return bulk_ref<19, 32, 8, 3>();
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return bulk_ref<9, 128, 1, 4>();
      case 1: return bulk_ref<9, 256, 1, 4>();
    }
  }
  return {nullptr, 0};
}

}  // namespace cgevap
