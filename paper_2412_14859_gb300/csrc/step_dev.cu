// step_dev.cu -- instantiations of the fused step for the FP16 / BF16 deviation storages.
#include "launch.h"
#include "step_dev_kernel.cuh"

namespace cgevap {

// Generic register-pipelined kernel (one cell per thread, decoded pairs parked).
template <int Q, int S, int TX, int TY, int MINB, int CPT>
static KernelRef reg_ref() {
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

// Deviation kernel (raw 4-byte words parked, CPT cells per thread).
template <int Q, int S, int TX, int TY, int MINB, int CPT>
static KernelRef dev_ref() {
  constexpr int smem = DevShape<Q, S, TX, TY, CPT>::SMEM;
  const void* fn = (const void*)cg_step_dev_kernel<Q, S, TX, TY, MINB, CPT>;
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
      case 0: return reg_ref<19, S, 16, 8, 4, 1>();  // the fastest: smallest staged box per cell
      case 1: return dev_ref<19, S, 32, 8, 2, 1>();
      case 2: return reg_ref<19, S, 16, 16, 2, 1>();
      case 3: return dev_ref<19, S, 32, 4, 4, 1>();
      case 4: return reg_ref<19, S, 32, 4, 4, 1>();
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return dev_ref<9, S, 128, 1, 4, 1>();
      case 1: return reg_ref<9, S, 128, 1, 4, 1>();
    }
  }
  return {nullptr, 0};
}

KernelRef step_kernel_dev(int q, int storage, int variant) {
  return storage == ST_F16 ? pick<ST_F16>(q, variant) : pick<ST_BF16>(q, variant);
}

}  // namespace cgevap
