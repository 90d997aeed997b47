// step_dev.cu -- instantiations of the fused step for the FP16 / BF16 deviation storages.
#include "launch.h"
#include "step_kernel.cuh"

namespace cgevap {

template <int S>
static KernelRef pick(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return {(const void*)cg_step_kernel<19, S, 32, 8, 2>, 256};
      case 1: return {(const void*)cg_step_kernel<19, S, 32, 4, 4>, 128};
      case 2: return {(const void*)cg_step_kernel<19, S, 64, 4, 2>, 256};
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return {(const void*)cg_step_kernel<9, S, 128, 1, 4>, 128};
      case 1: return {(const void*)cg_step_kernel<9, S, 64, 1, 8>, 64};
    }
  }
  return {nullptr, 0};
}

KernelRef step_kernel_dev(int q, int storage, int variant) {
  return storage == ST_F16 ? pick<ST_F16>(q, variant) : pick<ST_BF16>(q, variant);
}

}  // namespace cgevap
