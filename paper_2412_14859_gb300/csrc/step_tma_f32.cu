// step_tma_f32.cu -- instantiations of the TMA-pipelined step for FP32 storage, and the tensor
// maps that describe a population buffer to the TMA unit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "launch.h"
#include "step_tma.cuh"

namespace cgevap {

template <int Q, int TX, int TY, int NST>
static KernelRef tma_ref() {
  constexpr int smem = tma_smem_bytes<Q, ST_F32, TX, TY, NST>();
  static_assert(smem <= 232448, "dynamic shared memory per block is at most 227 KB");
  const void* fn = (const void*)cg_step_tma_kernel<Q, ST_F32, TX, TY, NST>;
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
  k.needs_map = 1;
  return k;
}

KernelRef step_tma_f32(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return tma_ref<19, 32, 8, 4>();
      case 1: return tma_ref<19, 32, 8, 3>();
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return tma_ref<9, 128, 1, 4>();
      case 1: return tma_ref<9, 192, 1, 4>();
    }
  }
  return {nullptr, 0};
}

int make_pop_tensor_map(void* map, const void* base, const Geom& g, int q, int elem_bytes,
                        int box_w, int box_h) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const CUtensorMapDataType dt =
      elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
  cuuint32_t rank;
  if (q == 19) {
    rank = 4;
    dims[0] = (cuuint64_t)g.pitch;
    dims[1] = (cuuint64_t)g.rows;
    dims[2] = (cuuint64_t)g.nm;
    dims[3] = (cuuint64_t)q;
    strides[0] = (cuuint64_t)g.pitch * elem_bytes;
    strides[1] = strides[0] * g.rows;
    strides[2] = strides[1] * g.nm;
    box[0] = (cuuint32_t)box_w;
    box[1] = (cuuint32_t)box_h;
    box[2] = 1;
    box[3] = 1;
  } else {
    rank = 3;
    dims[0] = (cuuint64_t)g.pitch;
    dims[1] = (cuuint64_t)g.nm;
    dims[2] = (cuuint64_t)q;
    strides[0] = (cuuint64_t)g.pitch * elem_bytes;
    strides[1] = strides[0] * g.nm;
    box[0] = (cuuint32_t)box_w;
    box[1] = 1;
    box[2] = 1;
  }
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), dt, rank, const_cast<void*>(base), dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

}  // namespace cgevap
