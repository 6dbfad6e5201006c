// Tensor-map descriptors for the TMA-fed V-cycle passes (complex64).
//
// 2D: a level's vectors are P x P complex64 fields (padded layout, row pitch P).  The
// maps describe them as P rows of 2P floats and move 136 x 18 float boxes: the
// 64 x 16 tile of a pass plus a halo of one point, starting two points left of the
// tile so that every box starts on a 16-byte boundary.
// 3D: P x P x P fields as P planes of P rows of 2P floats, moved one plane at a time
// in 72 x (TY + 2) x 1 float boxes (a 32 x TY column tile plus its halo, from two
// points left of the tile).  Out-of-range parts of a box are filled with zeros.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "helm_internal.h"

namespace helm {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

}  // namespace

bool encode_level_tmaps(int P, const void* const* vectors, int count, CUtensorMap* out) {
  const EncodeTiledFn fn = encoder();
  if (!fn || P < 2 || (P & 1)) return false;  // row pitch 8P bytes must be a multiple of 16
  const cuuint64_t dims[2] = {(cuuint64_t)2 * P, (cuuint64_t)P};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * P * sizeof(float)};
  const cuuint32_t box[2] = {2 * (64 + 4), 16 + 2};
  const cuuint32_t estr[2] = {1, 1};
  for (int i = 0; i < count; ++i) {
    std::memset(&out[i], 0, sizeof(CUtensorMap));
    if (!vectors[i]) continue;  // a vector the level does not have (never loaded)
    if (reinterpret_cast<uintptr_t>(vectors[i]) & 15) return false;
    if (fn(&out[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(vectors[i]), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

bool encode_level_tmaps3(int P, int box_rows, const void* const* vectors, int count, CUtensorMap* out) {
  const EncodeTiledFn fn = encoder();
  if (!fn || P < 32 || (P % 32)) return false;  // whole 32-point tiles; row pitch 8P bytes
  const cuuint64_t dims[3] = {(cuuint64_t)2 * P, (cuuint64_t)P, (cuuint64_t)P};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * P * sizeof(float), (cuuint64_t)2 * P * P * sizeof(float)};
  if (box_rows < 1 || box_rows > 256) return false;
  const cuuint32_t box[3] = {2 * (32 + 4), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int i = 0; i < count; ++i) {
    std::memset(&out[i], 0, sizeof(CUtensorMap));
    if (!vectors[i]) continue;
    if (reinterpret_cast<uintptr_t>(vectors[i]) & 15) return false;
    if (fn(&out[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(vectors[i]), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace helm
