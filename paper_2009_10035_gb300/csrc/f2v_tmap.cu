// f2v_tmap.cu -- TMA tensor maps over row-major embedding buffers.
//
// The staged force kernel gathers partner rows with TMA tile::gather4 loads,
// which fetch four arbitrary rows of a 2-D tensor per instruction.  A map
// here describes `rows` rows of d elements (FP32 or BF16), one box = one
// whole row (box height 1, as gather4 requires).  The driver entry point is
// resolved through the runtime, so the library does not link libcuda.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "f2v_internal.h"

namespace f2v {

namespace {
std::once_flag g_encode_once;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}  // namespace

bool make_row_map(CUtensorMap *map, void *base, int64_t rows, int d, bool bf16, std::string *err)
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        *err = "cuTensorMapEncodeTiled is not available";
        return false;
    }
    const cuuint64_t esz = bf16 ? 2 : 4;
    const cuuint64_t gdim[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)d * esz};
    const cuuint32_t box[2] = {(cuuint32_t)d, 1};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                2, base, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

}  // namespace f2v
