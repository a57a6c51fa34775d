// f2v_bulk_bf16.cu -- staged-kernel instantiations for BF16 storage of the
// gathered rows with an FP32 master copy (the precision form).
#include "f2v_bulk.cuh"

namespace f2v {

cudaError_t launch_bulk_bf16(int d, int model, const EpochArgs<__nv_bfloat16> &a,
                             const CUtensorMap &zmap, const CUtensorMap &mmap, int blocks,
                             int warps, int smem_bytes, cudaStream_t st)
{
    return launch_bulk_t<__nv_bfloat16>(d, model, a, zmap, mmap, blocks, warps, smem_bytes, st);
}

int bulk_resident_bf16(int d, int warps, int smem_bytes)
{
    return bulk_resident_t<__nv_bfloat16>(d, warps, smem_bytes);
}

}  // namespace f2v
