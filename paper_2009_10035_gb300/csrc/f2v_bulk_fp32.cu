// f2v_bulk_fp32.cu -- staged-kernel instantiations for FP32 storage of Z.
#include "f2v_bulk.cuh"

namespace f2v {

cudaError_t launch_bulk_fp32(int d, int model, const EpochArgs<float> &a,
                             const CUtensorMap &zmap, const CUtensorMap &mmap, int blocks,
                             int warps, int smem_bytes, cudaStream_t st)
{
    return launch_bulk_t<float>(d, model, a, zmap, mmap, blocks, warps, smem_bytes, st);
}

int bulk_resident(int d, bool bf16, int warps, int smem_bytes)
{
    return bf16 ? bulk_resident_bf16(d, warps, smem_bytes)
                : bulk_resident_t<float>(d, warps, smem_bytes);
}

bool bulk_config(int d, bool bf16, int *warps_per_block, int *smem_bytes)
{
    return bf16 ? bulk_config_t<__nv_bfloat16>(d, warps_per_block, smem_bytes)
                : bulk_config_t<float>(d, warps_per_block, smem_bytes);
}

}  // namespace f2v
