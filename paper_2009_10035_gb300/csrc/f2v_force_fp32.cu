// f2v_force_fp32.cu -- force kernel instantiations for FP32 storage of Z.
#include "f2v_bulk.cuh"
#include "f2v_force.cuh"

namespace f2v {

cudaError_t launch_force_fp32(const Shape &sh, const ForceArgs<float> &a, int blocks_cap,
                              cudaStream_t st)
{
    return launch_force_any<float>(sh, a, blocks_cap, st);
}

cudaError_t launch_bulk_fp32(int d, int model, const EpochArgs<float> &a,
                             const CUtensorMap &zmap, const CUtensorMap &mmap, int blocks,
                             int warps, int smem_bytes, cudaStream_t st)
{
    return launch_bulk_t<float>(d, model, a, zmap, mmap, blocks, warps, smem_bytes, st);
}

int bulk_resident(int d, bool bf16, int warps, int smem_bytes)
{
    return bf16 ? bulk_resident_t<__nv_bfloat16>(d, warps, smem_bytes)
                : bulk_resident_t<float>(d, warps, smem_bytes);
}

bool bulk_config(int d, bool bf16, int *warps_per_block, int *smem_bytes)
{
    return bf16 ? bulk_config_t<__nv_bfloat16>(d, warps_per_block, smem_bytes)
                : bulk_config_t<float>(d, warps_per_block, smem_bytes);
}

}  // namespace f2v
