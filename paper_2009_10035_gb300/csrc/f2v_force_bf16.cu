// f2v_force_bf16.cu -- force kernel instantiations for BF16 storage of the
// gathered rows with an FP32 master copy (the precision form).
#include "f2v_bulk.cuh"
#include "f2v_force.cuh"

namespace f2v {

cudaError_t launch_force_bf16(const Shape &sh, const ForceArgs<__nv_bfloat16> &a,
                              int blocks_cap, cudaStream_t st)
{
    return launch_force_any<__nv_bfloat16>(sh, a, blocks_cap, st);
}

cudaError_t launch_bulk_bf16(int d, int model, const EpochArgs<__nv_bfloat16> &a,
                             const CUtensorMap &zmap, const CUtensorMap &mmap, int blocks,
                             int warps, int smem_bytes, cudaStream_t st)
{
    return launch_bulk_t<__nv_bfloat16>(d, model, a, zmap, mmap, blocks, warps, smem_bytes, st);
}

}  // namespace f2v
