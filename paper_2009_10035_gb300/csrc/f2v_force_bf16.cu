// f2v_force_bf16.cu -- register-kernel instantiations for BF16 storage of the
// gathered rows with an FP32 master copy (the precision form).
#include "f2v_force.cuh"

namespace f2v {

cudaError_t launch_force_bf16(const Shape &sh, const ForceArgs<__nv_bfloat16> &a,
                              int blocks_cap, cudaStream_t st)
{
    return launch_force_any<__nv_bfloat16>(sh, a, blocks_cap, st);
}

}  // namespace f2v
