// f2v_force_fp32.cu -- register-kernel instantiations for FP32 storage of Z.
#include "f2v_force.cuh"

namespace f2v {

cudaError_t launch_force_fp32(const Shape &sh, const ForceArgs<float> &a, int blocks_cap,
                              cudaStream_t st)
{
    return launch_force_any<float>(sh, a, blocks_cap, st);
}

}  // namespace f2v
