// f2v_batch_bf16.cu -- batched-form kernels for BF16 storage of the gathered
// rows with an FP32 master copy.
#include "f2v_batch.cuh"

namespace f2v {

cudaError_t launch_batch_bf16(int shape, const BatchArgs<__nv_bfloat16> &a, int blocks,
                              cudaStream_t st)
{
    return launch_batch_t<__nv_bfloat16>(shape, a, blocks, st);
}

int batch_resident_bf16(int shape) { return batch_resident_t<__nv_bfloat16>(shape); }

}  // namespace f2v
