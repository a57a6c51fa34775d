// f2v_batch_fp32.cu -- batched-form kernels for FP32 storage of Z.
#include "f2v_batch.cuh"

namespace f2v {

cudaError_t launch_batch_fp32(int shape, const BatchArgs<float> &a, int blocks, cudaStream_t st)
{
    return launch_batch_t<float>(shape, a, blocks, st);
}

int batch_resident_fp32(int shape) { return batch_resident_t<float>(shape); }

}  // namespace f2v
