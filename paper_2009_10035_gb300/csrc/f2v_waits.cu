// f2v_waits.cu -- a test of the bounded device waits: one warp waits on a
// flag, a counter or an mbarrier that nothing sets, with the same bounded
// primitives and error codes the force kernels use, and returns once the
// wait runs out (about a second) with the code in the error word.  Nothing
// faults or hangs: the wait is a spin with a cycle limit.
#include <cuda_runtime.h>

#include "f2v_bulk.cuh"
#include "f2v_device.cuh"
#include "f2v_internal.h"

namespace f2v {

namespace {

// kind 0: a flag that was set (no time-out); 1: a row flag nothing sets
// (code 2); 2: a completion counter nothing increments (code 3); 3: an
// mbarrier nothing arrives on (code 1).
__global__ void wait_probe_kernel(int32_t *cells, int kind, int32_t *err)
{
    __shared__ __align__(8) uint64_t bar;
    const int lane = threadIdx.x & 31;
    if (kind == 3) {
        if (lane == 0) mbar_init(&bar, 1);
        fence_mbar_init();
        __syncwarp();
        const bool ok = mbar_wait_bounded(&bar, 0u);
        if (!ok && lane == 0) atomicExch(err, 1);
        return;
    }
    if (lane != 0) return;
    bool ok = true;
    if (kind == 0) {
        cells[0] = 7;
        __threadfence();
        ok = wait_equal(&cells[0], 7);
    } else if (kind == 1) {
        ok = wait_equal(&cells[0], 1);
    } else {
        ok = wait_at_least(&cells[1], 1);
    }
    if (!ok) atomicExch(err, kind == 1 ? 2 : 3);
}

}  // namespace

cudaError_t launch_wait_probe(int32_t *cells, int kind, int32_t *err, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(cells, kind, err);
    return cudaGetLastError();
}

}  // namespace f2v
