// f2v_batch.cuh -- the persistent kernel of the batched form: one epoch of
// every graph of a batch in one launch.
//
// Each graph runs Algorithm 1 on its own minibatches (ids [k b, (k+1) b) of
// that graph), with the forces of Algorithm 2 and the update of Eq. 10, as
// the single-graph kernel does (the per-item walk is the same force_item).
// What the launch adds is scheduling:
//   queue    warps take warp units in queue order from a global counter; the
//            host orders the minibatch records of all graphs by k / M_g, so
//            that a graph's minibatches are spread over the whole epoch and
//            minibatch k - 1 has long finished when minibatch k comes up;
//   barrier  a unit of minibatch k (> 0) of graph g first waits until every
//            unit of minibatch k - 1 of g has finished (done counter, acquire;
//            units increment it with a release after their last store), so
//            each graph keeps the synchronous-minibatch order of Sec. III-B;
//   buffers  rows of graph g's earlier minibatches come from its next buffer
//            through L2 (they were written in this launch), other rows from
//            its current buffer.
// One launch serves the graphs of one row shape (L lanes x VEC elements per
// row), so every shape keeps the register allocation of its own walk; the
// shapes present run as concurrent launches of one epoch.  A unit only waits
// on units earlier in its queue, which were taken by warps already running,
// so a launch makes progress without assuming that all of its blocks are
// resident.  Waits are bounded; on expiry the kernel sets
// the error word to 2 and every warp stops at its next unit.
#pragma once

#include "f2v_device.cuh"
#include "f2v_force.cuh"
#include "f2v_internal.h"

namespace f2v {

template <int L, int VEC, typename Ts, int MODEL>
__global__ void __launch_bounds__(kBatchBlock, 2) force_batch_kernel(const BatchArgs<Ts> a)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (grp * L));
    for (;;) {
        int idx = 0;
        if (lane == 0) {
            idx = atomicAdd(a.next_unit, 1);
            if (*reinterpret_cast<volatile int32_t *>(a.err) != 0) idx = a.n_units;
        }
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= a.n_units) return;
        const BatchUnit wu = a.units[idx];
        const BatchRec r = a.recs[wu.rec];
        if (r.prev >= 0) {
            int ok = 1;
            if (lane == 0) ok = wait_at_least(&a.done[r.prev], __ldg(&a.recs[r.prev].n_wunits));
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) atomicExch(a.err, 2);
                return;
            }
        }
        const BatchGraph &gr = a.graphs[r.g];
        const BatchState st = a.state[r.g];
        ForceArgs<Ts> f;
        f.row_ptr = gr.row_ptr;
        f.col_idx = gr.col_idx;
        f.apair = gr.apair;
        f.item_u0 = a.item_u0 + r.item_off;
        f.partner = nullptr;
        f.zcur = static_cast<const Ts *>(gr.z[st.cur]);
        f.znext = static_cast<Ts *>(gr.z[st.cur ^ 1]);
        f.master = gr.master;
        f.slots = a.slots + r.slot_off;
        f.unit_cnt = a.unit_cnt + r.cnt_off;
        f.units0 = r.n_items;
        f.counter = gr.counter;
        f.P0 = r.P0;
        f.Pk = r.Pk;
        f.n_items = r.n_items;
        f.mb_begin = r.mb_begin;
        f.mb_end = r.mb_end;
        f.n = gr.n;
        f.d = gr.d;
        f.ld = gr.d;
        f.s = a.s;
        f.C = r.C;
        f.epoch = st.epoch;
        f.key0 = gr.key0;
        f.key1 = gr.key1;
        f.eta = st.eta;
        f.model = a.model;
        f.err = a.err;
        const FinishCtx fc{r.C, f.slots, f.unit_cnt, nullptr, 0};
        const int item = wu.item0 + grp;
        if (item < r.n_items) force_item<L, VEC, 1, true, true, MODEL>(f, fc, item, gl, gmask);
        // every store of the unit (rows, tree parts) before the count
        __syncwarp();
        if (lane == 0)
            asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(&a.done[wu.rec])
                         : "memory");
    }
}

template <typename Ts, int MODEL>
const void *batch_kernel_ptr_m(int shape)
{
    switch (shape) {
        case 0: return (const void *)force_batch_kernel<1, 2, Ts, MODEL>;
        case 1: return (const void *)force_batch_kernel<1, 4, Ts, MODEL>;
        case 2: return (const void *)force_batch_kernel<2, 2, Ts, MODEL>;
        case 3: return (const void *)force_batch_kernel<2, 4, Ts, MODEL>;
        case 4: return (const void *)force_batch_kernel<4, 2, Ts, MODEL>;
        case 5: return (const void *)force_batch_kernel<4, 4, Ts, MODEL>;
        case 6: return (const void *)force_batch_kernel<8, 2, Ts, MODEL>;
        case 7: return (const void *)force_batch_kernel<8, 4, Ts, MODEL>;
        case 8: return (const void *)force_batch_kernel<16, 2, Ts, MODEL>;
        case 9: return (const void *)force_batch_kernel<16, 4, Ts, MODEL>;
        case 10: return (const void *)force_batch_kernel<32, 2, Ts, MODEL>;
        case 11: return (const void *)force_batch_kernel<32, 4, Ts, MODEL>;
        default: return nullptr;
    }
}

// The kernel of a shape and force model (one instantiation per model, so
// the model's branches leave the inner loops).
template <typename Ts>
const void *batch_kernel_ptr(int shape, int model)
{
    return model == 0 ? batch_kernel_ptr_m<Ts, 0>(shape) : batch_kernel_ptr_m<Ts, 1>(shape);
}

template <typename Ts>
cudaError_t launch_batch_t(int shape, const BatchArgs<Ts> &a, int blocks, cudaStream_t st)
{
    const void *fn = batch_kernel_ptr<Ts>(shape, a.model);
    if (!fn) return cudaErrorInvalidValue;
    void *args[] = {const_cast<BatchArgs<Ts> *>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kBatchBlock), args, 0, st);
}

template <typename Ts>
int batch_resident_t(int shape)
{
    int best = -1;
    for (int model = 0; model < 2; ++model) {
        const void *fn = batch_kernel_ptr<Ts>(shape, model);
        int blocks = 0;
        if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kBatchBlock, 0) !=
                       cudaSuccess)
            return 0;
        best = (best < 0) ? blocks : (blocks < best ? blocks : best);
    }
    return best;
}

}  // namespace f2v
