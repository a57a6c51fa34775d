// f2v_internal.h -- declarations shared by the translation units of libf2v
// (host driver, force kernels, auxiliary kernels).  Not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

namespace f2v {

// Arguments of one launch of the fused force+update kernel: the work of one
// minibatch V_b = [mb_begin, mb_end) of Algorithm 1.
//
// Pair space.  Vertex u owns c(u) = deg(u) + s force pairs (plus one empty
// pair when deg(u) + s == 0, so that every vertex is visited and its row is
// carried into the next buffer).  apair[u] is the exclusive prefix sum of
// c(u); pair apair[u] + j of u is its j-th neighbour for j < deg(u) and its
// negative sample k = j - deg(u) otherwise.  The minibatch's pairs
// [P0, P1) are cut into items of C consecutive pairs; item i starts inside
// vertex item_u0[i].
//
// Double buffering.  zcur holds every row as it stood before this epoch;
// znext receives the new rows.  Within epoch e, minibatch k reads row v from
// znext if v < mb_begin (already updated this epoch) and from zcur otherwise
// (not yet updated, including the minibatch's own rows -- the synchronous
// minibatch rule of Sec. III-B).  Nothing is copied back: the buffers swap
// roles at the end of the epoch.
//
// Split vertices.  A vertex whose pairs span several items is summed in
// parts, combined up a fixed tree whose level-l units are runs of 16^l
// consecutive items.  At each level a split vertex meets a unit either at
// the unit's first pair or at its last one, so it owns slot 2*unit or
// 2*unit+1 of that level (`slots`, `unit_cnt`).  The part of the last child
// to arrive (arrival counter) adds the children's parts in unit order and
// passes the sum up; at the level where one unit covers the whole vertex the
// sum is the gradient, and that final arrival counts on counter[u].  Every
// counter is reset to zero by the part that completes it.  The order of
// every addition is fixed, so results do not depend on scheduling.
constexpr int kFan = 16;        // tree fan-out
constexpr int kMaxLevels = 8;   // 16^8 items per minibatch at most

template <typename Ts>
struct ForceArgs {
    const int32_t *row_ptr;    // n + 1
    const int32_t *col_idx;    // nnz
    const int64_t *apair;      // n + 1
    const int32_t *item_u0;    // items of this minibatch
    const Ts *zcur;            // n x ld
    Ts *znext;                 // n x ld
    float *master;             // BF16 form: FP32 master rows (n x ld); else nullptr
    float *slots;              // level l: 2 * units_l rows of ld floats, levels in order
    int32_t *unit_cnt;         // level l >= 1: 2 * units_l arrival counters, in order
    int64_t units0;            // units of level 0 (the most items of any minibatch)
    int32_t *counter;          // n final arrival counters, zero outside a launch
    int64_t P0;                // first pair of the minibatch
    int32_t Pk;                // pairs in the minibatch (< 2^31)
    int32_t n_items;
    int32_t mb_begin, mb_end;
    int32_t n, d, ld, s;
    int32_t C;                 // pairs per item
    uint32_t epoch;
    uint32_t key0, key1;       // Philox key = (seed lo, seed hi)
    float eta;
    int32_t model;             // 0 = t-distribution, 1 = sigmoid
    int32_t *err;              // device error word (1 = a bounded wait timed out)
};

// Arguments of one launch: minibatches [k_begin, k_end) of epoch f.epoch.
// The per-minibatch fields of `f` (P0, Pk, n_items, mb_begin, mb_end, C,
// item_u0, slots, unit_cnt) are not used; each minibatch's values come from
// the tables below.
template <typename Ts>
struct EpochArgs {
    ForceArgs<Ts> f;
    const int32_t *partner;        // partner of every pair of the epoch (expand_partners)
    const int32_t *items;          // chunk start vertices of every minibatch
    const int64_t *mb_item_base;   // M + 1: first chunk of each minibatch in `items`
    const int32_t *mb_C;           // M: pairs per chunk of each minibatch
    int32_t *row_flag;             // n: epoch + 1 once row v is written this epoch
    int32_t *mb_done;              // M: chunks finished (zeroed before the launch)
    float *slots;                  // ring regions of combine-tree slots
    int32_t *unit_cnt;             // ring regions of combine-tree counters
    int64_t slot_stride, cnt_stride;
    int32_t k_begin, k_end, b, ring;
    // rows of the tensor maps: both Z buffers form one map of 2n rows
    int32_t zcur_row0, znext_row0;  // first map row of each buffer
    int32_t own_row0;               // first own row in the own-row map
};

// TMA map over `rows` rows of d elements (FP32 or BF16) starting at `base`,
// one box per row, for tile::gather4 loads.  False (and *err) on failure.
bool make_row_map(CUtensorMap *map, void *base, int64_t rows, int d, bool bf16,
                  std::string *err);

// Partner codes of the expanded pair list: v >= 0 a neighbour (attractive
// force), -2 - w a negative sample w (repulsive force), -1 no force (a sample
// that drew u itself, or the empty pair of a vertex with deg + s = 0).
constexpr int32_t kPartnerNone = -1;

// Writes the partner code of every pair of epoch `epoch` (pair apair[u] + j
// of vertex u), one warp per vertex.
cudaError_t launch_expand_partners(const int32_t *row_ptr, const int32_t *col_idx,
                                   const int64_t *apair, int32_t n, int32_t s, uint32_t epoch,
                                   uint32_t key0, uint32_t key1, int32_t *partner,
                                   cudaStream_t st);

// Kernel shape chosen from d: a group of L lanes owns one force pair at a
// time; each lane holds NV vectors of VEC consecutive elements of a row.
struct Shape {
    int L, VEC, NV;
    bool exact;                // L * VEC * NV == d (else masked generic shape)
};

Shape choose_shape(int d);

// Pairs per item for a shape.
int items_pairs(const Shape &sh);

// The shared-memory staged kernel (f2v_bulk.cuh) serves FP32 and BF16 rows
// of d in {64, 128, 256}; it runs `warps` warps per block, one block per SM,
// each warp walking one chunk.  Returns false if d has no such kernel.
bool bulk_config(int d, bool bf16, int *warps_per_block, int *smem_bytes);
// Blocks of that kernel resident per SM (0 if it cannot run).
int bulk_resident(int d, bool bf16, int warps, int smem_bytes);
// `zmap` covers both Z buffers (2n rows of the storage type); `mmap` the FP32
// own rows (the master in the BF16 form, zmap again in the FP32 form).
cudaError_t launch_bulk_fp32(int d, const EpochArgs<float> &a, const CUtensorMap &zmap,
                             const CUtensorMap &mmap, int blocks, int warps, int smem_bytes,
                             cudaStream_t st);
cudaError_t launch_bulk_bf16(int d, const EpochArgs<__nv_bfloat16> &a, const CUtensorMap &zmap,
                             const CUtensorMap &mmap, int blocks, int warps, int smem_bytes,
                             cudaStream_t st);

// Launches the force kernel for one minibatch.  Returns the CUDA error of the
// launch.  `blocks_cap` bounds the grid (0 = no bound).
cudaError_t launch_force_fp32(const Shape &sh, const ForceArgs<float> &a, int blocks_cap,
                              cudaStream_t st);
cudaError_t launch_force_bf16(const Shape &sh, const ForceArgs<__nv_bfloat16> &a,
                              int blocks_cap, cudaStream_t st);

}  // namespace f2v
