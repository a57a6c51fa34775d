// f2v_internal.h -- declarations shared by the translation units of libf2v
// (host driver, force kernels, auxiliary kernels).  Not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "f2v.h"

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
    const int32_t *partner;    // if not null: the epoch's partner codes (pair P0 + q),
                               // read instead of col_idx and Philox (rForce2Vec)
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
    int32_t *mb_next;              // M: chunks claimed (zeroed before the launch)
    float *slots;                  // ring regions of combine-tree slots
    int32_t *unit_cnt;             // ring regions of combine-tree counters
    int64_t slot_stride, cnt_stride;
    int32_t k_begin, k_end, b, ring;
    int32_t groups;                 // chunks handed out in groups of kFan per block
    // rows of the tensor maps: both Z buffers form one map of 2n rows
    int32_t zcur_row0, znext_row0;  // first map row of each buffer
    int32_t own_row0;               // first own row in the own-row map
};

// TMA map over `rows` rows of d elements (FP32 or BF16) starting at `base`,
// one box per row, for tile::gather4 loads.  False (and *err) on failure.
bool make_row_map(CUtensorMap *map, void *base, int64_t rows, int d, bool bf16,
                  std::string *err);

// Partner codes of the expanded pair list: v >= 0 a neighbour or a vertex a
// walk reached (attractive force), -2 - w a negative sample w (repulsive
// force), -1 no force (a sample or walk step that drew u itself, a walk step
// after the walk stopped, or the empty pair of a vertex without pairs).
constexpr int32_t kPartnerNone = -1;

// Writes the partner code of every pair of epoch `epoch` (pair apair[u] + j
// of vertex u), one warp per vertex.  shared_b > 0: the samples are the
// shared set of u's minibatch of that size (negative_sample).
// perm, rank (may be null): the graph is relabelled by a random partition;
// samples keep the counters of the original ids and are mapped to ranks.
cudaError_t launch_expand_partners(const int32_t *row_ptr, const int32_t *col_idx,
                                   const int64_t *apair, int32_t n, int32_t s, int32_t shared_b,
                                   const int32_t *perm, const int32_t *rank, uint32_t epoch,
                                   uint32_t key0, uint32_t key1, int32_t *partner,
                                   cudaStream_t st);

// The sample pairs of such a list (for the graph as given, no walks) for
// epoch `epoch`, in a buffer whose neighbour codes are already written (a
// list of another epoch): the neighbour codes are the same in every epoch.
cudaError_t launch_refresh_samples(const int32_t *row_ptr, const int64_t *apair, int32_t n,
                                   int32_t s, int32_t shared_b, uint32_t epoch, uint32_t key0,
                                   uint32_t key1, int32_t *partner, cudaStream_t st);

// rForce2Vec (Algorithm 3): the same list with vertex u's first `walk` pairs
// (if u has neighbours) the steps of a random walk from u, one thread per
// vertex: step i moves from w to its neighbour number
// Philox(key, ctr = (u, epoch, i, 1)).x0 mod deg(w).
cudaError_t launch_expand_walks(const int32_t *row_ptr, const int32_t *col_idx,
                                const int64_t *apair, int32_t n, int32_t s, int32_t walk,
                                int32_t shared_b, const int32_t *perm, const int32_t *rank,
                                uint32_t epoch, uint32_t key0, uint32_t key1, int32_t *partner,
                                cudaStream_t st);

// The random partition of an epoch (the partition step of Algorithm 1), f2v_partition.cu.
struct PartitionScratch {
    uint32_t *keys, *keys2;    // n: sort keys
    int32_t *vals;             // n: sort values (vertex ids)
    int32_t *deg;              // n + 1
    int64_t *cnt;              // n + 1
    int64_t *nch;              // M + 1
    void *temp;                // CUB temporary storage
    size_t temp_bytes;
};
size_t partition_temp_bytes(int32_t n, int32_t M);
// perm[p]: the vertex at position p in epoch `epoch`'s order (Philox key
// ctr = (v, epoch, 0, 3), ties by id); rank = its inverse.
cudaError_t launch_partition(int32_t n, uint32_t epoch, uint32_t key0, uint32_t key1,
                             const PartitionScratch &w, int32_t *perm, int32_t *rank,
                             cudaStream_t st);
// The graph relabelled into that order (row p = neighbours of perm[p] as
// ranks, in CSR order) and its pair prefix.
cudaError_t launch_relabel(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *perm,
                           const int32_t *rank, int32_t n, int32_t s, int32_t walk,
                           const PartitionScratch &w, int32_t *row_ptr2, int32_t *col_idx2,
                           int64_t *apair2, cudaStream_t st);
// Chunk sizes (staged kernel: W warps; register kernel: W = 0, Cfix pairs),
// chunk offsets, chunk start vertices and minibatch pair offsets (M + 1).
cudaError_t launch_mb_tables(const int64_t *apair2, int32_t n, int32_t b, int32_t M, int64_t W,
                             int32_t Cfix, const PartitionScratch &w, int32_t *mb_C,
                             int64_t *mb_base, int32_t *items, int64_t *mb_p0, cudaStream_t st);
// dst[p] = src[perm[p]] (gather) or dst[perm[p]] = src[p] (scatter), FP32 rows.
cudaError_t launch_permute_rows(const float *src, float *dst, const int32_t *perm, int64_t rows,
                                int32_t d, bool scatter, cudaStream_t st);

// One warp waiting, with the force kernels' bounded primitives, on a cell
// (kind 1, 2) or an mbarrier (kind 3) that nothing sets; kind 0 waits on a
// cell it has set (f2v_waits.cu).  cells: two zeroed ints.
cudaError_t launch_wait_probe(int32_t *cells, int kind, int32_t *err, cudaStream_t st);

// Downstream evaluations of Sec. IV (f2v_downstream.cu), FP64.
size_t lr_smem_bytes(int32_t d);
cudaError_t launch_lr_newton(const float *z, int32_t d, const int32_t *pos, int64_t npos,
                             const int32_t *neg, const int64_t *idx, int64_t m,
                             const double *theta, double *g, double *H, cudaStream_t st);
cudaError_t launch_lr_solve(int32_t d, double *H, double *g, double *theta, double *step_max,
                            cudaStream_t st);
cudaError_t launch_lr_accuracy(const float *z, int32_t d, const int32_t *pos, int64_t npos,
                               const int32_t *neg, const int64_t *idx, int64_t m,
                               const double *theta, unsigned long long *correct, cudaStream_t st);
cudaError_t launch_km_init(const float *z, int32_t d, const int32_t *init, int32_t k, double *C,
                           cudaStream_t st);
cudaError_t launch_km_assign(const float *z, int32_t n, int32_t d, const double *C, int32_t k,
                             int32_t *labels, double *sums, unsigned long long *counts,
                             unsigned long long *changed, cudaStream_t st);
cudaError_t launch_km_update(int32_t k, int32_t d, const double *sums,
                             const unsigned long long *counts, double *C, cudaStream_t st);
cudaError_t launch_modularity(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                              int64_t nnz, const int32_t *labels, int32_t k,
                              unsigned long long *e, unsigned long long *D, double *q,
                              cudaStream_t st);

// out[u * walk + i]: the code of walk step i of vertex u in the list
// `partner` (kPartnerNone for a vertex without neighbours).
cudaError_t launch_extract_walks(const int64_t *apair, const int32_t *row_ptr, int32_t n,
                                 int32_t walk, const int32_t *partner, int32_t *out,
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
int bulk_resident_bf16(int d, int warps, int smem_bytes);
// `zmap` covers both Z buffers (2n rows of the storage type); `mmap` the FP32
// own rows (the master in the BF16 form, zmap again in the FP32 form).
// `model` selects the instantiation (0 t-distribution, 1 sigmoid).
cudaError_t launch_bulk_fp32(int d, int model, const EpochArgs<float> &a,
                             const CUtensorMap &zmap, const CUtensorMap &mmap, int blocks,
                             int warps, int smem_bytes, cudaStream_t st);
cudaError_t launch_bulk_bf16(int d, int model, const EpochArgs<__nv_bfloat16> &a,
                             const CUtensorMap &zmap, const CUtensorMap &mmap, int blocks,
                             int warps, int smem_bytes, cudaStream_t st);

// Launches the force kernel for one minibatch.  Returns the CUDA error of the
// launch.  `blocks_cap` bounds the grid (0 = no bound).
cudaError_t launch_force_fp32(const Shape &sh, const ForceArgs<float> &a, int blocks_cap,
                              cudaStream_t st);
cudaError_t launch_force_bf16(const Shape &sh, const ForceArgs<__nv_bfloat16> &a,
                              int blocks_cap, cudaStream_t st);

// Host-side checks shared by the entry points (f2v_api.cu): the CSR rules of
// f2v_create (message in the thread's global error), and that error string.
f2v_status check_csr(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, uint32_t flags);
// The same checks with at most max_threads host threads, the reason in *msg
// and no global state touched (graphs may be checked concurrently).
f2v_status check_csr_quiet(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                           uint32_t flags, int max_threads, std::string *msg);
void set_global_error(const std::string &msg);
std::string global_error();

// ---- batched form (f2v_batch.cuh, f2v_batch.cu) -----------------------------
//
// A batch is a set of independent graphs stepped one epoch at a time by one
// persistent launch per row shape.  A launch's work is a queue of warp units;
// a unit is 32 / L consecutive items (one per lane group) of one minibatch
// record.

// Row shapes of the batched kernel: (L lanes per row, VEC elements per lane),
// L * VEC = d, NV = 1.  kBatchShapes lists them; the code of a shape is its
// index.
struct BatchShape {
    int d, L, VEC;
};
constexpr int kNumBatchShapes = 12;
constexpr BatchShape kBatchShapes[kNumBatchShapes] = {
    {2, 1, 2},   {4, 1, 4},   {4, 2, 2},   {8, 2, 4},   {8, 4, 2},   {16, 4, 4},
    {16, 8, 2},  {32, 8, 4},  {32, 16, 2}, {64, 16, 4}, {64, 32, 2}, {128, 32, 4},
};

// One graph of a batch (device table, rebuilt with the work tables).
struct BatchGraph {
    const int32_t *row_ptr;    // n + 1, local offsets into col_idx
    const int32_t *col_idx;    // local vertex ids
    const int64_t *apair;      // n + 1 pair prefix (as ForceArgs::apair)
    void *z[2];                // storage rows of the two buffers (n x d)
    float *master;             // BF16 form: FP32 master rows; else nullptr
    int32_t *counter;          // n final-arrival counters of the combine tree
    int32_t n, d, shape;       // shape: index into kBatchShapes
    uint32_t key0, key1;       // Philox key = (seed lo, seed hi)
    float lr;                  // eta schedule of this graph
    int32_t schedule, total_epochs;
};

// Epoch state of one graph, advanced on the device after each epoch.
struct BatchState {
    uint32_t epoch;            // epoch counter e (samples, eta)
    int32_t cur;               // buffer holding Z as of the epoch's start
    float eta;                 // eta_e
    int32_t pad;
};

// One minibatch (graph g, minibatch k) of an epoch.
struct BatchRec {
    int64_t P0;                // local index of its first pair
    int64_t slot_off;          // its combine-tree slots (floats into the pool)
    int64_t cnt_off;           // its combine-tree counters (ints into the pool)
    int32_t g, mb_begin, mb_end;
    int32_t Pk, C, n_items;
    int32_t item_off;          // its items' start vertices in BatchArgs::item_u0
    int32_t n_wunits;          // warp units of this minibatch
    int32_t prev;              // record of minibatch k - 1 of graph g, or -1
    int32_t unit_off;          // its first warp unit in the unit table
    int32_t gsize;             // items per warp unit (32 / L)
    int32_t pad;
};

struct BatchUnit {
    int32_t rec, item0;        // items item0 .. item0 + 32/L - 1 of record rec
};

template <typename Ts>
struct BatchArgs {
    const BatchGraph *graphs;
    BatchState *state;
    const BatchRec *recs;
    const BatchUnit *units;    // this launch's queue (one shape), in order
    const int32_t *item_u0;
    float *slots;
    int32_t *unit_cnt;
    int32_t *done;             // per record: warp units finished (zero at launch)
    int32_t *next_unit;        // queue head (zero at launch)
    int32_t n_units, n_graphs;
    int32_t s, model;
    int32_t *err;              // 2 = a minibatch barrier wait timed out
};

constexpr int kBatchBlock = 256;

// Host: eta of epoch e (the same arithmetic as the single-graph context).
inline double batch_eta(float lr, int schedule, int total_epochs, int e)
{
    if (schedule == 1 && total_epochs > 0)
        return (double)lr * (1.0 - (double)e / (double)total_epochs);
    return (double)lr;
}

// Launches the batched kernel of one shape over the queue in `a`.
cudaError_t launch_batch_fp32(int shape, const BatchArgs<float> &a, int blocks, cudaStream_t st);
cudaError_t launch_batch_bf16(int shape, const BatchArgs<__nv_bfloat16> &a, int blocks,
                              cudaStream_t st);
// Blocks of the batched kernel of a shape resident per SM.
int batch_resident(int shape, bool bf16);
cudaError_t launch_batch_advance(const BatchGraph *graphs, BatchState *state, int n_graphs,
                                 cudaStream_t st);
cudaError_t launch_batch_init(const BatchGraph *graphs, int n_graphs, bool bf16, int64_t max_elems,
                              cudaStream_t st);

}  // namespace f2v
