/*
 * f2v_batch.h -- the batched form: many independent graphs trained together,
 * one persistent kernel per epoch.
 *
 * Every graph of a batch runs exactly the method of f2v.h on its own: the
 * epochs of Algorithm 1 over its own minibatches of b consecutive ids, the
 * forces of Algorithm 2 from its own neighbours and negative samples (Eq. 5/6
 * or Eq. 8/9), the update of Eq. 10, its own Z0 and samples from its own
 * seed.  Graph g of a batch therefore computes what f2v_create on graph g
 * alone with the same seed computes, up to the order of the FP32 additions of
 * a vertex's gradient (pairs are summed in items of a tiling-dependent size
 * and combined in a fixed order, so a batch is bit-reproducible for a given
 * tiling).  The synchronous-minibatch rule (Sec. III-B) holds per graph:
 * minibatch k of graph g sees the updates of its minibatches < k and none of
 * its own; graphs never read each other's rows.
 *
 * An epoch of the whole batch is one launch of a persistent kernel (plus two
 * small memsets and a one-thread-per-graph epoch advance), replayed from a
 * captured CUDA graph.  The kernel's warps take work units from a queue in
 * which the minibatches of all graphs are interleaved (graph g's minibatch k
 * sits near position k / M_g of the epoch); a unit of minibatch k of graph g
 * starts once all units of its minibatch k - 1 have finished (a per-graph
 * minibatch barrier made of completion counters, with a bounded wait).
 *
 * Tiling.  A graph's rows are read by groups of L lanes (L * vector width =
 * d, so a warp works on 32 / L pairs at a time), and each group walks an
 * item of C consecutive force pairs of one minibatch.  L and C are chosen per
 * row size d, by default or by f2v_batch_autotune, which times candidate
 * tilings on the batch itself.
 *
 * Conventions are those of f2v.h (status codes, sticky failure, host arrays
 * copied before return, embedding layout, Philox keys), with these additions:
 *   - Graphs are given concatenated: graph g's row_ptr (n[g] + 1 entries,
 *     starting at 0, local column offsets) follows graph g-1's in `row_ptr`,
 *     and its col_idx entries (local vertex ids, row_ptr_g[n[g]] of them)
 *     follow graph g-1's in `col_idx`.  Each graph obeys the CSR rules of
 *     f2v_create.
 *   - Row sizes d[g] must be one of 2, 4, 8, 16, 32, 64, 128.
 *   - A batch owns a CUDA stream (created at f2v_batch_create unless one is
 *     given); every call enqueues on it and returns without waiting unless it
 *     says otherwise.
 */
#ifndef F2V_BATCH_H
#define F2V_BATCH_H

#include "f2v.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct f2v_batch f2v_batch;

/* Tiling of the graphs with row size d: lanes_per_row = L (a power of two,
   L * 4 == d or L * 2 == d), item_pairs = C (a multiple of 32, 32..8192). */
typedef struct {
    int32_t d;
    int32_t lanes_per_row;
    int32_t item_pairs;
} f2v_tiling;

/*
 * Creates a batch of num_graphs >= 1 graphs on the current CUDA device:
 * validates and copies the concatenated host CSRs (layout above), allocates
 * every graph's Z (two buffers of n[g] x d[g] in the storage precision, plus
 * an FP32 master in the BF16 form) and draws each Z0 from seed[g].  The
 * shared parameters follow f2v_create: model (F2V_TDIST or F2V_SIGMOID; the
 * other force models are single-graph only), 0 <= s <= 65534, lr > 0 finite
 * (constant schedule until f2v_batch_set_schedule), minibatch >= 1, and the
 * storage precision.  `stream` is a cudaStream_t or NULL (the batch then
 * creates its own non-blocking stream).  Epoch counters start at 0.
 * *out receives the batch (NULL on failure, with f2v_last_error_global set).
 */
f2v_status f2v_batch_create(int32_t num_graphs, const int32_t *n, const int32_t *d,
                            const uint64_t *seed, const int32_t *row_ptr,
                            const int32_t *col_idx, f2v_model model, int32_t s, float lr,
                            int32_t minibatch, f2v_precision precision, void *stream,
                            f2v_batch **out);

/* Waits for the batch's work and frees everything it owns.  NULL-safe. */
void f2v_batch_destroy(f2v_batch *b);

/* Runs one epoch of every graph (Algorithm 1 per graph), enqueued. */
f2v_status f2v_batch_epoch(f2v_batch *b);

/* Runs `epochs` consecutive epochs, enqueued. */
f2v_status f2v_batch_train(f2v_batch *b, int32_t epochs);

/* Runs the next `count` minibatch positions of the current epoch: for each
   position k, minibatch k of every graph that has one (graph g has
   ceil(n[g] / minibatch) of them).  After the last position of the largest
   graph the epoch ends for every graph.  Enqueued.  For checking a run
   minibatch by minibatch; f2v_batch_epoch finishes a begun epoch. */
f2v_status f2v_batch_run_minibatches(f2v_batch *b, int32_t count);

/* Epoch counter and next minibatch position of the current epoch. */
f2v_status f2v_batch_get_progress(const f2v_batch *b, int32_t *epoch, int32_t *minibatch);

/* Waits for the batch's stream; reports F2V_ETIMEOUT if a device-side wait
   ran out (the results of the epochs since the last check are then not
   valid, and the batch is sticky-failed). */
f2v_status f2v_batch_synchronize(f2v_batch *b);

/* Learning-rate schedule of every graph, as f2v_set_schedule; takes effect
   from the next epoch. */
f2v_status f2v_batch_set_lr(f2v_batch *b, float lr);
f2v_status f2v_batch_set_schedule(f2v_batch *b, f2v_schedule schedule, int32_t total_epochs);

/* Epoch counter (the same for every graph of the batch). */
f2v_status f2v_batch_get_epoch(const f2v_batch *b, int32_t *epoch);

/* Z of graph g as it stands (n[g] x d[g] FP32; the master in the BF16
   form) into host memory; `count` must equal n[g] * d[g].  Synchronous. */
f2v_status f2v_batch_get_embedding(f2v_batch *b, int32_t g, float *out, size_t count);

/* Z of every graph, concatenated in graph order (count = sum n[g] * d[g]). */
f2v_status f2v_batch_get_embeddings(f2v_batch *b, float *out, size_t count);

/* Overwrites Z of graph g from host FP32 rows (count = n[g] * d[g]); the BF16
   form stores the master as given and its rows rounded to nearest even.
   Only between epochs (F2V_ESTATE otherwise).  Synchronous. */
f2v_status f2v_batch_set_embedding(f2v_batch *b, int32_t g, const float *z, size_t count);

/* Sets the tiling of the graphs with row size t->d (F2V_EINVAL if no graph
   has it or the tiling is not valid for it); takes effect from the next
   epoch. */
f2v_status f2v_batch_set_tiling(f2v_batch *b, const f2v_tiling *t);
f2v_status f2v_batch_get_tiling(const f2v_batch *b, int32_t d, f2v_tiling *t);

/*
 * Chooses the tiling of every row size present by timing: for each d in
 * turn, every candidate (L in the shapes valid for d, C in 64, 128, 256,
 * 512, 1024) runs `epochs_per_candidate` >= 1 whole-batch epochs with the
 * other sizes' tilings fixed, and the fastest (CUDA events) is kept.  The
 * embeddings and epoch counter are restored afterwards, so tuning changes
 * no result beyond the summation order that the tiling fixes.  The chosen
 * tilings are applied and written to out[0 .. *count) (at most max_out,
 * ordered by d).  Synchronous.
 */
f2v_status f2v_batch_autotune(f2v_batch *b, int32_t epochs_per_candidate, f2v_tiling *out,
                              int32_t max_out, int32_t *count);

/* Force pairs of one epoch over all graphs (sum of nnz_g + n_g * s), and the
   algorithmic bytes of one epoch: sum of pairs_g * d_g * sizeof(storage). */
f2v_status f2v_batch_pairs_per_epoch(const f2v_batch *b, int64_t *pairs);
f2v_status f2v_batch_bytes_per_epoch(const f2v_batch *b, int64_t *bytes);

/* Device bytes held by the batch. */
f2v_status f2v_batch_device_bytes(const f2v_batch *b, size_t *bytes);

/* Number of graphs, and kernels launched so far (the epoch kernel and the
   epoch-advance kernel count one each per epoch). */
f2v_status f2v_batch_num_graphs(const f2v_batch *b, int32_t *num_graphs);
f2v_status f2v_batch_launch_count(const f2v_batch *b, int64_t *launches);

/* The batch's CUDA stream (a cudaStream_t). */
f2v_status f2v_batch_stream(const f2v_batch *b, void **stream);

/* Message of the last failure on this batch. */
const char *f2v_batch_last_error(const f2v_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* F2V_BATCH_H */
