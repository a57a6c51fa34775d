/*
 * f2v.h -- C ABI of the GB300 Force2Vec epoch engine.
 *
 * Force2Vec (Rahman, Sujon, Azad, arXiv:2009.10035) embeds the vertices of an
 * undirected graph G(V, E) with 0/1 adjacency A (Sec. II-A) into Z in R^{n x d}
 * by minibatch SGD on the negative-sampling loss of Eq. 2.  Each epoch
 * (Algorithm 1) visits the vertices in minibatches V_b of b consecutive ids
 * (or, with F2V_FLAG_RANDOM_PARTITION, b consecutive positions of a new
 * random order); for every u in V_b it sums the attractive gradient over its
 * neighbours N(u) (or, for a context made by f2v_create_rw, over the
 * vertices of a random walk from u, Algorithm 3) and the repulsive gradient
 * over s negative samples (Algorithm 2), using Z as it stood when the
 * minibatch began, and then applies z_u -= eta * grad (Eq. 10).  The force
 * models (f2v_model below):
 *   F2V_TDIST    t-distribution similarity, Eq. 7; gradients Eq. 8 / Eq. 9
 *                times the unit vector (z_u - z_x)/t of Sec. III-B.  t^2 is
 *                floored at 1e-8 in the repulsive term.
 *   F2V_SIGMOID  sigmoid of the dot product, Eq. 3; gradients Eq. 5 / Eq. 6;
 *                after each update the coordinates of z_u are clamped to
 *                [-4, 4] (the paper is silent; unbounded, the summed
 *                gradients of high-degree vertices make the run diverge).
 *   F2V_FR, F2V_LINLOG, F2V_FORCEATLAS  the force laws of Table "diffmodels",
 *                with the same repulsion and clamp.
 *
 * Conventions shared by every entry point:
 *   - All functions return f2v_status and never abort.  A failure leaves a
 *     message readable through f2v_last_error (per context) or
 *     f2v_last_error_global (for f2v_create* before a context exists).
 *   - An invalid argument (a size out of range, a NULL buffer where one is
 *     required, a combination a form does not support) returns F2V_EINVAL
 *     before any device work and leaves the context usable.
 *   - A CUDA error inside a context makes it sticky-failed: every later call
 *     on it returns F2V_ESTATE until f2v_destroy.
 *   - Host arrays passed in stay owned by the caller and are copied before the
 *     call returns; device pointers passed in must stay valid only for the
 *     duration of the call (they are read on the context's stream, which the
 *     call synchronises unless stated otherwise).
 *   - Graph: symmetric CSR, int32 row_ptr[n+1] with row_ptr[0] = 0, monotone,
 *     row_ptr[n] = nnz < 2^31, and int32 col_idx[nnz] in [0, n).  Self-loops
 *     and duplicate entries are rejected (F2V_EINVAL); symmetry is the
 *     caller's responsibility (checked only with F2V_FLAG_CHECK_SYMMETRY).
 *   - Embedding layout: row-major n x d FP32, row u = z_u.
 *   - Randomness is counter-based Philox4x32-10 keyed by `seed`:
 *       initial z_u[j] = (Philox(ctr=(u, j, 0xFFFF, 0)).x0 >> 8) * 2^-24 - 0.5
 *       sample k of u in epoch e = Philox(ctr=(u, e, k, 0)).x0 mod n
 *     (key = (seed & 0xffffffff, seed >> 32)); a sample equal to u adds no
 *     force.  Results therefore depend only on the inputs and the epoch
 *     counter, and runs are bit-reproducible.
 *   - One context must not be used from two host threads at once.
 */
#ifndef F2V_H
#define F2V_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct f2v_ctx f2v_ctx;

typedef enum {
    F2V_OK = 0,
    F2V_EINVAL = 1,    /* invalid argument or graph */
    F2V_ENOMEM = 2,    /* device or host allocation failed */
    F2V_ECUDA = 3,     /* a CUDA call failed (context is now sticky-failed) */
    F2V_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    F2V_ESTATE = 5     /* context already failed, or call not valid now */
} f2v_status;

/* Force model.  F2V_TDIST: t-distribution, Eq. 8/9 times the unit vector
   (Sec. III-B).  F2V_SIGMOID: Eq. 5/6.  F2V_FR, F2V_LINLOG, F2V_FORCEATLAS:
   Fruchterman-Reingold, LinLog, ForceAtlas (Table "diffmodels"): the
   table's force on u along the unit vector (z_u - z_x)/t, t = |z_u - z_x|,
   is -t^2, -log(1 + t), -t for a neighbour and 1/t for a sample; Eq. 10
   steps against the gradient, so a pair adds minus that force times the
   unit vector: t (z_u - z_v), log(1 + t)/t (z_u - z_v), (z_u - z_v), and
   -(z_u - z_w)/t^2 for a sample (t^2 floored at 1e-8, as in the t model).
   Every model but F2V_TDIST bounds each coordinate of an updated row to
   [-4, 4] (their forces do not vanish with distance). */
typedef enum {
    F2V_TDIST = 0,
    F2V_SIGMOID = 1,
    F2V_FR = 2,
    F2V_LINLOG = 3,
    F2V_FORCEATLAS = 4
} f2v_model;

/* Storage of Z.  F2V_FP32: Z in FP32.  F2V_BF16: gathered rows stored in
   BF16 with an FP32 master copy; forces are accumulated and the update
   applied in FP32 against the master, and the BF16 rows are re-rounded
   (round-to-nearest-even) from it after each update. */
typedef enum { F2V_FP32 = 0, F2V_BF16 = 1 } f2v_precision;

/* Learning-rate schedule (Algorithm 1 gives eta = 0.02 as the initial rate).
   F2V_LR_CONSTANT: eta_e = lr.  F2V_LR_LINEAR: eta_e = lr * (1 - e / E) for a
   run of E = total_epochs epochs, e the epoch counter. */
typedef enum { F2V_LR_CONSTANT = 0, F2V_LR_LINEAR = 1 } f2v_schedule;

/* f2v_create_ex flags */
#define F2V_FLAG_CHECK_SYMMETRY 0x1u   /* reject a CSR that is not symmetric */
#define F2V_FLAG_NO_STAGING 0x2u       /* use the register-gather kernel even where
                                          the shared-memory staged one exists */
#define F2V_FLAG_SHARED_SAMPLES 0x4u   /* Algorithm 1's sampling step read
                                          literally: one set S_b of s negative
                                          samples per minibatch, used
                                          by every vertex of it (sample j of
                                          minibatch k in epoch e = Philox(key = seed,
                                          ctr = (k, e, j, 2)).x0 mod n; a sample equal
                                          to u adds no force).  Without it each vertex
                                          u draws its own s samples, ctr = (u, e, j, 0)
                                          (the O(nsd) cost of Sec. III-C). */
#define F2V_FLAG_RANDOM_PARTITION 0x8u /* Algorithm 1's partition step read
                                          literally: a new random partition of V
                                          every epoch.  Epoch e orders
                                          the vertices by Philox(key = seed, ctr =
                                          (v, e, 0, 3)).x0, ties by id; minibatch k is
                                          positions [k b, (k+1) b) of that order.
                                          Without it minibatch k is the ids
                                          [k b, (k+1) b) in every epoch.  Needs
                                          F2V_FP32.  Costs a sort, a relabelling of
                                          the CSR and a gather and scatter of Z per
                                          epoch. */

/*
 * Creates a context for one graph on the current CUDA device: validates and
 * copies the host CSR (row_ptr[n+1], col_idx[nnz]) to the device, allocates
 * Z and draws Z0 from `seed` (Sec. III-C, "Initialization").  n >= 1,
 * 1 <= d <= 1024, 0 <= s <= 65534, 1 <= minibatch, lr > 0 finite.
 * Epoch counter starts at 0, schedule F2V_LR_CONSTANT, precision FP32, the
 * legacy default stream.  *out receives the context (NULL on failure).
 */
f2v_status f2v_create(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                      f2v_model model, int32_t s, float lr, int32_t minibatch, uint64_t seed,
                      f2v_ctx **out);

/* As f2v_create, with a storage precision, flags (F2V_FLAG_*) and the CUDA
   stream (a cudaStream_t, may be NULL) all later work of the context is
   issued on. */
f2v_status f2v_create_ex(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                         f2v_model model, int32_t s, float lr, int32_t minibatch,
                         uint64_t seed, f2v_precision precision, uint32_t flags,
                         void *stream, f2v_ctx **out);

/*
 * rForce2Vec (Sec. III-C, Algorithm 3): as f2v_create_ex, but in every epoch
 * N(u) is formed by a random walk of walk_length steps from u (1 <=
 * walk_length <= 1024) instead of u's neighbours; the force model, the
 * negative samples and the update are unchanged.  Step i (0-based) of the
 * walk from u in epoch e moves from the current vertex w (initially u) to
 * col_idx[row_ptr[w] + Philox4x32-10(key = seed, ctr = (u, e, i, 1)).x0 mod
 * deg(w)].  Every step is one attractive pair, repeats included; a step that
 * lands on u exerts no force (as a negative sample equal to u); a walk that
 * reaches a vertex without out-neighbours (only possible in a CSR that is
 * not symmetric) stops, its remaining steps exerting no force.  Vertex u's
 * pairs are its walk_length steps (none if u has no neighbours), then its s
 * negative samples, so an epoch has walk_length * |{u : deg(u) > 0}| + n * s
 * pairs.  Walks are drawn on the device once per epoch, one thread per vertex.
 */
f2v_status f2v_create_rw(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                         f2v_model model, int32_t s, int32_t walk_length, float lr,
                         int32_t minibatch, uint64_t seed, f2v_precision precision,
                         uint32_t flags, void *stream, f2v_ctx **out);

/* Frees every device and host resource of the context.  NULL is a no-op. */
void f2v_destroy(f2v_ctx *ctx);

/*
 * Runs one epoch of Algorithm 1 at the current epoch counter e with
 * eta_e from the schedule, then increments e.  (If minibatches of epoch e
 * were already run with f2v_run_minibatches, only the remaining ones run.)
 * The work is enqueued on the context's stream; the call returns without
 * waiting for it (errors of the enqueued kernels surface on the next
 * synchronising call).
 */
f2v_status f2v_epoch(f2v_ctx *ctx);

/* Runs `epochs` consecutive epochs (as f2v_epoch repeated). */
f2v_status f2v_train(f2v_ctx *ctx, int32_t epochs);

/* Runs the next `count` minibatches (V_b = ids [k*b, min((k+1)*b, n)) for
   k = 0, 1, ... within each epoch), crossing into the next epoch when one
   ends.  Every other call sees Z as of the last minibatch run. */
f2v_status f2v_run_minibatches(f2v_ctx *ctx, int32_t count);

/* Current epoch counter and the index of the next minibatch within it. */
f2v_status f2v_get_progress(const f2v_ctx *ctx, int32_t *epoch, int32_t *minibatch);

/* Waits for all work of the context; reports any device error. */
f2v_status f2v_synchronize(f2v_ctx *ctx);

/* Copies Z (n*d FP32, row-major; the FP32 master in the BF16 form) to host
   memory `out` of `count` floats; count must equal n*d.  Synchronous. */
f2v_status f2v_get_embedding(f2v_ctx *ctx, float *out, size_t count);

/* As f2v_get_embedding into device memory `dev_out`, enqueued on the
   context's stream without waiting. */
f2v_status f2v_get_embedding_device(f2v_ctx *ctx, float *dev_out, size_t count);

/* Replaces Z by the host array `z` (n*d FP32).  In the BF16 form the master
   takes z and the BF16 rows its rounding.  Synchronous. */
f2v_status f2v_set_embedding(f2v_ctx *ctx, const float *z, size_t count);

f2v_status f2v_set_lr(f2v_ctx *ctx, float lr);
f2v_status f2v_set_schedule(f2v_ctx *ctx, f2v_schedule schedule, int32_t total_epochs);
/* Sets the epoch counter (selects the negative samples and eta of the next
   epoch, which starts at its first minibatch from the current Z); with
   f2v_set_embedding it resumes a run bit-identically. */
f2v_status f2v_set_epoch(f2v_ctx *ctx, int32_t epoch);
f2v_status f2v_get_epoch(const f2v_ctx *ctx, int32_t *epoch);

/* Switches the context to another CUDA stream (a cudaStream_t, may be NULL).
   Work already enqueued on the old stream is waited for first. */
f2v_status f2v_set_stream(f2v_ctx *ctx, void *stream);

/*
 * Link-prediction AUC of the current Z on held-out pairs: pos_pairs[2*npos]
 * and neg_pairs[2*nneg] are host int32 (u, v) pairs.  Score of a pair:
 * z_u . z_v (sigmoid model) or -||z_u - z_v||^2 (the other models), in FP64
 * from the stored rows on the device; AUC = (#{pos > neg} + #{pos == neg}/2)
 * / (npos * nneg), with the counts reduced exactly in integers.  Synchronous.
 */
f2v_status f2v_eval_auc(f2v_ctx *ctx, const int32_t *pos_pairs, int64_t npos,
                        const int32_t *neg_pairs, int64_t nneg, double *auc);

/*
 * The loss of Eq. 2 on the current Z, in FP64 on the device: *loss = the sum
 * over all vertices u of L(u) = sum over the neighbours v of u (the CSR as
 * given to f2v_create) of -log delta(z_u, z_v), plus the sum over u's s
 * negative samples w of epoch `epoch` (Philox(ctr = (u, epoch, k, 0)).x0 mod
 * n, k < s; a sample equal to u adds nothing) of -log(1 - delta(z_u, z_w)).
 * delta is Eq. 3's sigma(z_u . z_x) for the sigmoid model and Eq. 7's
 * 1/(1 + |z_u - z_x|^2) for the t model, with |z_u - z_w|^2 floored at 1e-8
 * in the repulsive term as in training.  Rows are read as stored (the FP32
 * master in the BF16 form) and every product, sum and logarithm is FP64;
 * the pairs are summed in a fixed order, so the result is reproducible.
 * F2V_EINVAL for the other force models (the paper gives no loss for them)
 * or epoch < 0.  Synchronous.
 */
f2v_status f2v_eval_loss(f2v_ctx *ctx, int32_t epoch, double *loss);

/* Negative samples the device draws in epoch `epoch`: out[u*s + k] for all
   u < n, k < s (count must equal n*s).  With F2V_FLAG_SHARED_SAMPLES row u
   is the set of u's minibatch in that epoch (under F2V_FLAG_RANDOM_PARTITION,
   the minibatch of u's position in the epoch's order).  For checking;
   synchronous. */
f2v_status f2v_debug_samples(f2v_ctx *ctx, int32_t epoch, int32_t *out, size_t count);

/*
 * Link prediction as in Sec. IV ("Link prediction"), on the current Z, in
 * FP64 on the device.  Pair i of the combined list (pos_pairs[2*npos] with
 * label 1, then neg_pairs[2*nneg] with label 0; host int32 (u, v)) has the
 * Hadamard features x_i = z_u * z_v (element by element); train_mask[npos +
 * nneg] (host, nonzero = training pair) splits the list.  An L2-regularised
 * logistic regression, theta = (w, b) minimising sum_i log(1 + exp(-s_i
 * (w . x_i + b))) + |w|^2 / 2 over the training pairs (s_i = +-1, the
 * intercept unpenalised), is fitted by Newton's method until a step's
 * max-norm is below 1e-10 or after 100 steps; *accuracy = (TP + TN) / (test
 * pairs), a pair predicted positive when w . x + b > 0.  theta (d + 1
 * doubles, w then b) is written if not NULL.  Needs d <= 150 and at least
 * one training and one test pair.  Synchronous.
 */
f2v_status f2v_eval_link_lr(f2v_ctx *ctx, const int32_t *pos_pairs, int64_t npos,
                            const int32_t *neg_pairs, int64_t nneg, const uint8_t *train_mask,
                            double *accuracy, double *theta);

/*
 * Clustering as in Sec. IV ("Clustering"), on the current Z, in FP64 on the
 * device: Lloyd's k-means from the centres z_{init[c]} (host, k vertex ids,
 * 1 <= k <= 64, d <= 256), a vertex joining its nearest centre (the lowest
 * index on a tie), a centre moving to its cluster's mean (an empty cluster
 * keeps its centre), until no label changes or after `iters` rounds.
 * labels[n] (host, may be NULL) receives the clusters; *modularity the
 * modularity of the clustering on the context's graph, sum_c [e_c / nnz -
 * (D_c / nnz)^2] with e_c the CSR entries inside cluster c and D_c its summed
 * degree; *rounds (may be NULL) the rounds run.  Synchronous.
 */
f2v_status f2v_eval_kmeans(f2v_ctx *ctx, int32_t k, const int32_t *init, int32_t iters,
                           int32_t *labels, double *modularity, int32_t *rounds);

/*
 * A test of the device's bounded waits, which end every wait of the force
 * kernels (rows of earlier minibatches, completion counters, TMA
 * mbarriers).  One warp waits, with the same primitives and error codes,
 * on: kind 0 a flag it has set itself (returns F2V_OK); kind 1 a row flag
 * nothing sets; kind 2 a completion counter nothing increments; kind 3 an
 * mbarrier nothing arrives on.  Kinds 1-3 run out after about a second and
 * return F2V_ETIMEOUT, which, as after any timed-out epoch, leaves the
 * context failed (F2V_ESTATE from then on); the device itself stays usable.
 * Synchronous.
 */
f2v_status f2v_debug_wait(f2v_ctx *ctx, int32_t kind);

/* Walks the device draws in epoch `epoch` (contexts made by f2v_create_rw):
   out[u*walk_length + i] is the vertex step i of u's walk reaches, or -1
   where the step exerts no force (u has no neighbours, the walk has
   stopped, or the step lands on u).  count must equal n*walk_length.  The
   walks come from the same kernel and list the force launches read.  For
   checking; synchronous. */
f2v_status f2v_debug_walks(f2v_ctx *ctx, int32_t epoch, int32_t *out, size_t count);

/* Force pairs of one epoch: nnz + n*s (Sec. III-C complexity: O(md + nsd));
   rForce2Vec: walk_length * |{u : deg(u) > 0}| + n*s (O(nkd + nsd)). */
f2v_status f2v_pairs_per_epoch(const f2v_ctx *ctx, int64_t *pairs);

/* Device bytes held by the context. */
f2v_status f2v_device_bytes(const f2v_ctx *ctx, size_t *bytes);

/* Number of kernels the context has launched so far. */
f2v_status f2v_launch_count(const f2v_ctx *ctx, int64_t *launches);

/*
 * Per-launch timing of the force kernel: when enabled, every force-kernel
 * launch is bracketed by CUDA events on the context's stream.  Reading
 * (synchronous) returns the number of timed launches and their summed
 * duration in milliseconds, and resets both.
 */
f2v_status f2v_set_kernel_timing(f2v_ctx *ctx, int32_t enable);
f2v_status f2v_read_kernel_timing(f2v_ctx *ctx, int64_t *launches, double *total_ms);

/*
 * One minibatch of an epoch on caller-owned device buffers, allocating
 * nothing.  (The paper has no counterpart: this exists for callers that
 * cannot allocate device memory while the step runs -- software that owns
 * all device memory through its own allocator or arena and forbids libraries
 * from calling cudaMalloc, or that plans its memory for the whole run up
 * front -- and therefore cannot use f2v_create, which allocates.)
 *
 * All pointers are device memory owned by the caller: the CSR (row_ptr[n+1],
 * col_idx[nnz], with the rules of f2v_create, not re-checked here) and the
 * two FP32 embedding buffers (n x d, row-major).  z_cur and z_next must
 * start on a 16-byte boundary (8 bytes is enough for d = 2, and 4 for a d
 * that is not a power of two from 4 to 1024), and row_ptr and col_idx on a
 * 4-byte boundary: the kernel moves rows with vector loads and stores, so
 * the call returns F2V_EINVAL, before any device work, for a pointer that
 * is not aligned.  It computes, for the
 * vertices u in [mb_begin, mb_end), the same update as a context's epoch
 * `epoch` (negative samples from `seed`, learning rate `eta`): partner rows
 * v < mb_begin are read from z_next (already updated this epoch) and all
 * other rows, the minibatch's own included, from z_cur; the new rows are
 * written to z_next[mb_begin..mb_end).  Other rows of z_next are untouched.
 * A caller runs the minibatches of an epoch in order and then swaps the
 * buffers.  Work is enqueued on `stream` (a cudaStream_t, may be NULL); the
 * call waits on that stream once, to read the minibatch's pair count.
 *
 * Scratch lives in one fixed 8 MiB device array inside the library, which
 * every device that loads the library keeps until the process exits.  A
 * minibatch fits if about 8 * (mb_end - mb_begin + 33) + 4 * (mb_end -
 * mb_begin) + (9 * d + 5) * ceil(pairs / 32) bytes stay within it (pairs =
 * sum over the minibatch of max(deg(u) + s, 1)); for d = 128 that is about
 * 7,000 pairs per 1 MiB, so a 4096-vertex minibatch of average degree 30
 * fits.  Larger minibatches return F2V_EINVAL with the caller's buffers
 * untouched.  All
 * calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads on the same device) race and give wrong
 * results.  The first call on each device looks up the array's address with
 * that device current; make it before any stream capture.  The address is
 * kept until the process exits, so after a cudaDeviceReset on a device this
 * entry point must not be called on that device again.  Errors are read
 * with f2v_noalloc_last_error.
 */
f2v_status f2v_minibatch_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                                 int32_t d, f2v_model model, int32_t s, float eta, uint64_t seed,
                                 int32_t epoch, int32_t mb_begin, int32_t mb_end,
                                 const float *z_cur, float *z_next, void *stream);

/* Message of the last f2v_minibatch_noalloc failure on this thread. */
const char *f2v_noalloc_last_error(void);

/* Message of the last failure on this context ("" if none). */
const char *f2v_last_error(const f2v_ctx *ctx);

/* Message of the last failure of a call that had no context (thread-local). */
const char *f2v_last_error_global(void);

#ifdef __cplusplus
}
#endif

#endif /* F2V_H */
