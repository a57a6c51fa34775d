/*
 * f2v_serve.h -- the served form: a job server that embeds graphs as
 * requests arrive, with continuous batching.
 *
 * A job is one run of the method of f2v.h on one graph (Algorithm 1 for
 * `epochs` epochs, learning rate lr * (1 - e / epochs), its own seed).  The
 * server keeps every admitted job's CSR and Z resident on the device across
 * its epochs and steps all of them together: each step runs one epoch of
 * every job on the device, in the batched form of f2v_batch.h (jobs of the
 * same model, s, minibatch and precision share one persistent launch per row
 * shape; each such group has its own stream, so groups overlap too).  Between
 * steps it retires the jobs that reached their epoch count (their Z is copied
 * to the caller's buffer) and admits queued jobs, in arrival order, while the
 * device bytes of the admitted jobs stay within the budget and the number of
 * running jobs stays within max_active.  A job's result does not depend on
 * the other jobs it shared steps with: it is what a batch holding that graph
 * alone computes, bit for bit.
 *
 * The server runs its own host thread; the entry points may be called from
 * any thread.  Times are seconds since the server was created (steady
 * clock).  Row sizes d follow the batched form: 2, 4, 8, ..., 128.
 */
#ifndef F2V_SERVE_H
#define F2V_SERVE_H

#include "f2v.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct f2v_server f2v_server;

/* One embedding request.  row_ptr/col_idx (host, the CSR rules of
   f2v_create) and out (host, n * d floats) are owned by the caller and must
   stay valid and unchanged until the job is done or failed; the server reads
   the CSR once, when it admits the job, and writes out once, when the job
   completes (out then holds Z, row-major n x d FP32; the master in the BF16
   form). */
typedef struct {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    int32_t n, d;
    f2v_model model;        /* F2V_TDIST or F2V_SIGMOID */
    int32_t s;
    float lr;               /* eta_0; decayed linearly over `epochs` */
    int32_t minibatch;
    uint64_t seed;
    int32_t epochs;         /* >= 1 */
    f2v_precision precision;
    float *out;
} f2v_job;

typedef enum {
    F2V_JOB_QUEUED = 0,
    F2V_JOB_RUNNING = 1,
    F2V_JOB_DONE = 2,
    F2V_JOB_FAILED = 3
} f2v_job_state;

typedef struct {
    int32_t state;          /* f2v_job_state */
    int32_t epochs_done;
    double submit_s, admit_s, finish_s;   /* -1 until they happen */
    int64_t pairs;          /* force pairs of the job (epochs x per-epoch pairs) */
    size_t device_bytes;    /* bytes charged to the budget while running */
    f2v_status status;      /* F2V_OK, or why the job failed */
} f2v_job_info;

typedef struct {
    int64_t submitted, done, failed, running, queued;
    int64_t steps;          /* device steps run (one epoch of every running job) */
    int64_t pairs_done;     /* force pairs of all epochs run so far */
    size_t bytes_in_use, peak_bytes, budget;
    double busy_s;          /* time with at least one job running */
} f2v_server_stats;

/* Starts a server on the current CUDA device with a device-memory budget
   for admitted jobs (bytes, > 0) and at most max_active (>= 1) jobs
   running at once. */
f2v_status f2v_server_create(size_t budget_bytes, int32_t max_active, f2v_server **out);

/* Enqueues a job (validated on the calling thread: F2V_EINVAL for a bad
   graph or parameter, or a job larger than the whole budget) and returns its
   id (ids count from 0 in submission order).  A CSR this server has already
   validated (same row_ptr and col_idx pointers, n and nnz) is not checked
   again: the caller keeps a submitted graph unchanged. */
f2v_status f2v_server_submit(f2v_server *srv, const f2v_job *job, int64_t *id);

/* State and times of a job. */
f2v_status f2v_server_job(f2v_server *srv, int64_t id, f2v_job_info *info);

/* Blocks until job `id` is done or failed (returns its status). */
f2v_status f2v_server_wait(f2v_server *srv, int64_t id);

/* Blocks until every job submitted so far is done or failed. */
f2v_status f2v_server_wait_all(f2v_server *srv);

f2v_status f2v_server_get_stats(f2v_server *srv, f2v_server_stats *stats);

/* Stops the server: running jobs finish their current step and are marked
   failed with F2V_ESTATE, as are queued ones; frees everything.  NULL-safe. */
void f2v_server_destroy(f2v_server *srv);

/* Message of the last failure of a server call (or of job `id`'s failure,
   through f2v_server_job_error). */
const char *f2v_server_last_error(const f2v_server *srv);
const char *f2v_server_job_error(f2v_server *srv, int64_t id);

#ifdef __cplusplus
}
#endif

#endif /* F2V_SERVE_H */
