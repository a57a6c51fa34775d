// f2v_batch_engine.h -- host side of the batched form: a set of independent
// graphs with their device state, the work tables of one epoch, and the
// captured CUDA graph that runs it.  Used by the f2v_batch_* entry points
// (a fixed set of graphs) and by the job server (graphs added and retired
// between epochs).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "f2v.h"
#include "f2v_internal.h"

namespace f2v {

// Tiling of one row size: the shape (index into kBatchShapes) and the pairs
// per item.
struct BatchTile {
    int shape = -1;
    int C = 0;
};

// Default shape of a row size (widest vectors), -1 if none.
int batch_default_shape(int d);
// Index of row size d in the per-size tables (0 for d = 2 ... 6 for d = 128),
// -1 if the batched form does not serve d.
int batch_size_index(int d);

class BatchEngine {
public:
    BatchEngine() = default;
    ~BatchEngine();
    BatchEngine(const BatchEngine &) = delete;
    BatchEngine &operator=(const BatchEngine &) = delete;

    // Binds to the current device and `stream` (NULL: a new non-blocking
    // stream the engine owns).
    f2v_status init(int model, int s, int b, bool bf16, cudaStream_t stream);

    // Adds a graph (validated host CSR, copied before return) whose Z0 is
    // drawn from `seed` on the engine's stream; returns its id (>= 0) or -1
    // with err() set.  The graph joins from the next epoch.
    int add_graph(const int32_t *row_ptr, const int32_t *col_idx, int n, int d, uint64_t seed,
                  float lr, int schedule, int total_epochs, f2v_status *st,
                  bool validated = false);
    // Removes a graph after the work enqueued so far (synchronises).
    f2v_status remove_graph(int id);

    // Enqueues `epochs` epochs of every graph present (an epoch already
    // begun with run_minibatches is finished first and counts as one).
    f2v_status run(int epochs);
    // Enqueues the next `count` minibatch positions of the current epoch:
    // minibatch k of every graph that has one, for k in [pos, pos + count);
    // at the last position of the longest graph the epoch ends for all.
    f2v_status run_minibatches(int count);
    int minibatch_position() const { return mb_pos_; }
    // Waits for the stream and checks the device error word.
    f2v_status sync();

    // Z of graph `id` (FP32 rows, the master in the BF16 form): to host
    // (synchronous) or from host (synchronous).
    f2v_status get_z(int id, float *out, size_t count);
    f2v_status set_z(int id, const float *z, size_t count);
    // Enqueues a device-to-host copy of Z of `id` into pinned host memory.
    f2v_status get_z_async(int id, float *out);

    f2v_status set_lr(int id, float lr, int schedule, int total_epochs);
    f2v_status set_tile(int d, const BatchTile &t);
    BatchTile tile(int d) const;
    f2v_status autotune(int epochs_per_candidate, std::vector<std::pair<int, BatchTile>> *out);

    int graph_epoch(int id) const;
    int graph_n(int id) const;
    int graph_d(int id) const;
    bool has_graph(int id) const;
    int num_graphs() const;
    int64_t pairs_per_epoch() const;     // over the graphs present
    int64_t bytes_per_epoch() const;     // pairs x d x storage bytes
    size_t device_bytes() const { return dev_bytes_; }
    int64_t launches() const { return launches_; }
    cudaStream_t stream() const { return stream_; }
    bool failed() const { return failed_; }
    const std::string &err() const { return err_; }
    f2v_status fail(f2v_status st, const char *fmt, ...);
    // Device bytes a graph of size (n, d, nnz) takes (its arrays, plus the
    // work tables and combine-tree scratch of its pairs): for admission.
    size_t graph_bytes(int64_t n, int d, int64_t nnz) const;
    size_t table_bytes(int64_t pairs, int64_t n, int d) const;

private:
    struct Graph {
        bool active = false;
        int n = 0, d = 0;
        int64_t nnz = 0;
        uint64_t seed = 0;
        float lr = 0.02f;
        int schedule = 0, total_epochs = 0;
        int epoch = 0, cur = 0;
        std::vector<int64_t> apair;
        void *mem = nullptr;
        size_t bytes = 0;
        BatchGraph dev{};
    };
    struct Queue {
        int shape = 0;
        int64_t unit_off = 0;
        int32_t n_units = 0;
        int blocks = 0;
        double weight = 0.0;
    };

    f2v_status rebuild(int k_lo, int k_hi);
    f2v_status capture(bool advance);
    f2v_status launch_range(int k_lo, int k_hi);
    f2v_status sync_current();
    int max_minibatches() const;
    f2v_status upload_params();
    f2v_status grow(void **p, size_t *cap, size_t bytes);
    void drop_graph_exec();

    int device_ = 0, sms_ = 1;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    int model_ = 0, s_ = 0, b_ = 1;
    bool bf16_ = false;
    BatchTile tiles_[7];

    std::vector<Graph> graphs_;
    std::vector<int> free_ids_;
    bool dirty_ = true;          // tables must be rebuilt
    int tab_lo_ = -1, tab_hi_ = -1;   // minibatch range the tables and graph cover
    int mb_pos_ = 0;             // next minibatch position of the current epoch
    bool params_dirty_ = false;  // lr / schedule / epoch changed

    // device tables
    BatchGraph *d_graphs_ = nullptr;
    BatchState *d_state_ = nullptr;
    BatchRec *d_recs_ = nullptr;
    BatchUnit *d_units_ = nullptr;
    int32_t *d_item_u0_ = nullptr;
    float *d_slots_ = nullptr;
    int32_t *d_cnt_ = nullptr;
    int32_t *d_done_ = nullptr;
    int32_t *d_next_ = nullptr;
    int32_t *d_err_ = nullptr;
    size_t cap_graphs_ = 0, cap_state_ = 0, cap_recs_ = 0, cap_units_ = 0, cap_items_ = 0,
           cap_slots_ = 0, cap_cnt_ = 0, cap_done_ = 0, cap_next_ = 0;
    std::vector<int> pos_;         // position in the device table -> graph id
    std::vector<Queue> queues_;
    int n_recs_ = 0;

    std::vector<cudaStream_t> side_;
    cudaEvent_t fork_ = nullptr;
    std::vector<cudaEvent_t> join_;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;

    size_t dev_bytes_ = 0;
    int64_t launches_ = 0;
    bool failed_ = false;
    std::string err_;
};

}  // namespace f2v
