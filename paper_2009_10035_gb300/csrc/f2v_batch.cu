// f2v_batch.cu -- host side of the batched form (include/f2v_batch.h): the
// graphs' device state, the work tables of an epoch, the captured epoch
// graph, the tiling autotuner, and the f2v_batch_* entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <atomic>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "f2v.h"
#include "f2v_batch.h"
#include "f2v_batch_engine.h"
#include "f2v_device.cuh"
#include "f2v_internal.h"

namespace f2v {

int batch_resident_fp32(int shape);
int batch_resident_bf16(int shape);

int batch_resident(int shape, bool bf16)
{
    return bf16 ? batch_resident_bf16(shape) : batch_resident_fp32(shape);
}

namespace {

// eta_e in the same double arithmetic as the host (IEEE division and
// multiplication), rounded to FP32.
__device__ double batch_eta_dev(float lr, int schedule, int total_epochs, int e)
{
    if (schedule == 1 && total_epochs > 0)
        return (double)lr * (1.0 - (double)e / (double)total_epochs);
    return (double)lr;
}

__global__ void batch_advance_kernel(const BatchGraph *graphs, BatchState *state, int n_graphs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_graphs) return;
    BatchState st = state[i];
    st.epoch += 1;
    st.cur ^= 1;
    const BatchGraph &g = graphs[i];
    st.eta = (float)batch_eta_dev(g.lr, g.schedule, g.total_epochs, (int)st.epoch);
    state[i] = st;
}

// Z0 of one graph (the formula of the single-graph context), into buffer 0
// (and the FP32 master in the BF16 form).
template <typename Ts>
__global__ void batch_init_kernel(Ts *z, float *master, int64_t n, int d, uint32_t k0, uint32_t k1)
{
    const int64_t total = n * (int64_t)d;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float v = z0_value((uint32_t)(t / d), (uint32_t)(t % d), k0, k1);
        if constexpr (sizeof(Ts) == 2) {
            z[t] = __float2bfloat16_rn(v);
            master[t] = v;
        } else {
            z[t] = v;
        }
    }
}

__global__ void batch_round_kernel(__nv_bfloat16 *z, const float *master, int64_t total)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        z[t] = __float2bfloat16_rn(master[t]);
}

// Expands the records of an epoch into the start vertex of every item (the
// vertex holding pair P0 + i C, found by binary search over the minibatch's
// pair prefix) and the warp units of every record, at the offsets the host
// assigned.
__global__ void batch_expand_kernel(const BatchGraph *graphs, const BatchRec *recs, int R,
                                    int32_t *item_u0, BatchUnit *units)
{
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const BatchRec rec = recs[r];
        const int64_t *ap = graphs[rec.g].apair;
        for (int i = threadIdx.x; i < rec.n_items; i += blockDim.x) {
            const int64_t q = rec.P0 + (int64_t)i * rec.C;
            int lo = rec.mb_begin, hi = rec.mb_end - 1;   // largest u with apair[u] <= q
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ap[mid] <= q)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            item_u0[rec.item_off + i] = lo;
        }
        for (int w = threadIdx.x; w < rec.n_wunits; w += blockDim.x)
            units[rec.unit_off + w] = BatchUnit{r, w * rec.gsize};
    }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int grid_for(int64_t elems)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((elems + 255) / 256, 4096));
}

}  // namespace

int batch_size_index(int d)
{
    switch (d) {
        case 2: return 0;
        case 4: return 1;
        case 8: return 2;
        case 16: return 3;
        case 32: return 4;
        case 64: return 5;
        case 128: return 6;
        default: return -1;
    }
}

int batch_default_shape(int d)
{
    for (int i = 0; i < kNumBatchShapes; ++i)
        if (kBatchShapes[i].d == d) return i;     // listed widest vectors first
    return -1;
}

namespace {
// Default pairs per item: long enough to amortise the item's set-up, short
// enough that a minibatch of b vertices spreads over many groups.
int default_item_pairs(int d) { return d <= 8 ? 128 : 256; }

// Relative GPU time of one pair in a shape's kernel, used to split the SMs
// between the concurrent launches of an epoch so that they end together.
// Measured on the 4,096-graph SBM workload with each row size alone (ps per
// pair on the whole GPU): one-lane shapes (L = 1, eight pairs in flight per
// lane) ~19; wider shapes a shared decode plus the row, ~30 + d.
double pair_cost(int shape)
{
    const BatchShape &s = kBatchShapes[shape];
    return s.L == 1 ? 19.0 : 30.0 + (double)s.d;
}
}  // namespace

BatchEngine::~BatchEngine()
{
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device_);
    if (stream_) cudaStreamSynchronize(stream_);
    drop_graph_exec();
    for (Graph &g : graphs_)
        if (g.mem) cudaFree(g.mem);
    void *bufs[] = {d_graphs_, d_state_, d_recs_, d_units_, d_item_u0_, d_slots_,
                    d_cnt_,    d_done_,  d_next_, d_err_};
    for (void *p : bufs)
        if (p) cudaFree(p);
    for (cudaStream_t s : side_) cudaStreamDestroy(s);
    for (cudaEvent_t e : join_) cudaEventDestroy(e);
    if (fork_) cudaEventDestroy(fork_);
    if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    if (prev >= 0) cudaSetDevice(prev);
}

f2v_status BatchEngine::fail(f2v_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err_ = buf;
    if (st == F2V_ECUDA || st == F2V_ETIMEOUT) failed_ = true;
    return st;
}

#define ENG_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? F2V_ENOMEM : F2V_ECUDA,           \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                   \
    } while (0)

f2v_status BatchEngine::init(int model, int s, int b, bool bf16, cudaStream_t stream)
{
    model_ = model;
    s_ = s;
    b_ = b;
    bf16_ = bf16;
    ENG_CUDA(cudaGetDevice(&device_));
    cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device_);
    sms_ = std::max(sms_, 1);
    if (stream) {
        stream_ = stream;
    } else {
        ENG_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
        own_stream_ = true;
    }
    ENG_CUDA(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
    ENG_CUDA(cudaMalloc(&d_err_, 16));
    dev_bytes_ += 16;
    ENG_CUDA(cudaMemsetAsync(d_err_, 0, sizeof(int32_t), stream_));
    for (int i = 0; i < 7; ++i) {
        const int d = 2 << i;
        tiles_[i].shape = batch_default_shape(d);
        tiles_[i].C = default_item_pairs(d);
    }
    return F2V_OK;
}

size_t BatchEngine::graph_bytes(int64_t n, int d, int64_t nnz) const
{
    const size_t es = bf16_ ? 2 : 4;
    size_t b = align256((size_t)(n + 1) * 4) + align256((size_t)std::max<int64_t>(nnz, 1) * 4) +
               align256((size_t)(n + 1) * 8) + 2 * align256((size_t)n * d * es) +
               align256((size_t)n * 4);
    if (bf16_) b += align256((size_t)n * d * 4);
    return b;
}

size_t BatchEngine::table_bytes(int64_t pairs, int64_t n, int d) const
{
    // items (4 B) and up to two slot rows per item, records per minibatch,
    // warp units: bounded with the smallest item size in use
    int Cmin = 8192;
    for (const BatchTile &t : tiles_) Cmin = std::min(Cmin, std::max(t.C, 32));
    const int64_t items = pairs / Cmin + (n + b_ - 1) / b_ + 1;
    return (size_t)items * (4 + 8 + 2 * 2 * (size_t)d * 4 + 16) +
           (size_t)((n + b_ - 1) / b_ + 1) * (sizeof(BatchRec) + 4);
}

int BatchEngine::add_graph(const int32_t *row_ptr, const int32_t *col_idx, int n, int d,
                           uint64_t seed, float lr, int schedule, int total_epochs,
                           f2v_status *st, bool validated)
{
    *st = F2V_OK;
    if (failed_) {
        *st = F2V_ESTATE;
        return -1;
    }
    if (n < 1) {
        *st = fail(F2V_EINVAL, "n = %d, must be >= 1", n);
        return -1;
    }
    if (batch_size_index(d) < 0) {
        *st = fail(F2V_EINVAL, "d = %d: the batched form serves d in {2, 4, 8, 16, 32, 64, 128}", d);
        return -1;
    }
    if (!(lr > 0.f) || !std::isfinite(lr)) {
        *st = fail(F2V_EINVAL, "lr must be finite and > 0");
        return -1;
    }
    if (schedule == 1 && total_epochs < 1) {
        *st = fail(F2V_EINVAL, "linear schedule needs total_epochs >= 1");
        return -1;
    }
    if (!validated) {
        f2v_status vs = check_csr(row_ptr, col_idx, n, 0);
        if (vs != F2V_OK) {
            *st = fail(vs, "%s", global_error().c_str());
            return -1;
        }
    }
    Graph g;
    g.n = n;
    g.d = d;
    g.nnz = row_ptr[n];
    g.seed = seed;
    g.lr = lr;
    g.schedule = schedule;
    g.total_epochs = total_epochs;
    try {
        g.apair.assign((size_t)n + 1, 0);
    } catch (const std::bad_alloc &) {
        *st = fail(F2V_ENOMEM, "host allocation failed");
        return -1;
    }
    for (int u = 0; u < n; ++u) {
        int64_t c = (int64_t)(row_ptr[u + 1] - row_ptr[u]) + s_;
        if (c == 0) c = 1;     // the empty pair: the row is still carried over
        g.apair[(size_t)u + 1] = g.apair[(size_t)u] + c;
    }
    const int M = (n + b_ - 1) / b_;
    for (int k = 0; k < M; ++k) {
        const int u0 = k * b_, u1 = std::min(n, u0 + b_);
        if (g.apair[(size_t)u1] - g.apair[(size_t)u0] >= (int64_t)INT32_MAX - 8192) {
            *st = fail(F2V_EINVAL, "a minibatch holds 2^31 or more force pairs");
            return -1;
        }
    }
    g.bytes = graph_bytes(n, d, g.nnz);
    cudaError_t ce = cudaMalloc(&g.mem, g.bytes);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        *st = fail(F2V_ENOMEM, "cudaMalloc(%zu bytes): %s", g.bytes, cudaGetErrorString(ce));
        return -1;
    }
    const size_t es = bf16_ ? 2 : 4;
    char *p = static_cast<char *>(g.mem);
    int32_t *d_rp = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)(n + 1) * 4);
    int32_t *d_ci = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)std::max<int64_t>(g.nnz, 1) * 4);
    int64_t *d_ap = reinterpret_cast<int64_t *>(p);
    p += align256((size_t)(n + 1) * 8);
    void *z0 = p;
    p += align256((size_t)n * d * es);
    void *z1 = p;
    p += align256((size_t)n * d * es);
    int32_t *cnt = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)n * 4);
    float *master = nullptr;
    if (bf16_) master = reinterpret_cast<float *>(p);
    g.dev.row_ptr = d_rp;
    g.dev.col_idx = d_ci;
    g.dev.apair = d_ap;
    g.dev.z[0] = z0;
    g.dev.z[1] = z1;
    g.dev.master = master;
    g.dev.counter = cnt;
    g.dev.n = n;
    g.dev.d = d;
    g.dev.shape = 0;
    g.dev.key0 = (uint32_t)(seed & 0xffffffffu);
    g.dev.key1 = (uint32_t)(seed >> 32);
    g.dev.lr = lr;
    g.dev.schedule = schedule;
    g.dev.total_epochs = total_epochs;

    auto bail = [&](cudaError_t e) {
        cudaGetLastError();
        cudaFree(g.mem);
        *st = fail(F2V_ECUDA, "graph upload: %s", cudaGetErrorString(e));
        return -1;
    };
    if ((ce = cudaMemcpyAsync(d_rp, row_ptr, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice,
                              stream_)) != cudaSuccess)
        return bail(ce);
    if (g.nnz > 0 && (ce = cudaMemcpyAsync(d_ci, col_idx, (size_t)g.nnz * 4,
                                           cudaMemcpyHostToDevice, stream_)) != cudaSuccess)
        return bail(ce);
    if ((ce = cudaMemcpyAsync(d_ap, g.apair.data(), (size_t)(n + 1) * 8, cudaMemcpyHostToDevice,
                              stream_)) != cudaSuccess)
        return bail(ce);
    if ((ce = cudaMemsetAsync(cnt, 0, (size_t)n * 4, stream_)) != cudaSuccess) return bail(ce);
    const int64_t elems = (int64_t)n * d;
    if (bf16_)
        batch_init_kernel<__nv_bfloat16><<<grid_for(elems), 256, 0, stream_>>>(
            (__nv_bfloat16 *)z0, master, n, d, g.dev.key0, g.dev.key1);
    else
        batch_init_kernel<float><<<grid_for(elems), 256, 0, stream_>>>((float *)z0, nullptr, n, d,
                                                                       g.dev.key0, g.dev.key1);
    if ((ce = cudaGetLastError()) != cudaSuccess) return bail(ce);
    // the host copies above read pageable memory before returning; the
    // apair upload reads g.apair, which stays alive with the graph
    ++launches_;
    g.active = true;
    dev_bytes_ += g.bytes;
    int id;
    if (!free_ids_.empty()) {
        id = free_ids_.back();
        free_ids_.pop_back();
        graphs_[(size_t)id] = std::move(g);
    } else {
        id = (int)graphs_.size();
        graphs_.push_back(std::move(g));
    }
    dirty_ = true;
    return id;
}

f2v_status BatchEngine::remove_graph(int id)
{
    if (!has_graph(id)) return fail(F2V_EINVAL, "no graph %d", id);
    ENG_CUDA(cudaStreamSynchronize(stream_));
    Graph &g = graphs_[(size_t)id];
    ENG_CUDA(cudaFree(g.mem));
    dev_bytes_ -= g.bytes;
    g = Graph();
    free_ids_.push_back(id);
    dirty_ = true;
    return F2V_OK;
}

bool BatchEngine::has_graph(int id) const
{
    return id >= 0 && (size_t)id < graphs_.size() && graphs_[(size_t)id].active;
}
int BatchEngine::graph_epoch(int id) const { return has_graph(id) ? graphs_[(size_t)id].epoch : -1; }
int BatchEngine::graph_n(int id) const { return has_graph(id) ? graphs_[(size_t)id].n : 0; }
int BatchEngine::graph_d(int id) const { return has_graph(id) ? graphs_[(size_t)id].d : 0; }

int BatchEngine::num_graphs() const
{
    int c = 0;
    for (const Graph &g : graphs_) c += g.active;
    return c;
}

int64_t BatchEngine::pairs_per_epoch() const
{
    int64_t p = 0;
    for (const Graph &g : graphs_)
        if (g.active) p += g.apair.back();
    return p;
}

int64_t BatchEngine::bytes_per_epoch() const
{
    const int64_t es = bf16_ ? 2 : 4;
    int64_t b = 0;
    for (const Graph &g : graphs_)
        if (g.active) b += g.apair.back() * g.d * es;
    return b;
}

f2v_status BatchEngine::grow(void **p, size_t *cap, size_t bytes)
{
    bytes = std::max<size_t>(bytes, 16);
    if (*p && *cap >= bytes) return F2V_OK;
    if (*p) {
        ENG_CUDA(cudaStreamSynchronize(stream_));
        cudaFree(*p);
        dev_bytes_ -= *cap;
        *p = nullptr;
        *cap = 0;
    }
    const size_t want = bytes + bytes / 4;     // headroom for later additions
    ENG_CUDA(cudaMalloc(p, want));
    *cap = want;
    dev_bytes_ += want;
    return F2V_OK;
}

void BatchEngine::drop_graph_exec()
{
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
}

// Builds the records, queues and items of one epoch over the graphs
// present, uploads them, and captures the epoch graph.
int BatchEngine::max_minibatches() const
{
    int m = 0;
    for (const Graph &g : graphs_)
        if (g.active) m = std::max(m, (g.n + b_ - 1) / b_);
    return m;
}

f2v_status BatchEngine::rebuild(int k_lo, int k_hi)
{
    drop_graph_exec();
    tab_lo_ = k_lo;
    tab_hi_ = k_hi;
    pos_.clear();
    for (size_t i = 0; i < graphs_.size(); ++i)
        if (graphs_[i].active) pos_.push_back((int)i);
    const int P = (int)pos_.size();
    queues_.clear();
    n_recs_ = 0;
    dirty_ = false;
    params_dirty_ = false;
    if (P == 0) return F2V_OK;

    std::vector<BatchGraph> hg((size_t)P);
    std::vector<BatchState> hs((size_t)P);
    std::vector<BatchRec> recs;
    std::vector<double> keys;
    int64_t slot_total = 0, cnt_total = 0, item_total = 0;
    try {
        for (int p = 0; p < P; ++p) {
            Graph &g = graphs_[(size_t)pos_[(size_t)p]];
            const BatchTile &t = tiles_[batch_size_index(g.d)];
            g.dev.shape = t.shape;
            hg[(size_t)p] = g.dev;
            hs[(size_t)p] = BatchState{(uint32_t)g.epoch, g.cur,
                                       (float)batch_eta(g.lr, g.schedule, g.total_epochs, g.epoch),
                                       0};
            const int G = 32 / kBatchShapes[t.shape].L;
            const int C = t.C;
            const int M = (g.n + b_ - 1) / b_;
            for (int k = k_lo; k < std::min(M, k_hi); ++k) {
                const int u0 = k * b_, u1 = std::min(g.n, u0 + b_);
                const int64_t P0 = g.apair[(size_t)u0], P1 = g.apair[(size_t)u1];
                BatchRec r{};
                r.P0 = P0;
                r.g = p;
                r.mb_begin = u0;
                r.mb_end = u1;
                r.Pk = (int32_t)(P1 - P0);
                r.C = C;
                r.n_items = (int32_t)((P1 - P0 + C - 1) / C);
                r.item_off = (int32_t)std::min<int64_t>(item_total, INT32_MAX);
                item_total += r.n_items;
                r.n_wunits = (r.n_items + G - 1) / G;
                r.gsize = G;
                r.prev = (k > k_lo) ? (int32_t)recs.size() - 1 : -1;
                // combine-tree scratch of this minibatch (see f2v_internal.h)
                r.slot_off = slot_total;
                r.cnt_off = cnt_total;
                if (r.n_items > 1) {
                    int64_t units = r.n_items, lvl_slots = 0, lvl_cnt = 0;
                    for (int l = 0; l < kMaxLevels && units > 0; ++l) {
                        lvl_slots += 2 * units;
                        if (l > 0) lvl_cnt += 2 * units;
                        if (units == 1) break;
                        units = (units + kFan - 1) / kFan;
                    }
                    slot_total += lvl_slots * g.d;
                    cnt_total += lvl_cnt + 2;
                }
                recs.push_back(r);
                keys.push_back((double)k / (double)M);
            }
        }
    } catch (const std::bad_alloc &) {
        return fail(F2V_ENOMEM, "host allocation failed (batch tables)");
    }
    if (item_total >= (int64_t)INT32_MAX)
        return fail(F2V_EINVAL, "the batch holds 2^31 or more items; use a larger item size");
    n_recs_ = (int)recs.size();

    // one queue per shape present: its records by k / M_g, then graph; the
    // records' warp units are laid out in that order
    int64_t unit_total = 0;
    for (int sh = 0; sh < kNumBatchShapes; ++sh) {
        std::vector<int> rs;
        double weight = 0.0;
        for (int i = 0; i < n_recs_; ++i)
            if (hg[(size_t)recs[(size_t)i].g].shape == sh) {
                rs.push_back(i);
                weight += (double)recs[(size_t)i].Pk * pair_cost(sh);
            }
        if (rs.empty()) continue;
        std::stable_sort(rs.begin(), rs.end(), [&](int a, int b) {
            if (keys[(size_t)a] != keys[(size_t)b]) return keys[(size_t)a] < keys[(size_t)b];
            return recs[(size_t)a].g < recs[(size_t)b].g;
        });
        Queue q;
        q.shape = sh;
        q.unit_off = unit_total;
        q.weight = weight;
        for (int i : rs) {
            BatchRec &r = recs[(size_t)i];
            r.unit_off = (int32_t)std::min<int64_t>(unit_total, INT32_MAX);
            unit_total += r.n_wunits;
        }
        q.n_units = (int32_t)std::min<int64_t>(unit_total - q.unit_off, INT32_MAX);
        queues_.push_back(q);
    }
    if (unit_total >= (int64_t)INT32_MAX)
        return fail(F2V_EINVAL, "the batch holds 2^31 or more work units; use a larger item size");
    // grids: every launch of the epoch runs at once, sized by its share of
    // the work, so each graph's minibatches spread over the whole epoch
    double wsum = 0.0;
    for (const Queue &q : queues_) wsum += q.weight;
    for (Queue &q : queues_) {
        const int res = std::max(1, batch_resident(q.shape, bf16_));
        const int full = sms_ * res;
        int blocks = (int)std::lround(full * (wsum > 0 ? q.weight / wsum : 1.0));
        blocks = std::max(blocks, std::max(1, sms_ / 8));
        const int useful = (int)std::min<int64_t>((q.n_units + 7) / 8, full);
        q.blocks = std::max(1, std::min(blocks, useful));
    }

    f2v_status st;
    const size_t R = recs.size();
    if ((st = grow((void **)&d_graphs_, &cap_graphs_, sizeof(BatchGraph) * P)) != F2V_OK) return st;
    if ((st = grow((void **)&d_state_, &cap_state_, sizeof(BatchState) * P)) != F2V_OK) return st;
    if ((st = grow((void **)&d_recs_, &cap_recs_, sizeof(BatchRec) * R)) != F2V_OK) return st;
    if ((st = grow((void **)&d_units_, &cap_units_, sizeof(BatchUnit) * (size_t)unit_total)) != F2V_OK) return st;
    if ((st = grow((void **)&d_item_u0_, &cap_items_, sizeof(int32_t) * (size_t)item_total)) != F2V_OK) return st;
    if ((st = grow((void **)&d_slots_, &cap_slots_, sizeof(float) * (size_t)slot_total)) != F2V_OK) return st;
    if ((st = grow((void **)&d_cnt_, &cap_cnt_, sizeof(int32_t) * (size_t)cnt_total)) != F2V_OK) return st;
    if ((st = grow((void **)&d_done_, &cap_done_, sizeof(int32_t) * R)) != F2V_OK) return st;
    if ((st = grow((void **)&d_next_, &cap_next_, sizeof(int32_t) * queues_.size())) != F2V_OK) return st;
    ENG_CUDA(cudaMemcpyAsync(d_graphs_, hg.data(), sizeof(BatchGraph) * P, cudaMemcpyHostToDevice, stream_));
    ENG_CUDA(cudaMemcpyAsync(d_state_, hs.data(), sizeof(BatchState) * P, cudaMemcpyHostToDevice, stream_));
    ENG_CUDA(cudaMemcpyAsync(d_recs_, recs.data(), sizeof(BatchRec) * R, cudaMemcpyHostToDevice, stream_));
    ENG_CUDA(cudaMemsetAsync(d_cnt_, 0, std::max<size_t>(16, sizeof(int32_t) * (size_t)cnt_total), stream_));
    if (R > 0) {
        batch_expand_kernel<<<(int)std::min<size_t>(R, 8192), 128, 0, stream_>>>(
            d_graphs_, d_recs_, (int)R, d_item_u0_, d_units_);
        ENG_CUDA(cudaGetLastError());
        ++launches_;
    }
    // pageable sources: the copies have read them when they return
    return capture(k_hi >= max_minibatches());
}

f2v_status BatchEngine::capture(bool advance)
{
    while (side_.size() < queues_.size()) {
        cudaStream_t s;
        ENG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        side_.push_back(s);
        cudaEvent_t e;
        ENG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        join_.push_back(e);
    }
    const int P = (int)pos_.size();
    ENG_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) {
        if (e == cudaSuccess && r != cudaSuccess) e = r;
    };
    step(cudaMemsetAsync(d_done_, 0, sizeof(int32_t) * (size_t)std::max(n_recs_, 1), stream_));
    step(cudaMemsetAsync(d_next_, 0, sizeof(int32_t) * std::max<size_t>(queues_.size(), 1), stream_));
    step(cudaEventRecord(fork_, stream_));
    for (size_t i = 0; i < queues_.size(); ++i) {
        const Queue &q = queues_[i];
        step(cudaStreamWaitEvent(side_[i], fork_, 0));
        if (bf16_) {
            BatchArgs<__nv_bfloat16> a{d_graphs_, d_state_, d_recs_, d_units_ + q.unit_off,
                                       d_item_u0_, d_slots_, d_cnt_, d_done_, d_next_ + i,
                                       q.n_units, P, s_, model_, d_err_};
            step(launch_batch_bf16(q.shape, a, q.blocks, side_[i]));
        } else {
            BatchArgs<float> a{d_graphs_, d_state_, d_recs_, d_units_ + q.unit_off, d_item_u0_,
                               d_slots_, d_cnt_, d_done_, d_next_ + i, q.n_units, P, s_,
                               model_, d_err_};
            step(launch_batch_fp32(q.shape, a, q.blocks, side_[i]));
        }
        step(cudaEventRecord(join_[i], side_[i]));
        step(cudaStreamWaitEvent(stream_, join_[i], 0));
    }
    if (advance) {
        batch_advance_kernel<<<(P + 255) / 256, 256, 0, stream_>>>(d_graphs_, d_state_, P);
        step(cudaGetLastError());
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(stream_, &g);
    if (e == cudaSuccess) e = ee;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(F2V_ECUDA, "capturing the epoch graph: %s", cudaGetErrorString(e));
    }
    graph_ = g;
    ENG_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
    return F2V_OK;
}

f2v_status BatchEngine::upload_params()
{
    const int P = (int)pos_.size();
    std::vector<BatchGraph> hg((size_t)P);
    std::vector<BatchState> hs((size_t)P);
    for (int p = 0; p < P; ++p) {
        Graph &g = graphs_[(size_t)pos_[(size_t)p]];
        hg[(size_t)p] = g.dev;
        hs[(size_t)p] = BatchState{(uint32_t)g.epoch, g.cur,
                                   (float)batch_eta(g.lr, g.schedule, g.total_epochs, g.epoch), 0};
    }
    if (P > 0) {
        ENG_CUDA(cudaMemcpyAsync(d_graphs_, hg.data(), sizeof(BatchGraph) * P, cudaMemcpyHostToDevice, stream_));
        ENG_CUDA(cudaMemcpyAsync(d_state_, hs.data(), sizeof(BatchState) * P, cudaMemcpyHostToDevice, stream_));
    }
    params_dirty_ = false;
    return F2V_OK;
}

// Runs minibatch positions [k_lo, k_hi) of the current epoch (one replay of
// the graph for that range; the epoch ends if k_hi is the last position).
f2v_status BatchEngine::launch_range(int k_lo, int k_hi)
{
    f2v_status st;
    if (dirty_ || tab_lo_ != k_lo || tab_hi_ != k_hi) {
        if ((st = rebuild(k_lo, k_hi)) != F2V_OK) return st;
    } else if (params_dirty_) {
        if ((st = upload_params()) != F2V_OK) return st;
    }
    if (!exec_) return F2V_OK;
    ENG_CUDA(cudaGraphLaunch(exec_, stream_));
    const bool ends = k_hi >= max_minibatches();
    launches_ += (int64_t)queues_.size() + (ends ? 1 : 0);
    mb_pos_ = ends ? 0 : k_hi;
    if (ends) {
        for (int id : pos_) {
            Graph &g = graphs_[(size_t)id];
            g.epoch += 1;
            g.cur ^= 1;
        }
    }
    return F2V_OK;
}

f2v_status BatchEngine::run(int epochs)
{
    if (failed_) return F2V_ESTATE;
    if (epochs < 0) return fail(F2V_EINVAL, "epochs = %d", epochs);
    if (epochs == 0 || num_graphs() == 0) return F2V_OK;
    f2v_status st;
    const int M = max_minibatches();
    if (mb_pos_ > 0) {
        if ((st = launch_range(mb_pos_, M)) != F2V_OK) return st;
        --epochs;
    }
    for (int e = 0; e < epochs; ++e)
        if ((st = launch_range(0, M)) != F2V_OK) return st;
    return F2V_OK;
}

f2v_status BatchEngine::run_minibatches(int count)
{
    if (failed_) return F2V_ESTATE;
    if (count < 0) return fail(F2V_EINVAL, "count = %d", count);
    if (num_graphs() == 0) return F2V_OK;
    const int M = max_minibatches();
    while (count > 0) {
        const int hi = std::min(M, mb_pos_ + count);
        count -= hi - mb_pos_;
        f2v_status st = launch_range(mb_pos_, hi);
        if (st != F2V_OK) return st;
    }
    return F2V_OK;
}

// Mid-epoch, rows of graph g's finished minibatches live in its next buffer:
// copy them into the current one so that it holds Z as it stands.
f2v_status BatchEngine::sync_current()
{
    if (mb_pos_ == 0) return F2V_OK;
    const size_t es = bf16_ ? 2 : 4;
    for (const Graph &g : graphs_) {
        if (!g.active) continue;
        const size_t rows = std::min<size_t>((size_t)mb_pos_ * b_, (size_t)g.n);
        if (rows == 0) continue;
        ENG_CUDA(cudaMemcpyAsync(g.dev.z[g.cur], g.dev.z[g.cur ^ 1], rows * g.d * es,
                                 cudaMemcpyDeviceToDevice, stream_));
    }
    return F2V_OK;
}

f2v_status BatchEngine::sync()
{
    if (failed_) return F2V_ESTATE;
    ENG_CUDA(cudaStreamSynchronize(stream_));
    int32_t w = 0;
    ENG_CUDA(cudaMemcpy(&w, d_err_, sizeof w, cudaMemcpyDeviceToHost));
    if (w != 0)
        return fail(F2V_ETIMEOUT, "a device-side minibatch barrier wait timed out (code %d); "
                                  "results of the last epochs are not valid", w);
    return F2V_OK;
}

f2v_status BatchEngine::get_z(int id, float *out, size_t count)
{
    if (failed_) return F2V_ESTATE;
    if (!has_graph(id)) return fail(F2V_EINVAL, "no graph %d", id);
    const Graph &g = graphs_[(size_t)id];
    if (!out || count != (size_t)g.n * g.d)
        return fail(F2V_EINVAL, "count = %zu, expected n*d = %zu", count, (size_t)g.n * g.d);
    f2v_status st = sync_current();
    if (st == F2V_OK) st = sync();
    if (st != F2V_OK) return st;
    const void *src = bf16_ ? (const void *)g.dev.master : g.dev.z[g.cur];
    ENG_CUDA(cudaMemcpy(out, src, count * sizeof(float), cudaMemcpyDeviceToHost));
    return F2V_OK;
}

f2v_status BatchEngine::get_z_async(int id, float *out)
{
    if (failed_) return F2V_ESTATE;
    if (!has_graph(id)) return fail(F2V_EINVAL, "no graph %d", id);
    f2v_status st = sync_current();
    if (st != F2V_OK) return st;
    const Graph &g = graphs_[(size_t)id];
    const void *src = bf16_ ? (const void *)g.dev.master : g.dev.z[g.cur];
    ENG_CUDA(cudaMemcpyAsync(out, src, (size_t)g.n * g.d * sizeof(float), cudaMemcpyDeviceToHost,
                             stream_));
    return F2V_OK;
}

f2v_status BatchEngine::set_z(int id, const float *z, size_t count)
{
    if (failed_) return F2V_ESTATE;
    if (!has_graph(id)) return fail(F2V_EINVAL, "no graph %d", id);
    const Graph &g = graphs_[(size_t)id];
    if (!z || count != (size_t)g.n * g.d)
        return fail(F2V_EINVAL, "count = %zu, expected n*d = %zu", count, (size_t)g.n * g.d);
    if (mb_pos_ != 0)
        return fail(F2V_ESTATE, "an embedding can be set only between epochs");
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(z[i])) return fail(F2V_EINVAL, "z[%zu] is not finite", i);
    if (bf16_) {
        ENG_CUDA(cudaMemcpyAsync(g.dev.master, z, count * 4, cudaMemcpyHostToDevice, stream_));
        batch_round_kernel<<<grid_for((int64_t)count), 256, 0, stream_>>>(
            (__nv_bfloat16 *)g.dev.z[g.cur], g.dev.master, (int64_t)count);
        ENG_CUDA(cudaGetLastError());
        ++launches_;
    } else {
        ENG_CUDA(cudaMemcpyAsync(g.dev.z[g.cur], z, count * 4, cudaMemcpyHostToDevice, stream_));
    }
    return sync();
}

f2v_status BatchEngine::set_lr(int id, float lr, int schedule, int total_epochs)
{
    if (!has_graph(id)) return fail(F2V_EINVAL, "no graph %d", id);
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(F2V_EINVAL, "lr must be finite and > 0");
    if (schedule == 1 && total_epochs < 1)
        return fail(F2V_EINVAL, "linear schedule needs total_epochs >= 1");
    Graph &g = graphs_[(size_t)id];
    g.lr = lr;
    g.schedule = schedule;
    g.total_epochs = total_epochs;
    g.dev.lr = lr;
    g.dev.schedule = schedule;
    g.dev.total_epochs = total_epochs;
    params_dirty_ = true;
    return F2V_OK;
}

f2v_status BatchEngine::set_tile(int d, const BatchTile &t)
{
    const int i = batch_size_index(d);
    if (i < 0) return fail(F2V_EINVAL, "d = %d has no batched shapes", d);
    if (t.shape < 0 || t.shape >= kNumBatchShapes || kBatchShapes[t.shape].d != d)
        return fail(F2V_EINVAL, "shape not valid for d = %d", d);
    if (t.C < 32 || t.C > 8192 || t.C % 32 != 0)
        return fail(F2V_EINVAL, "item_pairs = %d, must be a multiple of 32 in [32, 8192]", t.C);
    if (tiles_[i].shape != t.shape || tiles_[i].C != t.C) {
        tiles_[i] = t;
        dirty_ = true;
    }
    return F2V_OK;
}

BatchTile BatchEngine::tile(int d) const
{
    const int i = batch_size_index(d);
    return i < 0 ? BatchTile{} : tiles_[i];
}

f2v_status BatchEngine::autotune(int epochs_per_candidate,
                                 std::vector<std::pair<int, BatchTile>> *out)
{
    if (failed_) return F2V_ESTATE;
    if (epochs_per_candidate < 1) return fail(F2V_EINVAL, "epochs_per_candidate must be >= 1");
    if (mb_pos_ != 0) return fail(F2V_ESTATE, "autotune runs only between epochs");
    f2v_status st = sync();
    if (st != F2V_OK) return st;
    // snapshot every graph's Z (and master) and epoch state
    std::vector<int> ids;
    for (size_t i = 0; i < graphs_.size(); ++i)
        if (graphs_[i].active) ids.push_back((int)i);
    const size_t es = bf16_ ? 2 : 4;
    size_t snap_bytes = 0;
    for (int id : ids) {
        const Graph &g = graphs_[(size_t)id];
        snap_bytes += align256((size_t)g.n * g.d * es) + (bf16_ ? align256((size_t)g.n * g.d * 4) : 0);
    }
    void *snap = nullptr;
    ENG_CUDA(cudaMalloc(&snap, std::max<size_t>(snap_bytes, 16)));
    struct Saved { int epoch, cur; size_t off; };
    std::vector<Saved> saved;
    size_t off = 0;
    for (int id : ids) {
        const Graph &g = graphs_[(size_t)id];
        const size_t zb = (size_t)g.n * g.d * es;
        saved.push_back({g.epoch, g.cur, off});
        cudaMemcpyAsync((char *)snap + off, g.dev.z[g.cur], zb, cudaMemcpyDeviceToDevice, stream_);
        off += align256(zb);
        if (bf16_) {
            cudaMemcpyAsync((char *)snap + off, g.dev.master, (size_t)g.n * g.d * 4,
                            cudaMemcpyDeviceToDevice, stream_);
            off += align256((size_t)g.n * g.d * 4);
        }
    }
    auto restore = [&]() -> cudaError_t {
        for (size_t i = 0; i < ids.size(); ++i) {
            Graph &g = graphs_[(size_t)ids[i]];
            g.epoch = saved[i].epoch;
            g.cur = saved[i].cur;
            size_t o = saved[i].off;
            const size_t zb = (size_t)g.n * g.d * es;
            cudaError_t e = cudaMemcpyAsync(g.dev.z[g.cur], (char *)snap + o, zb,
                                            cudaMemcpyDeviceToDevice, stream_);
            if (e != cudaSuccess) return e;
            o += align256(zb);
            if (bf16_) {
                e = cudaMemcpyAsync(g.dev.master, (char *)snap + o, (size_t)g.n * g.d * 4,
                                    cudaMemcpyDeviceToDevice, stream_);
                if (e != cudaSuccess) return e;
            }
        }
        params_dirty_ = true;
        return cudaSuccess;
    };
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    auto time_current = [&](float *ms) -> f2v_status {
        cudaError_t e = restore();
        if (e != cudaSuccess) return fail(F2V_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
        f2v_status s2;
        const int M = max_minibatches();
        if ((dirty_ || tab_lo_ != 0 || tab_hi_ != M) && (s2 = rebuild(0, M)) != F2V_OK) return s2;
        if (params_dirty_ && (s2 = upload_params()) != F2V_OK) return s2;
        cudaEventRecord(t0, stream_);
        if ((s2 = run(epochs_per_candidate)) != F2V_OK) return s2;
        cudaEventRecord(t1, stream_);
        if ((s2 = sync()) != F2V_OK) return s2;
        cudaEventElapsedTime(ms, t0, t1);
        return F2V_OK;
    };
    std::vector<int> sizes;
    for (int id : ids) {
        const int d = graphs_[(size_t)id].d;
        if (std::find(sizes.begin(), sizes.end(), d) == sizes.end()) sizes.push_back(d);
    }
    std::sort(sizes.begin(), sizes.end());
    const int Cs[] = {64, 128, 256, 512, 1024};
    for (int d : sizes) {
        BatchTile best = tile(d);
        float best_ms = 0.f;
        if ((st = time_current(&best_ms)) != F2V_OK) break;
        for (int sh = 0; sh < kNumBatchShapes && st == F2V_OK; ++sh) {
            if (kBatchShapes[sh].d != d) continue;
            for (int C : Cs) {
                BatchTile t{sh, C};
                if (t.shape == best.shape && t.C == best.C) continue;
                if ((st = set_tile(d, t)) != F2V_OK) break;
                float ms = 0.f;
                if ((st = time_current(&ms)) != F2V_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
        }
        if (st != F2V_OK) break;
        set_tile(d, best);
        if (out) out->push_back({d, best});
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st == F2V_OK) {
        cudaError_t e = restore();
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
        if (e != cudaSuccess) st = fail(F2V_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
    }
    cudaStreamSynchronize(stream_);
    cudaFree(snap);
    return st;
}

}  // namespace f2v

// ---- f2v_batch_* entry points ------------------------------------------------

using namespace f2v;

struct f2v_batch {
    BatchEngine eng;
    std::vector<int> ids;       // graph g -> engine id
    float lr = 0.02f;
    int schedule = 0, total_epochs = 0;
    bool bf16 = false;
};

namespace {

f2v_status gfail(f2v_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_global_error(buf);
    return st;
}

#define BATCH_CHECK(b)                                                  \
    do {                                                                \
        if (!(b)) return gfail(F2V_EINVAL, "null batch");               \
        if ((b)->eng.failed()) return F2V_ESTATE;                       \
    } while (0)

}  // namespace

extern "C" {

f2v_status f2v_batch_create(int32_t num_graphs, const int32_t *n, const int32_t *d,
                            const uint64_t *seed, const int32_t *row_ptr,
                            const int32_t *col_idx, f2v_model model, int32_t s, float lr,
                            int32_t minibatch, f2v_precision precision, void *stream,
                            f2v_batch **out)
{
    if (!out) return gfail(F2V_EINVAL, "out is NULL");
    *out = nullptr;
    set_global_error("");
    if (num_graphs < 1) return gfail(F2V_EINVAL, "num_graphs = %d, must be >= 1", num_graphs);
    if (!n || !d || !seed || !row_ptr) return gfail(F2V_EINVAL, "n, d, seed and row_ptr must not be NULL");
    if (s < 0 || s > 65534) return gfail(F2V_EINVAL, "s = %d, must be in [0, 65534]", s);
    if (minibatch < 1) return gfail(F2V_EINVAL, "minibatch = %d, must be >= 1", minibatch);
    if (!(lr > 0.f) || !std::isfinite(lr)) return gfail(F2V_EINVAL, "lr must be finite and > 0");
    if (model != F2V_TDIST && model != F2V_SIGMOID) return gfail(F2V_EINVAL, "unknown model %d", (int)model);
    if (precision != F2V_FP32 && precision != F2V_BF16) return gfail(F2V_EINVAL, "unknown precision %d", (int)precision);
    for (int g = 0; g < num_graphs; ++g) {
        if (n[g] < 1) return gfail(F2V_EINVAL, "graph %d: n = %d, must be >= 1", g, n[g]);
        if (batch_size_index(d[g]) < 0)
            return gfail(F2V_EINVAL, "graph %d: d = %d; the batched form serves d in {2, 4, 8, 16, 32, 64, 128}", g, d[g]);
    }
    f2v_batch *b = new (std::nothrow) f2v_batch();
    if (!b) return gfail(F2V_ENOMEM, "host allocation failed");
    b->lr = lr;
    b->bf16 = (precision == F2V_BF16);
    f2v_status st = b->eng.init((int)model, s, minibatch, b->bf16, (cudaStream_t)stream);
    if (st != F2V_OK) {
        gfail(st, "%s", b->eng.err().c_str());
        delete b;
        return st;
    }
    // offsets of every graph, then every CSR checked, graphs spread over the
    // host threads (one thread per graph)
    std::vector<int64_t> roffs((size_t)num_graphs + 1, 0), coffs((size_t)num_graphs + 1, 0);
    for (int g = 0; g < num_graphs; ++g) {
        roffs[(size_t)g + 1] = roffs[(size_t)g] + (int64_t)n[g] + 1;
        coffs[(size_t)g + 1] = coffs[(size_t)g] + row_ptr[roffs[(size_t)g] + n[g]];
        if (coffs[(size_t)g + 1] > coffs[(size_t)g] && !col_idx) {
            delete b;
            return gfail(F2V_EINVAL, "graph %d: col_idx is NULL", g);
        }
    }
    {
        std::vector<std::string> msgs((size_t)num_graphs);
        std::vector<f2v_status> sts((size_t)num_graphs, F2V_OK);
        std::atomic<int> next{0};
        auto work = [&]() {
            for (int g; (g = next.fetch_add(1)) < num_graphs;)
                sts[(size_t)g] = check_csr_quiet(row_ptr + roffs[(size_t)g],
                                                 col_idx ? col_idx + coffs[(size_t)g] : nullptr,
                                                 n[g], 0, 1, &msgs[(size_t)g]);
        };
        const int nt = (int)std::max<unsigned>(1, std::min<unsigned>(
                                                       16, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 1; t < std::min(nt, num_graphs); ++t) pool.emplace_back(work);
        work();
        for (auto &th : pool) th.join();
        for (int g = 0; g < num_graphs; ++g)
            if (sts[(size_t)g] != F2V_OK) {
                delete b;
                return gfail(sts[(size_t)g], "graph %d: %s", g, msgs[(size_t)g].c_str());
            }
    }
    int64_t roff = 0, coff = 0;
    for (int g = 0; g < num_graphs; ++g) {
        const int32_t *rp = row_ptr + roff;
        const int64_t nnz = rp[n[g]];
        const int id = b->eng.add_graph(rp, col_idx ? col_idx + coff : nullptr, n[g], d[g], seed[g],
                                        lr, 0, 0, &st, /*validated=*/true);
        if (id < 0) {
            gfail(st, "graph %d: %s", g, b->eng.err().c_str());
            delete b;
            return st;
        }
        b->ids.push_back(id);
        roff += (int64_t)n[g] + 1;
        coff += nnz;
    }
    st = b->eng.sync();
    if (st != F2V_OK) {
        gfail(st, "%s", b->eng.err().c_str());
        delete b;
        return st;
    }
    *out = b;
    return F2V_OK;
}

void f2v_batch_destroy(f2v_batch *b) { delete b; }

f2v_status f2v_batch_epoch(f2v_batch *b) { return f2v_batch_train(b, 1); }

f2v_status f2v_batch_train(f2v_batch *b, int32_t epochs)
{
    BATCH_CHECK(b);
    if (epochs < 0) return b->eng.fail(F2V_EINVAL, "epochs = %d", epochs);
    return b->eng.run(epochs);
}

f2v_status f2v_batch_run_minibatches(f2v_batch *b, int32_t count)
{
    BATCH_CHECK(b);
    return b->eng.run_minibatches(count);
}

f2v_status f2v_batch_get_progress(const f2v_batch *b, int32_t *epoch, int32_t *minibatch)
{
    if (!b || !epoch || !minibatch) return gfail(F2V_EINVAL, "null argument");
    *epoch = b->eng.graph_epoch(b->ids[0]);
    *minibatch = b->eng.minibatch_position();
    return F2V_OK;
}

f2v_status f2v_batch_synchronize(f2v_batch *b)
{
    BATCH_CHECK(b);
    return b->eng.sync();
}

f2v_status f2v_batch_set_lr(f2v_batch *b, float lr)
{
    BATCH_CHECK(b);
    for (int id : b->ids) {
        f2v_status st = b->eng.set_lr(id, lr, b->schedule, b->total_epochs);
        if (st != F2V_OK) return st;
    }
    b->lr = lr;
    return F2V_OK;
}

f2v_status f2v_batch_set_schedule(f2v_batch *b, f2v_schedule schedule, int32_t total_epochs)
{
    BATCH_CHECK(b);
    if (schedule != F2V_LR_CONSTANT && schedule != F2V_LR_LINEAR)
        return b->eng.fail(F2V_EINVAL, "unknown schedule %d", (int)schedule);
    for (int id : b->ids) {
        f2v_status st = b->eng.set_lr(id, b->lr, (int)schedule, total_epochs);
        if (st != F2V_OK) return st;
    }
    b->schedule = (int)schedule;
    b->total_epochs = total_epochs;
    return F2V_OK;
}

f2v_status f2v_batch_get_epoch(const f2v_batch *b, int32_t *epoch)
{
    if (!b || !epoch) return gfail(F2V_EINVAL, "null argument");
    *epoch = b->eng.graph_epoch(b->ids[0]);
    return F2V_OK;
}

f2v_status f2v_batch_get_embedding(f2v_batch *b, int32_t g, float *out, size_t count)
{
    BATCH_CHECK(b);
    if (g < 0 || g >= (int)b->ids.size()) return b->eng.fail(F2V_EINVAL, "graph %d out of range", g);
    return b->eng.get_z(b->ids[(size_t)g], out, count);
}

f2v_status f2v_batch_get_embeddings(f2v_batch *b, float *out, size_t count)
{
    BATCH_CHECK(b);
    size_t total = 0;
    for (int id : b->ids) total += (size_t)b->eng.graph_n(id) * b->eng.graph_d(id);
    if (!out || count != total)
        return b->eng.fail(F2V_EINVAL, "count = %zu, expected %zu", count, total);
    f2v_status st = b->eng.sync();
    if (st != F2V_OK) return st;
    size_t off = 0;
    for (int id : b->ids) {
        st = b->eng.get_z_async(id, out + off);
        if (st != F2V_OK) return st;
        off += (size_t)b->eng.graph_n(id) * b->eng.graph_d(id);
    }
    return b->eng.sync();
}

f2v_status f2v_batch_set_embedding(f2v_batch *b, int32_t g, const float *z, size_t count)
{
    BATCH_CHECK(b);
    if (g < 0 || g >= (int)b->ids.size()) return b->eng.fail(F2V_EINVAL, "graph %d out of range", g);
    return b->eng.set_z(b->ids[(size_t)g], z, count);
}

f2v_status f2v_batch_set_tiling(f2v_batch *b, const f2v_tiling *t)
{
    BATCH_CHECK(b);
    if (!t) return b->eng.fail(F2V_EINVAL, "tiling is NULL");
    bool present = false;
    for (int id : b->ids) present |= (b->eng.graph_d(id) == t->d);
    if (!present) return b->eng.fail(F2V_EINVAL, "no graph of the batch has d = %d", t->d);
    int shape = -1;
    for (int i = 0; i < kNumBatchShapes; ++i)
        if (kBatchShapes[i].d == t->d && kBatchShapes[i].L == t->lanes_per_row) shape = i;
    if (shape < 0)
        return b->eng.fail(F2V_EINVAL, "lanes_per_row = %d is not a shape of d = %d",
                           t->lanes_per_row, t->d);
    return b->eng.set_tile(t->d, BatchTile{shape, t->item_pairs});
}

f2v_status f2v_batch_get_tiling(const f2v_batch *b, int32_t d, f2v_tiling *t)
{
    if (!b || !t) return gfail(F2V_EINVAL, "null argument");
    const BatchTile bt = b->eng.tile(d);
    if (bt.shape < 0) return gfail(F2V_EINVAL, "d = %d has no batched shapes", d);
    t->d = d;
    t->lanes_per_row = kBatchShapes[bt.shape].L;
    t->item_pairs = bt.C;
    return F2V_OK;
}

f2v_status f2v_batch_autotune(f2v_batch *b, int32_t epochs_per_candidate, f2v_tiling *out,
                              int32_t max_out, int32_t *count)
{
    BATCH_CHECK(b);
    std::vector<std::pair<int, BatchTile>> chosen;
    f2v_status st = b->eng.autotune(epochs_per_candidate, &chosen);
    if (st != F2V_OK) return st;
    int c = 0;
    for (const auto &p : chosen) {
        if (out && c < max_out) {
            out[c].d = p.first;
            out[c].lanes_per_row = kBatchShapes[p.second.shape].L;
            out[c].item_pairs = p.second.C;
        }
        ++c;
    }
    if (count) *count = std::min(c, std::max(max_out, 0));
    return F2V_OK;
}

f2v_status f2v_batch_pairs_per_epoch(const f2v_batch *b, int64_t *pairs)
{
    if (!b || !pairs) return gfail(F2V_EINVAL, "null argument");
    *pairs = b->eng.pairs_per_epoch();
    return F2V_OK;
}

f2v_status f2v_batch_bytes_per_epoch(const f2v_batch *b, int64_t *bytes)
{
    if (!b || !bytes) return gfail(F2V_EINVAL, "null argument");
    *bytes = b->eng.bytes_per_epoch();
    return F2V_OK;
}

f2v_status f2v_batch_device_bytes(const f2v_batch *b, size_t *bytes)
{
    if (!b || !bytes) return gfail(F2V_EINVAL, "null argument");
    *bytes = b->eng.device_bytes();
    return F2V_OK;
}

f2v_status f2v_batch_num_graphs(const f2v_batch *b, int32_t *num_graphs)
{
    if (!b || !num_graphs) return gfail(F2V_EINVAL, "null argument");
    *num_graphs = (int32_t)b->ids.size();
    return F2V_OK;
}

f2v_status f2v_batch_launch_count(const f2v_batch *b, int64_t *launches)
{
    if (!b || !launches) return gfail(F2V_EINVAL, "null argument");
    *launches = b->eng.launches();
    return F2V_OK;
}

f2v_status f2v_batch_stream(const f2v_batch *b, void **stream)
{
    if (!b || !stream) return gfail(F2V_EINVAL, "null argument");
    *stream = (void *)b->eng.stream();
    return F2V_OK;
}

const char *f2v_batch_last_error(const f2v_batch *b)
{
    static thread_local std::string msg;
    msg = b ? b->eng.err() : global_error();
    return msg.c_str();
}

}  // extern "C"
