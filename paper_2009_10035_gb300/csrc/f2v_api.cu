// f2v_api.cu -- host driver and C ABI of libf2v (declared in include/f2v.h).
//
// The context owns, on one device: the CSR graph, the pair prefix apair and
// the item table of every minibatch (built once here, since the graph and
// the minibatch partition are fixed), two embedding buffers that swap roles
// every epoch, the FP32 master in the BF16 form, and the scratch of split
// vertices.  An epoch is one launch of the fused force kernel per minibatch,
// in order, on the context's stream: the launch boundary is the barrier
// between minibatch k (whose rows it writes) and k+1 (which reads them).
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>
#include <thread>
#include <vector>

#include "f2v.h"
#include "f2v_device.cuh"
#include "f2v_internal.h"

namespace f2v {

Shape choose_shape(int d)
{
    switch (d) {
        case 2: return {1, 2, 1, true};
        case 4: return {1, 4, 1, true};
        case 8: return {2, 4, 1, true};
        case 16: return {4, 4, 1, true};
        case 32: return {8, 4, 1, true};
        case 64: return {16, 4, 1, true};
        case 128: return {32, 4, 1, true};
        case 256: return {32, 4, 2, true};
        case 512: return {32, 4, 4, true};
        case 1024: return {32, 4, 8, true};
        default: break;
    }
    int nv = 1;
    while (nv * 32 < d) nv *= 2;
    return {32, 1, nv, false};
}

int items_pairs(const Shape &sh)
{
    return sh.L >= 32 ? 32 : 32;
}

}  // namespace f2v

using namespace f2v;

// Kernels of the auxiliary entry points (initial embedding, sample dump).
namespace {

// Z0[i][j] = (Philox(ctr=(i, j, 0xFFFF, 0)).x0 >> 8) * 2^-24 - 0.5, written
// to both the storage rows and (BF16 form) the FP32 master.  The value is a
// multiple of 2^-24 in [-0.5, 0.5), so BF16 rounding of it is the only loss.
template <typename Ts>
__global__ void init_kernel(Ts *z, float *master, int64_t n, int d, uint32_t k0, uint32_t k1)
{
    const int64_t total = n * (int64_t)d;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(t / d), j = (uint32_t)(t % d);
        const float v = z0_value(i, j, k0, k1);
        if constexpr (sizeof(Ts) == 2) {
            z[t] = __float2bfloat16_rn(v);
            master[t] = v;
        } else {
            z[t] = v;
        }
    }
}

// rank (may be null): positions of the vertices in the epoch's random
// partition, which decide a vertex's minibatch for shared samples.
__global__ void samples_kernel(int32_t *out, int64_t n, int s, int32_t shared_b,
                               const int32_t *rank, uint32_t epoch, uint32_t k0, uint32_t k1)
{
    const int64_t total = n * (int64_t)s;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = t / s;
        const uint32_t k = (uint32_t)(t % s);
        const int64_t kb = shared_b > 0 ? (rank ? rank[u] : u) / shared_b : -1;
        out[t] = (int32_t)negative_sample(u, kb, epoch, k, (int32_t)n, k0, k1);
    }
}

template <typename Ts>
__global__ void round_rows_kernel(Ts *z, const float *master, int64_t total)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        z[t] = __float2bfloat16_rn(master[t]);
}

thread_local std::string g_last_error;

}  // namespace

// Evaluation entry points live in f2v_eval.cu.
namespace f2v {
cudaError_t eval_auc_device(const float *zf, const __nv_bfloat16 *zb, int d, int model,
                            const int32_t *pos, int64_t npos, const int32_t *neg, int64_t nneg,
                            cudaStream_t st, double *auc, std::string *err);
cudaError_t eval_loss_device(const float *z, int d, int model, const int32_t *row_ptr,
                             const int32_t *col_idx, int n, int64_t nnz, int s, uint32_t epoch,
                             uint32_t key0, uint32_t key1, cudaStream_t st, double *loss,
                             std::string *err);
}

// One epoch's random partition: its order, the graph relabelled into it and
// the chunk tables (two sets: the current epoch's, and the next one's, which
// the side stream builds while the current epoch runs).
struct PartSet {
    int32_t *perm = nullptr, *rank = nullptr, *row_ptr = nullptr, *col_idx = nullptr;
    int64_t *apair = nullptr;
    int32_t *mb_C = nullptr, *items = nullptr;
    int64_t *mb_base = nullptr, *mb_p0 = nullptr;
    int epoch = -1;                        // epoch whose order the set holds
};

struct f2v_ctx {
    int device = 0;
    int n = 0, d = 0, ld = 0, s = 0, b = 0;
    int walk = 0;                          // rForce2Vec walk length (0: neighbours, Alg. 2)
    bool shared = false;                   // one sample set S_b per minibatch (Alg. 1's sampling step)
    bool partition = false;                // a new random partition every epoch (Alg. 1's partition step)
    int64_t nnz = 0;
    int64_t pairs = 0;                     // force pairs per epoch
    int model = 0;
    f2v_precision precision = F2V_FP32;
    uint64_t seed = 0;
    float lr = 0.02f;
    f2v_schedule schedule = F2V_LR_CONSTANT;
    int total_epochs = 0;
    int epoch = 0;
    cudaStream_t stream = nullptr;
    Shape shape{};
    int C = 32;                            // pairs per item (register kernel)
    bool bulk = false;                     // shared-memory staged kernel in use
    int bulk_warps = 0, bulk_smem = 0, bulk_sms = 0;

    // host copies of the schedule of work
    std::vector<int64_t> h_apair;          // n + 1
    std::vector<int64_t> mb_item_base;     // M + 1
    std::vector<int32_t> mb_C;             // pairs per item (chunk) of each minibatch
    std::vector<int64_t> mb_p0;            // M + 1: first pair of each minibatch (and the end)
    int64_t max_items = 0;

    // device buffers
    int32_t *err_word = nullptr;           // set by a device wait that timed out
    // the graph the kernels walk (with a random partition, relabelled into
    // the epoch's order) and the graph as given (the same arrays otherwise)
    int32_t *row_ptr = nullptr, *col_idx = nullptr, *item_u0 = nullptr, *counter = nullptr;
    int64_t *apair = nullptr;
    int32_t *row_ptr0 = nullptr, *col_idx0 = nullptr;
    int64_t *apair0 = nullptr;
    // Z: z[cur] holds it as of the epoch's start (rows in id order), z[cur ^ 1]
    // receives the epoch's updates.  With a random partition, z[cur ^ 1] holds
    // Z gathered into the epoch's order and z[2] the updates in that order,
    // scattered back into z[cur] when the epoch ends.
    void *z[3] = {nullptr, nullptr, nullptr};   // float or bf16 rows
    int32_t *perm = nullptr, *rank = nullptr;  // the current epoch's order and its inverse
    PartSet part[2];                       // random partition: epoch e uses part[e & 1]
    PartitionScratch pw{};
    int64_t *d_mb_p0 = nullptr;            // M + 1 (random partition)
    float *master = nullptr;
    int levels = 0;                        // combine-tree levels in use
    float *slots = nullptr;                // all levels, in order
    int32_t *unit_cnt = nullptr;
    // staged (persistent) kernel only
    int ring = 1;                          // combine-tree scratch regions
    int64_t slot_stride = 0, cnt_stride = 0;   // elements between regions
    int64_t *d_mb_item_base = nullptr;     // M + 1
    int32_t *d_mb_C = nullptr;             // M
    int32_t *row_flag = nullptr;           // n: epoch + 1 once written this epoch
    int32_t *mb_done = nullptr;            // M: chunks finished in this launch
    CUtensorMap zmap{};                    // both Z buffers: 2n rows of the storage type
    CUtensorMap mmap{};                    // the FP32 master (BF16 form)
    // partner codes of every pair of an epoch: two buffers, epoch e in e & 1,
    // so the next epoch's list is written (on xstream) while this one runs
    int32_t *partner_buf[2] = {nullptr, nullptr};
    int partner_epoch[2] = {-1, -1};       // epoch whose partners each buffer holds
    cudaStream_t xstream = nullptr;        // the next epoch's partner list
    cudaEvent_t ev_xdone[2] = {nullptr, nullptr};   // buffer written
    cudaEvent_t ev_xfree[2] = {nullptr, nullptr};   // buffer's last reader done
    int cur = 0;                           // buffer holding Z as of the epoch's start
    int mb_pos = 0;                        // next minibatch of the current epoch
    size_t device_bytes = 0;

    int blocks_cap = 0;
    int64_t launches = 0;

    bool timing = false;
    std::vector<cudaEvent_t> ev_free, ev_pending;   // pairs (start, stop)
    int64_t timed_launches = 0;
    double timed_ms = 0.0;

    bool failed = false;
    std::string err;
    std::vector<void *> owned;             // every device allocation, freed once by release()
};

namespace {

f2v_status fail(f2v_ctx *c, f2v_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (st == F2V_ECUDA) c->failed = true;
    } else {
        g_last_error = buf;
    }
    return st;
}

#define F2V_CUDA(ctx, call)                                                             \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? F2V_ENOMEM : F2V_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define F2V_CHECK_CTX(ctx)                                                   \
    do {                                                                     \
        if (!(ctx)) return fail(nullptr, F2V_EINVAL, "null context");        \
        if ((ctx)->failed) return F2V_ESTATE;                                \
    } while (0)

size_t elem_size(const f2v_ctx *c) { return c->precision == F2V_BF16 ? 2 : 4; }

f2v_status alloc(f2v_ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, F2V_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->device_bytes += bytes;
    c->owned.push_back(*p);
    return F2V_OK;
}

void release(f2v_ctx *c)
{
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    if (c->xstream) cudaStreamSynchronize(c->xstream);
    // the pointer fields are views; the allocations are in `owned`
    for (auto it = c->owned.rbegin(); it != c->owned.rend(); ++it) cudaFree(*it);
    c->owned.clear();
    for (int i = 0; i < 2; ++i) {
        if (c->ev_xdone[i]) cudaEventDestroy(c->ev_xdone[i]);
        if (c->ev_xfree[i]) cudaEventDestroy(c->ev_xfree[i]);
    }
    if (c->xstream) cudaStreamDestroy(c->xstream);
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_pending) cudaEventDestroy(e);
    if (prev >= 0) cudaSetDevice(prev);
}

// Host-side validation of the CSR (Sec. II-A: 0/1 adjacency, no self-loops).
// The checks of f2v_create's CSR, with up to `max_threads` host threads;
// on failure *msg says why.  Touches no global state (several graphs may be
// checked at once).
f2v_status csr_check(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, uint32_t flags,
                     int max_threads, std::string *msg)
{
    auto bad = [&](const char *fmt, ...) {
        char buf[256];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        *msg = buf;
        return F2V_EINVAL;
    };
    if (!row_ptr) return bad("row_ptr is NULL");
    if (row_ptr[0] != 0) return bad("row_ptr[0] = %d, expected 0", row_ptr[0]);
    for (int32_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u])
            return bad("row_ptr not monotone at row %d", u);
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return bad("col_idx is NULL");
    // Rows are checked in parallel ranges of about equal entries.  A row whose
    // columns strictly increase has no duplicate (a sequential test); only
    // other rows need the per-thread stamp array.  The first bad row found in
    // row order is the one reported.
    const int nthreads = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)std::thread::hardware_concurrency(),
                              (int64_t)max_threads, (nnz + n) / 65536 + 1}));
    std::vector<int32_t> bad_row((size_t)nthreads, INT32_MAX), bad_kind((size_t)nthreads, 0);
    std::vector<int32_t> bounds((size_t)nthreads + 1, n);
    bounds[0] = 0;
    for (int t = 1; t < nthreads; ++t) {   // split by entries
        const int64_t target = nnz * t / nthreads;
        bounds[(size_t)t] = (int32_t)(std::upper_bound(row_ptr, row_ptr + n + 1, (int32_t)target) -
                                      row_ptr - 1);
        bounds[(size_t)t] = std::max(bounds[(size_t)t], bounds[(size_t)t - 1]);
    }
    auto check_range = [&](int t) {
        std::vector<int32_t> stamp;
        for (int32_t u = bounds[(size_t)t]; u < bounds[(size_t)t + 1]; ++u) {
            const int32_t lo = row_ptr[u], hi = row_ptr[u + 1];
            bool sorted = true;
            for (int32_t e = lo; e < hi; ++e) {
                const int32_t v = col_idx[e];
                if (v < 0 || v >= n || v == u) {
                    bad_row[(size_t)t] = u;
                    bad_kind[(size_t)t] = (v == u) ? 2 : 1;
                    return;
                }
                if (e > lo && v <= col_idx[e - 1]) sorted = false;
            }
            if (sorted) continue;
            if (stamp.empty()) stamp.assign((size_t)n, -1);
            for (int32_t e = lo; e < hi; ++e) {
                if (stamp[(size_t)col_idx[e]] == u) {
                    bad_row[(size_t)t] = u;
                    bad_kind[(size_t)t] = 3;
                    return;
                }
                stamp[(size_t)col_idx[e]] = u;
            }
        }
    };
    {
        std::vector<std::thread> pool;
        for (int t = 1; t < nthreads; ++t) pool.emplace_back(check_range, t);
        check_range(0);
        for (auto &th : pool) th.join();
    }
    for (int t = 0; t < nthreads; ++t) {
        if (bad_kind[(size_t)t] == 0) continue;
        const int32_t u = bad_row[(size_t)t];
        if (bad_kind[(size_t)t] == 2) return bad("self-loop at vertex %d", u);
        if (bad_kind[(size_t)t] == 3)
            return bad("duplicate entry in row %d", u);
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (col_idx[e] < 0 || col_idx[e] >= n)
                return bad("col_idx[%d] = %d out of range [0, %d)", e,
                            col_idx[e], n);
    }
    if (flags & F2V_FLAG_CHECK_SYMMETRY) {
        // count (u, v) against (v, u): transpose counts must match row by row
        std::vector<int64_t> tcount((size_t)n + 1, 0);
        for (int64_t e = 0; e < nnz; ++e) tcount[(size_t)col_idx[e] + 1]++;
        for (int32_t u = 0; u < n; ++u)
            if (tcount[(size_t)u + 1] != row_ptr[u + 1] - row_ptr[u])
                return bad("CSR not symmetric (row %d)", u);
        for (int32_t u = 0; u < n; ++u) tcount[(size_t)u + 1] += tcount[(size_t)u];
        std::vector<int32_t> tcol((size_t)nnz);
        std::vector<int64_t> fill(tcount.begin(), tcount.end() - 1);
        for (int32_t u = 0; u < n; ++u)
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
                tcol[(size_t)fill[(size_t)col_idx[e]]++] = u;
        for (int32_t u = 0; u < n; ++u) {
            std::vector<int32_t> a(col_idx + row_ptr[u], col_idx + row_ptr[u + 1]);
            std::vector<int32_t> b(tcol.begin() + tcount[(size_t)u],
                                   tcol.begin() + tcount[(size_t)u + 1]);
            std::sort(a.begin(), a.end());
            std::sort(b.begin(), b.end());
            if (a != b) return bad("CSR not symmetric (row %d)", u);
        }
    }
    return F2V_OK;
}

f2v_status validate_graph(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                          uint32_t flags)
{
    std::string msg;
    const f2v_status st = csr_check(row_ptr, col_idx, n, flags, 16, &msg);
    if (st != F2V_OK) return fail(nullptr, st, "%s", msg.c_str());
    return F2V_OK;
}

// Builds the pair prefix and the per-minibatch item table on the host.
// Returns false if a minibatch holds 2^31 pairs or more.
bool build_schedule(f2v_ctx *c, const int32_t *row_ptr, std::vector<int32_t> &items)
{
    const int n = c->n;
    c->h_apair.assign((size_t)n + 1, 0);
    c->pairs = 0;
    for (int u = 0; u < n; ++u) {
        // N(u): the neighbours, or a walk of c->walk steps if u has any (Alg. 3)
        const int64_t deg = row_ptr[u + 1] - row_ptr[u];
        int64_t cu = (c->walk > 0 ? (deg > 0 ? c->walk : 0) : deg) + c->s;
        c->pairs += cu;
        if (cu == 0) cu = 1;     // the empty pair: the row is still carried over
        c->h_apair[(size_t)u + 1] = c->h_apair[(size_t)u] + cu;
    }
    const int M = (n + c->b - 1) / c->b;
    c->mb_item_base.assign((size_t)M + 1, 0);
    c->mb_C.assign((size_t)M, c->C);
    items.clear();
    c->max_items = 0;
    const int64_t W = (int64_t)c->bulk_sms * c->bulk_warps;   // warps of a staged launch
    for (int k = 0; k < M; ++k) {
        const int u0 = k * c->b, u1 = std::min(n, u0 + c->b);
        const int64_t P0 = c->h_apair[(size_t)u0], P1 = c->h_apair[(size_t)u1];
        int64_t C = c->C;
        if (c->bulk) {   // two chunks per warp, a multiple of 32 pairs
            C = (P1 - P0 + W - 1) / W;
            C = std::max<int64_t>(32, ((C + 1) / 2 + 31) / 32 * 32);
        }
        if (P1 - P0 >= (int64_t)INT32_MAX - C) return false;
        c->mb_C[(size_t)k] = (int32_t)C;
        const int64_t nit = (P1 - P0 + C - 1) / C;
        int u = u0;
        for (int64_t i = 0; i < nit; ++i) {
            const int64_t q = P0 + i * C;
            while (c->h_apair[(size_t)u + 1] <= q) ++u;
            items.push_back(u);
        }
        c->mb_item_base[(size_t)k + 1] = c->mb_item_base[(size_t)k] + nit;
        c->max_items = std::max(c->max_items, nit);
    }
    c->mb_p0.assign((size_t)M + 1, 0);
    for (int k = 0; k <= M; ++k)
        c->mb_p0[(size_t)k] = c->h_apair[(size_t)std::min<int64_t>(n, (int64_t)k * c->b)];
    if (c->partition) {
        // any b vertices may share a minibatch: size for the b largest
        std::vector<int64_t> cnt((size_t)n);
        for (int u = 0; u < n; ++u) cnt[(size_t)u] = c->h_apair[(size_t)u + 1] - c->h_apair[(size_t)u];
        const size_t top = std::min<size_t>((size_t)c->b, cnt.size());
        std::partial_sort(cnt.begin(), cnt.begin() + top, cnt.end(), std::greater<int64_t>());
        int64_t maxPk = 0;
        for (size_t i = 0; i < top; ++i) maxPk += cnt[i];
        if (maxPk >= (int64_t)INT32_MAX - 32) return false;
        // (the staged kernel cuts a minibatch into at most two chunks per warp)
        const int64_t worst = c->bulk ? std::max<int64_t>(2 * W, 1) : (maxPk + c->C - 1) / c->C;
        c->max_items = std::max(c->max_items, worst);
    }
    return true;
}

}  // namespace

namespace f2v {
f2v_status check_csr(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, uint32_t flags)
{
    return validate_graph(row_ptr, col_idx, n, flags);
}
f2v_status check_csr_quiet(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                           uint32_t flags, int max_threads, std::string *msg)
{
    return csr_check(row_ptr, col_idx, n, flags, max_threads, msg);
}
void set_global_error(const std::string &msg) { g_last_error = msg; }
std::string global_error() { return g_last_error; }
}  // namespace f2v

namespace {

// Device scratch of one synchronous call, freed on every return path.
struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t get(T **p, size_t count)
    {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count * sizeof(T), 16), st);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
    ~Scratch()
    {
        for (void *q : ptrs) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
    }
};

bool pairs_in_range(const int32_t *pairs, int64_t np, int32_t n)
{
    for (int64_t i = 0; i < 2 * np; ++i)
        if (pairs[i] < 0 || pairs[i] >= n) return false;
    return true;
}

}  // namespace

namespace {

double lr_for_epoch(const f2v_ctx *c, int e)
{
    if (c->schedule == F2V_LR_LINEAR && c->total_epochs > 0)
        return (double)c->lr * (1.0 - (double)e / (double)c->total_epochs);
    return (double)c->lr;
}

cudaError_t launch_init(f2v_ctx *c)
{
    const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
    const int64_t total = (int64_t)c->n * c->d;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (c->precision == F2V_BF16)
        init_kernel<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>(
            (__nv_bfloat16 *)c->z[c->cur], c->master, c->n, c->d, k0, k1);
    else
        init_kernel<float><<<blocks, 256, 0, c->stream>>>((float *)c->z[c->cur], nullptr, c->n,
                                                          c->d, k0, k1);
    c->launches++;
    return cudaGetLastError();
}

f2v_status collect_timing(f2v_ctx *c)
{
    for (size_t i = 0; i + 1 < c->ev_pending.size(); i += 2) {
        F2V_CUDA(c, cudaEventSynchronize(c->ev_pending[i + 1]));
        float ms = 0.f;
        F2V_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pending[i], c->ev_pending[i + 1]));
        c->timed_ms += ms;
        c->timed_launches++;
        c->ev_free.push_back(c->ev_pending[i]);
        c->ev_free.push_back(c->ev_pending[i + 1]);
    }
    c->ev_pending.clear();
    return F2V_OK;
}

f2v_status get_event(f2v_ctx *c, cudaEvent_t *e)
{
    if (!c->ev_free.empty()) {
        *e = c->ev_free.back();
        c->ev_free.pop_back();
        return F2V_OK;
    }
    F2V_CUDA(c, cudaEventCreate(e));
    return F2V_OK;
}

int num_minibatches(const f2v_ctx *c) { return (c->n + c->b - 1) / c->b; }

// The staged kernel reads every pair's partner from an expanded list, and
// so does the register kernel in the rForce2Vec form (walks are drawn once
// per epoch into the list).
bool uses_partner_list(const f2v_ctx *c)
{
    return c->bulk || c->walk > 0 || c->shared || c->partition;
}

// The partner list of `epoch` for the graph the kernels walk (given = true:
// for the graph as given, in id order).
cudaError_t launch_partner_list(f2v_ctx *c, int epoch, int32_t *buf, cudaStream_t st,
                                bool given = false, const PartSet *ps = nullptr,
                                bool refresh = false)
{
    c->launches++;
    const int32_t shared_b = c->shared ? c->b : 0;
    // a list of another epoch of the same graph in this buffer: only the
    // samples change (neighbourhoods without walks, no relabelling)
    if (refresh && c->walk == 0 && !c->partition && !given)
        return launch_refresh_samples(c->row_ptr, c->apair, c->n, c->s, shared_b,
                                      (uint32_t)epoch, (uint32_t)c->seed,
                                      (uint32_t)(c->seed >> 32), buf, st);
    const bool relabelled = c->partition && !given;
    // a random partition's set: ps if given, else the current epoch's
    const int32_t *rp = given ? c->row_ptr0 : (ps ? ps->row_ptr : c->row_ptr);
    const int32_t *ci = given ? c->col_idx0 : (ps ? ps->col_idx : c->col_idx);
    const int64_t *ap = given ? c->apair0 : (ps ? ps->apair : c->apair);
    const int32_t *perm = relabelled ? (ps ? ps->perm : c->perm) : nullptr;
    const int32_t *rank = relabelled ? (ps ? ps->rank : c->rank) : nullptr;
    if (c->walk > 0)
        return launch_expand_walks(rp, ci, ap, c->n, c->s, c->walk, shared_b, perm, rank,
                                   (uint32_t)epoch, (uint32_t)c->seed, (uint32_t)(c->seed >> 32),
                                   buf, st);
    return launch_expand_partners(rp, ci, ap, c->n, c->s, shared_b, perm, rank, (uint32_t)epoch,
                                  (uint32_t)c->seed, (uint32_t)(c->seed >> 32), buf, st);
}

// Buffers (and their row offsets in the TMA map) the epoch reads from and
// writes to.
int zcur_index(const f2v_ctx *c) { return c->partition ? (c->cur ^ 1) : c->cur; }
int znext_index(const f2v_ctx *c) { return c->partition ? 2 : (c->cur ^ 1); }

// Reads (and clears) the device error word after the stream has drained.
// A set word means a bounded device wait ran out: the epoch's result is not
// valid, and the context is marked failed.
f2v_status check_device_error(f2v_ctx *c)
{
    int32_t word = 0;
    F2V_CUDA(c, cudaMemcpyAsync(&word, c->err_word, sizeof word, cudaMemcpyDeviceToHost,
                                c->stream));
    F2V_CUDA(c, cudaStreamSynchronize(c->stream));
    if (word != 0) {
        c->failed = true;
        c->err = "a device-side wait timed out; results of the last epochs are not valid";
        return F2V_ETIMEOUT;
    }
    return F2V_OK;
}

// Arguments of the force kernel for minibatch k of the current epoch.
template <typename Ts>
void fill_args(const f2v_ctx *c, int k, float eta, ForceArgs<Ts> &a)
{
    const int u0 = k * c->b, u1 = std::min(c->n, u0 + c->b);
    a.row_ptr = c->row_ptr;
    a.col_idx = c->col_idx;
    a.apair = c->apair;
    a.item_u0 = c->item_u0 + c->mb_item_base[(size_t)k];
    a.zcur = (const Ts *)c->z[zcur_index(c)];
    a.znext = (Ts *)c->z[znext_index(c)];
    a.counter = c->counter;
    a.slots = c->slots;
    a.unit_cnt = c->unit_cnt;
    a.units0 = std::max<int64_t>(c->max_items, 1);
    (void)u1;
    a.P0 = c->mb_p0[(size_t)k];
    a.Pk = (int32_t)(c->mb_p0[(size_t)k + 1] - a.P0);
    a.n_items = (int32_t)(c->mb_item_base[(size_t)k + 1] - c->mb_item_base[(size_t)k]);
    a.mb_begin = u0;
    a.mb_end = u1;
    a.n = c->n; a.d = c->d; a.ld = c->ld; a.s = c->s;
    a.C = c->mb_C[(size_t)k];
    a.epoch = (uint32_t)c->epoch;
    a.key0 = (uint32_t)c->seed;
    a.key1 = (uint32_t)(c->seed >> 32);
    a.eta = eta;
    a.model = c->model;
    a.err = c->err_word;
    a.partner = (c->walk > 0 || c->shared || c->partition) ? c->partner_buf[c->epoch & 1]
                                                            : nullptr;
}

template <typename Ts>
void fill_epoch_args(const f2v_ctx *c, int k_begin, int k_end, float eta, EpochArgs<Ts> &ea)
{
    fill_args(c, k_begin, eta, ea.f);
    ea.partner = c->partner_buf[c->epoch & 1];
    ea.items = c->item_u0;
    ea.mb_item_base = c->d_mb_item_base;
    ea.mb_C = c->d_mb_C;
    ea.row_flag = c->row_flag;
    ea.mb_done = c->mb_done;
    ea.mb_next = c->mb_done + c->mb_C.size();
    ea.slots = c->slots;
    ea.unit_cnt = c->unit_cnt;
    ea.slot_stride = c->slot_stride;
    ea.cnt_stride = c->cnt_stride;
    ea.k_begin = k_begin;
    ea.k_end = k_end;
    ea.b = c->b;
    ea.ring = c->ring;
    // group claims (FP32 rows): for chunks of up to 512 pairs (16 tiles); a
    // block's group of larger chunks ends with most of its warps idle
    int32_t cmax = 0;
    for (int k = k_begin; k < k_end; ++k) cmax = std::max(cmax, c->mb_C[(size_t)k]);
    ea.groups = (c->precision == F2V_FP32 && cmax <= 512) ? 1 : 0;
    ea.zcur_row0 = zcur_index(c) * c->n;
    ea.znext_row0 = znext_index(c) * c->n;
    ea.own_row0 = (c->precision == F2V_BF16) ? 0 : zcur_index(c) * c->n;
}

// Launches the force kernel(s) for minibatches [k_begin, k_end) of the
// current epoch: one persistent launch for the staged kernel, one launch
// per minibatch for the register kernel.  Each launch is bracketed by timing
// events when timing is on.
// Random partition.  build_partition writes epoch e's order, the graph
// relabelled into it and its chunk tables into set ps, on stream st (the
// main stream, or the side stream one epoch ahead); it uses the scratch c->pw,
// so two builds never overlap.
cudaError_t build_partition(f2v_ctx *c, int e, PartSet &ps, cudaStream_t st)
{
    const int M = num_minibatches(c);
    cudaError_t err = launch_partition(c->n, (uint32_t)e, (uint32_t)c->seed,
                                       (uint32_t)(c->seed >> 32), c->pw, ps.perm, ps.rank, st);
    if (err == cudaSuccess)
        err = launch_relabel(c->row_ptr0, c->col_idx0, ps.perm, ps.rank, c->n, c->s, c->walk,
                             c->pw, ps.row_ptr, ps.col_idx, ps.apair, st);
    const int64_t W = c->bulk ? (int64_t)c->bulk_sms * c->bulk_warps : 0;
    if (err == cudaSuccess)
        err = launch_mb_tables(ps.apair, c->n, c->b, M, W, c->C, c->pw, ps.mb_C, ps.mb_base,
                               ps.items, ps.mb_p0, st);
    c->launches += 9;
    ps.epoch = e;
    return err;
}

// The kernels of the current epoch read set ps.
void use_partition(f2v_ctx *c, const PartSet &ps)
{
    c->perm = ps.perm;
    c->rank = ps.rank;
    c->row_ptr = ps.row_ptr;
    c->col_idx = ps.col_idx;
    c->apair = ps.apair;
    c->item_u0 = ps.items;
    c->d_mb_C = ps.mb_C;
    c->d_mb_item_base = ps.mb_base;
    c->d_mb_p0 = ps.mb_p0;
}

// At the start of epoch e: its set (built ahead on the side stream, else
// now), the register kernel's host copy of the tables, and Z gathered into
// the order (every time the epoch starts, since Z may have been set or
// synchronised since).
f2v_status prepare_partition(f2v_ctx *c, int e)
{
    const int M = num_minibatches(c);
    const int slot = e & 1;
    PartSet &ps = c->part[slot];
    if (ps.epoch != e) {
        // the side stream may still be building the other set with the scratch
        if (c->xstream) F2V_CUDA(c, cudaStreamSynchronize(c->xstream));
        F2V_CUDA(c, build_partition(c, e, ps, c->stream));
        c->partner_epoch[slot] = -1;      // its partner list belongs to another order
    } else {
        F2V_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_xdone[slot], 0));
    }
    use_partition(c, ps);
    if (!c->bulk) {
        // the register kernel takes each minibatch's tables from the host
        F2V_CUDA(c, cudaMemcpyAsync(c->mb_C.data(), c->d_mb_C, sizeof(int32_t) * M,
                                    cudaMemcpyDeviceToHost, c->stream));
        F2V_CUDA(c, cudaMemcpyAsync(c->mb_item_base.data(), c->d_mb_item_base,
                                    sizeof(int64_t) * (M + 1), cudaMemcpyDeviceToHost,
                                    c->stream));
        F2V_CUDA(c, cudaMemcpyAsync(c->mb_p0.data(), c->d_mb_p0, sizeof(int64_t) * (M + 1),
                                    cudaMemcpyDeviceToHost, c->stream));
        F2V_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    F2V_CUDA(c, launch_permute_rows((const float *)c->z[c->cur], (float *)c->z[c->cur ^ 1],
                                    c->perm, c->n, c->ld, false, c->stream));
    c->launches++;
    return F2V_OK;
}

f2v_status run_range(f2v_ctx *c, int k_begin, int k_end)
{
    const int e = c->epoch;
    const float eta = (float)lr_for_epoch(c, e);
    const int step = c->bulk ? (k_end - k_begin) : 1;
    const int slot = e & 1;
    if (c->partition && k_begin == 0) {
        f2v_status pst = prepare_partition(c, e);
        if (pst != F2V_OK) return pst;
    }
    const bool listed = uses_partner_list(c);
    if (listed && c->partner_epoch[slot] != e) {   // this epoch's partner list, now
        // (after any list still being written ahead into this buffer)
        F2V_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_xdone[slot], 0));
        cudaError_t ee = launch_partner_list(c, e, c->partner_buf[slot], c->stream, false,
                                             nullptr, c->partner_epoch[slot] >= 0);
        if (ee != cudaSuccess)
            return fail(c, F2V_ECUDA, "partner expansion launch: %s", cudaGetErrorString(ee));
        c->partner_epoch[slot] = e;
    } else if (listed) {
        // written ahead on the side stream
        F2V_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_xdone[slot], 0));
    }
    // the other buffer's last reader (epoch e - 1) is done once the work
    // enqueued so far is: the next epoch's list (with a random partition, the
    // next epoch's order, relabelled graph and tables too) may overwrite it
    const bool prefetch =
        listed && k_end == num_minibatches(c) &&
        (c->partition ? c->part[slot ^ 1].epoch != e + 1 : c->partner_epoch[slot ^ 1] != e + 1);
    if (prefetch) F2V_CUDA(c, cudaEventRecord(c->ev_xfree[slot ^ 1], c->stream));
    if (c->bulk)
        F2V_CUDA(c, cudaMemsetAsync(c->mb_done + k_begin, 0,
                                    sizeof(int32_t) * (size_t)(k_end - k_begin), c->stream));
    if (c->bulk)
        F2V_CUDA(c, cudaMemsetAsync(c->mb_done + c->mb_C.size() + k_begin, 0,
                                    sizeof(int32_t) * (size_t)(k_end - k_begin), c->stream));
    for (int k = k_begin; k < k_end; k += step) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->timing) {
            f2v_status st = get_event(c, &e0);
            if (st == F2V_OK) st = get_event(c, &e1);
            if (st != F2V_OK) return st;
            F2V_CUDA(c, cudaEventRecord(e0, c->stream));
        }
        cudaError_t err;
        if (c->precision == F2V_BF16) {
            if (c->bulk) {
                EpochArgs<__nv_bfloat16> ea{};
                fill_epoch_args(c, k, k + step, eta, ea);
                ea.f.master = c->master;
                err = launch_bulk_bf16(c->d, c->model, ea, c->zmap, c->mmap, c->bulk_sms, c->bulk_warps,
                                       c->bulk_smem, c->stream);
            } else {
                ForceArgs<__nv_bfloat16> a{};
                fill_args(c, k, eta, a);
                a.master = c->master;
                err = launch_force_bf16(c->shape, a, c->blocks_cap, c->stream);
            }
        } else {
            if (c->bulk) {
                EpochArgs<float> ea{};
                fill_epoch_args(c, k, k + step, eta, ea);
                ea.f.master = nullptr;
                err = launch_bulk_fp32(c->d, c->model, ea, c->zmap, c->zmap, c->bulk_sms, c->bulk_warps,
                                       c->bulk_smem, c->stream);
            } else {
                ForceArgs<float> a{};
                fill_args(c, k, eta, a);
                a.master = nullptr;
                err = launch_force_fp32(c->shape, a, c->blocks_cap, c->stream);
            }
        }
        c->launches++;
        if (err != cudaSuccess)
            return fail(c, F2V_ECUDA, "force kernel launch (epoch %d, minibatch %d): %s", e, k,
                        cudaGetErrorString(err));
        if (c->timing) {
            F2V_CUDA(c, cudaEventRecord(e1, c->stream));
            c->ev_pending.push_back(e0);
            c->ev_pending.push_back(e1);
        }
    }
    if (prefetch) {
        // the next epoch's partner list, on the side stream, overlapping this
        // epoch's force launch (it only reads the graph and the epoch number;
        // with a random partition, the order it builds first)
        const int ns = slot ^ 1;
        F2V_CUDA(c, cudaStreamWaitEvent(c->xstream, c->ev_xfree[ns], 0));
        const PartSet *nps = nullptr;
        if (c->partition) {
            F2V_CUDA(c, build_partition(c, e + 1, c->part[ns], c->xstream));
            nps = &c->part[ns];
        }
        cudaError_t ee = launch_partner_list(c, e + 1, c->partner_buf[ns], c->xstream, false, nps,
                                             c->partner_epoch[ns] >= 0);
        if (ee != cudaSuccess)
            return fail(c, F2V_ECUDA, "partner expansion launch: %s", cudaGetErrorString(ee));
        F2V_CUDA(c, cudaEventRecord(c->ev_xdone[ns], c->xstream));
        c->partner_epoch[ns] = e + 1;
    }
    if (c->partition && k_end == num_minibatches(c)) {
        // the epoch's rows back into id order
        F2V_CUDA(c, launch_permute_rows((const float *)c->z[2], (float *)c->z[c->cur], c->perm,
                                        c->n, c->ld, true, c->stream));
        c->launches++;
    }
    return F2V_OK;
}

// Advances the minibatch position by `count` within the epoch; at the end
// of an epoch the buffers swap.
void advance(f2v_ctx *c, int count)
{
    c->mb_pos += count;
    if (c->mb_pos == num_minibatches(c)) {
        c->mb_pos = 0;
        if (!c->partition) c->cur ^= 1;   // (a partition scatters into z[cur])
        c->epoch++;
    }
}

// Runs the remaining minibatches of the current epoch.
f2v_status run_epoch(f2v_ctx *c)
{
    const int M = num_minibatches(c);
    const int k0 = c->mb_pos;
    f2v_status st = run_range(c, k0, M);
    if (st != F2V_OK) return st;
    advance(c, M - k0);
    return F2V_OK;
}

// Mid-epoch, rows [0, mb_pos*b) are current in the next buffer only; copy
// them into the current buffer so that it holds all of Z.  The remaining
// minibatches read those rows from the next buffer, so progress is kept.
f2v_status sync_current(f2v_ctx *c)
{
    if (c->mb_pos == 0) return F2V_OK;
    const size_t rows = std::min<size_t>((size_t)c->mb_pos * c->b, (size_t)c->n);
    if (c->partition) {   // the updated positions, back to their ids
        F2V_CUDA(c, launch_permute_rows((const float *)c->z[2], (float *)c->z[c->cur], c->perm,
                                        (int64_t)rows, c->ld, true, c->stream));
        c->launches++;
        return F2V_OK;
    }
    const size_t bytes = rows * (size_t)c->ld * elem_size(c);
    F2V_CUDA(c, cudaMemcpyAsync(c->z[c->cur], c->z[c->cur ^ 1], bytes, cudaMemcpyDeviceToDevice,
                                c->stream));
    return F2V_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

f2v_status f2v_create(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                      f2v_model model, int32_t s, float lr, int32_t minibatch, uint64_t seed,
                      f2v_ctx **out)
{
    return f2v_create_ex(row_ptr, col_idx, n, d, model, s, lr, minibatch, seed, F2V_FP32, 0u,
                         nullptr, out);
}

namespace {

constexpr int kMaxWalk = 1024;     // longest rForce2Vec walk accepted

f2v_status create_impl(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                       f2v_model model, int32_t s, int32_t walk, float lr, int32_t minibatch,
                       uint64_t seed, f2v_precision precision, uint32_t flags, void *stream,
                       f2v_ctx **out)
{
    if (!out) return fail(nullptr, F2V_EINVAL, "out is NULL");
    *out = nullptr;
    g_last_error.clear();
    if (n < 1) return fail(nullptr, F2V_EINVAL, "n = %d, must be >= 1", n);
    if (d < 1 || d > 1024) return fail(nullptr, F2V_EINVAL, "d = %d, must be in [1, 1024]", d);
    if (s < 0 || s > 65534) return fail(nullptr, F2V_EINVAL, "s = %d, must be in [0, 65534]", s);
    if (minibatch < 1) return fail(nullptr, F2V_EINVAL, "minibatch = %d, must be >= 1", minibatch);
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(nullptr, F2V_EINVAL, "lr must be finite and > 0");
    if (model < F2V_TDIST || model > F2V_FORCEATLAS) return fail(nullptr, F2V_EINVAL, "unknown model %d", (int)model);
    if (precision != F2V_FP32 && precision != F2V_BF16) return fail(nullptr, F2V_EINVAL, "unknown precision %d", (int)precision);
    f2v_status st = validate_graph(row_ptr, col_idx, n, flags);
    if (st != F2V_OK) return st;

    f2v_ctx *c = new (std::nothrow) f2v_ctx();
    if (!c) return fail(nullptr, F2V_ENOMEM, "host allocation failed");
    cudaError_t ce = cudaGetDevice(&c->device);
    if (ce != cudaSuccess) {
        delete c;
        return fail(nullptr, F2V_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    }
    c->n = n; c->d = d; c->ld = d; c->s = s; c->b = minibatch; c->model = (int)model;
    c->walk = walk;
    c->shared = (flags & F2V_FLAG_SHARED_SAMPLES) != 0;
    c->partition = (flags & F2V_FLAG_RANDOM_PARTITION) != 0;
    if (c->partition && precision != F2V_FP32) {
        delete c;
        return fail(nullptr, F2V_EINVAL, "F2V_FLAG_RANDOM_PARTITION needs F2V_FP32 storage");
    }
    c->precision = precision; c->seed = seed; c->lr = lr;
    c->stream = (cudaStream_t)stream;
    c->nnz = row_ptr[n];
    c->shape = choose_shape(d);
    c->C = items_pairs(c->shape);

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    sms = std::max(sms, 1);
    c->blocks_cap = sms * 8;
    // the staged kernel is persistent: its grid (one block per SM) must fit
    // (its tensor map spans the Z buffers, 2n rows or 3n with a random
    // partition, addressed by int32 row coordinates)
    if (!(flags & F2V_FLAG_NO_STAGING) && (int64_t)n * (c->partition ? 3 : 2) <= INT32_MAX &&
        bulk_config(d, precision == F2V_BF16, &c->bulk_warps, &c->bulk_smem) &&
        bulk_resident(d, precision == F2V_BF16, c->bulk_warps, c->bulk_smem) >= 1) {
        c->bulk = true;
        c->bulk_sms = sms;
        // minibatches in flight: 8 lets warps run further ahead of a minibatch
        // whose rows are still being written (rForce2Vec at d = 128, b = 4096:
        // 2.61 -> 2.51 ms per epoch; 1-hop unchanged; 16 gains nothing more)
        c->ring = 8;
    }

    std::vector<int32_t> items;
    try {
        if (!build_schedule(c, row_ptr, items)) {
            delete c;
            return fail(nullptr, F2V_EINVAL,
                        "a minibatch holds 2^31 or more force pairs; use a smaller minibatch");
        }
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(nullptr, F2V_ENOMEM, "host allocation failed (schedule)");
    }


    const size_t es = elem_size(c);
    const size_t zbytes = (size_t)n * (size_t)c->ld * es;
    st = F2V_OK;
    if (st == F2V_OK) st = alloc(c, (void **)&c->err_word, sizeof(int32_t));
    if (st == F2V_OK) st = alloc(c, (void **)&c->row_ptr0, sizeof(int32_t) * ((size_t)n + 1));
    if (st == F2V_OK) st = alloc(c, (void **)&c->col_idx0, sizeof(int32_t) * (size_t)c->nnz);
    if (st == F2V_OK) st = alloc(c, (void **)&c->apair0, sizeof(int64_t) * ((size_t)n + 1));
    if (st == F2V_OK) {
        c->row_ptr = c->row_ptr0;
        c->col_idx = c->col_idx0;
        c->apair = c->apair0;
    }
    if (st == F2V_OK && c->partition) {
        // two sets of the epoch's order, relabelled graph and tables (the
        // current epoch's and the next one's), and the scratch that builds them
        const size_t M = c->mb_C.size();
        // chunk tables of any order: at most one chunk per 32 pairs plus one per minibatch
        const size_t worst = (size_t)(c->h_apair[(size_t)n] / 32) + M + 1;
        if (items.size() < worst) items.resize(worst, 0);
        for (int i = 0; i < 2 && st == F2V_OK; ++i) {
            PartSet &ps = c->part[i];
            st = alloc(c, (void **)&ps.perm, sizeof(int32_t) * (size_t)n);
            if (st == F2V_OK) st = alloc(c, (void **)&ps.rank, sizeof(int32_t) * (size_t)n);
            if (st == F2V_OK) st = alloc(c, (void **)&ps.row_ptr, sizeof(int32_t) * ((size_t)n + 1));
            if (st == F2V_OK) st = alloc(c, (void **)&ps.col_idx, sizeof(int32_t) * (size_t)c->nnz);
            if (st == F2V_OK) st = alloc(c, (void **)&ps.apair, sizeof(int64_t) * ((size_t)n + 1));
            if (st == F2V_OK) st = alloc(c, (void **)&ps.mb_C, sizeof(int32_t) * M);
            if (st == F2V_OK) st = alloc(c, (void **)&ps.mb_base, sizeof(int64_t) * (M + 1));
            if (st == F2V_OK) st = alloc(c, (void **)&ps.items, sizeof(int32_t) * items.size());
            if (st == F2V_OK) st = alloc(c, (void **)&ps.mb_p0, sizeof(int64_t) * (M + 1));
        }
        if (st == F2V_OK) {   // views of the set of epoch 0
            c->row_ptr = c->part[0].row_ptr;
            c->col_idx = c->part[0].col_idx;
            c->apair = c->part[0].apair;
            c->perm = c->part[0].perm;
            c->rank = c->part[0].rank;
            c->item_u0 = c->part[0].items;
            c->d_mb_C = c->part[0].mb_C;
            c->d_mb_item_base = c->part[0].mb_base;
            c->d_mb_p0 = c->part[0].mb_p0;
        }
        if (st == F2V_OK) st = alloc(c, (void **)&c->pw.keys, sizeof(uint32_t) * (size_t)n);
        if (st == F2V_OK) st = alloc(c, (void **)&c->pw.keys2, sizeof(uint32_t) * (size_t)n);
        if (st == F2V_OK) st = alloc(c, (void **)&c->pw.vals, sizeof(int32_t) * (size_t)n);
        if (st == F2V_OK) st = alloc(c, (void **)&c->pw.deg, sizeof(int32_t) * ((size_t)n + 1));
        if (st == F2V_OK) st = alloc(c, (void **)&c->pw.cnt, sizeof(int64_t) * ((size_t)n + 1));
        if (st == F2V_OK) st = alloc(c, (void **)&c->pw.nch, sizeof(int64_t) * (M + 1));
        c->pw.temp_bytes = std::max<size_t>(partition_temp_bytes(n, (int32_t)M), 16);
        if (st == F2V_OK) st = alloc(c, &c->pw.temp, c->pw.temp_bytes);
    }
    if (st == F2V_OK && !c->partition)
        st = alloc(c, (void **)&c->item_u0, sizeof(int32_t) * items.size());
    if (st == F2V_OK) st = alloc(c, (void **)&c->counter, sizeof(int32_t) * (size_t)n);
    // Z buffers in one allocation: one TMA map then covers all of them
    const int nz = c->partition ? 3 : 2;
    if (st == F2V_OK) st = alloc(c, &c->z[0], nz * zbytes);
    for (int i = 1; i < nz && st == F2V_OK; ++i) c->z[i] = static_cast<char *>(c->z[0]) + i * zbytes;
    if (st == F2V_OK && precision == F2V_BF16)
        st = alloc(c, (void **)&c->master, (size_t)n * c->ld * sizeof(float));
    // combine tree: level l has ceil(max_items / 16^l) units, two slots each
    // (and, from level 1 on, two arrival counters each)
    if (st == F2V_OK) {
        int64_t units = std::max<int64_t>(c->max_items, 1);
        size_t slot_rows = 0, counters = 0;
        c->levels = 0;
        while (true) {
            slot_rows += 2 * (size_t)units;
            if (c->levels > 0) counters += 2 * (size_t)units;
            c->levels++;
            if (units <= 1 || c->levels == kMaxLevels) break;
            units = (units + kFan - 1) / kFan;
        }
        // the persistent kernel keeps `ring` regions, one per minibatch in flight
        c->slot_stride = (int64_t)c->ld * (int64_t)slot_rows;
        c->cnt_stride = (int64_t)counters + 1;
        const size_t ring = (size_t)c->ring;
        st = alloc(c, (void **)&c->slots, sizeof(float) * (size_t)c->slot_stride * ring);
        if (st == F2V_OK)
            st = alloc(c, (void **)&c->unit_cnt, sizeof(int32_t) * (size_t)c->cnt_stride * ring);
        if (st == F2V_OK &&
            cudaMemsetAsync(c->unit_cnt, 0, sizeof(int32_t) * (size_t)c->cnt_stride * ring,
                            c->stream) != cudaSuccess)
            st = fail(c, F2V_ECUDA, "memset of combine counters failed");
    }
    if (st == F2V_OK && c->bulk && !c->partition) {
        const size_t M = c->mb_C.size();
        st = alloc(c, (void **)&c->d_mb_item_base, sizeof(int64_t) * (M + 1));
        if (st == F2V_OK) st = alloc(c, (void **)&c->d_mb_C, sizeof(int32_t) * M);
    }
    if (st == F2V_OK && c->bulk) {
        const size_t M = c->mb_C.size();
        if (st == F2V_OK) st = alloc(c, (void **)&c->row_flag, sizeof(int32_t) * (size_t)n);
        if (st == F2V_OK) st = alloc(c, (void **)&c->mb_done, sizeof(int32_t) * 2 * M);
        std::string merr;
        if (st == F2V_OK &&
            (!make_row_map(&c->zmap, c->z[0], nz * (int64_t)n, d, precision == F2V_BF16, &merr) ||
             (precision == F2V_BF16 &&
              !make_row_map(&c->mmap, c->master, (int64_t)n, d, false, &merr))))
            st = fail(c, F2V_ECUDA, "tensor map: %s", merr.c_str());
    }
    if (st == F2V_OK && uses_partner_list(c)) {
        for (int i = 0; i < 2 && st == F2V_OK; ++i)
            st = alloc(c, (void **)&c->partner_buf[i],
                       sizeof(int32_t) * (size_t)c->h_apair[(size_t)n]);
        for (int i = 0; i < 2 && st == F2V_OK; ++i)
            if (cudaEventCreateWithFlags(&c->ev_xdone[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&c->ev_xfree[i], cudaEventDisableTiming) != cudaSuccess)
                st = fail(c, F2V_ECUDA, "event creation failed");
        if (st == F2V_OK &&
            cudaStreamCreateWithFlags(&c->xstream, cudaStreamNonBlocking) != cudaSuccess)
            st = fail(c, F2V_ECUDA, "stream creation failed");
    }
    if (st != F2V_OK) {
        g_last_error = c->err;
        release(c);
        delete c;
        return st;
    }
#define CREATE_CUDA(call)                                                            \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            fail(nullptr, F2V_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
            release(c);                                                              \
            delete c;                                                                \
            return F2V_ECUDA;                                                        \
        }                                                                            \
    } while (0)
    CREATE_CUDA(cudaMemcpyAsync(c->row_ptr0, row_ptr, sizeof(int32_t) * ((size_t)n + 1),
                                cudaMemcpyHostToDevice, c->stream));
    if (c->nnz)
        CREATE_CUDA(cudaMemcpyAsync(c->col_idx0, col_idx, sizeof(int32_t) * (size_t)c->nnz,
                                    cudaMemcpyHostToDevice, c->stream));
    CREATE_CUDA(cudaMemcpyAsync(c->apair0, c->h_apair.data(), sizeof(int64_t) * ((size_t)n + 1),
                                cudaMemcpyHostToDevice, c->stream));
    if (!items.empty())
        CREATE_CUDA(cudaMemcpyAsync(c->item_u0, items.data(), sizeof(int32_t) * items.size(),
                                    cudaMemcpyHostToDevice, c->stream));
    CREATE_CUDA(cudaMemsetAsync(c->counter, 0, sizeof(int32_t) * (size_t)n, c->stream));
    CREATE_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(int32_t), c->stream));
    if (c->bulk || c->partition) {
        const size_t M = c->mb_C.size();
        CREATE_CUDA(cudaMemcpyAsync(c->d_mb_item_base, c->mb_item_base.data(),
                                    sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, c->stream));
        CREATE_CUDA(cudaMemcpyAsync(c->d_mb_C, c->mb_C.data(), sizeof(int32_t) * M,
                                    cudaMemcpyHostToDevice, c->stream));
    }
    if (c->bulk) {
        const size_t M = c->mb_C.size();
        CREATE_CUDA(cudaMemsetAsync(c->row_flag, 0, sizeof(int32_t) * (size_t)n, c->stream));
        CREATE_CUDA(cudaMemsetAsync(c->mb_done, 0, sizeof(int32_t) * 2 * M, c->stream));
    }
    CREATE_CUDA(launch_init(c));
    CREATE_CUDA(cudaStreamSynchronize(c->stream));
#undef CREATE_CUDA
    *out = c;
    return F2V_OK;
}

}  // namespace

f2v_status f2v_create_ex(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                         f2v_model model, int32_t s, float lr, int32_t minibatch,
                         uint64_t seed, f2v_precision precision, uint32_t flags,
                         void *stream, f2v_ctx **out)
{
    return create_impl(row_ptr, col_idx, n, d, model, s, 0, lr, minibatch, seed, precision,
                       flags, stream, out);
}

f2v_status f2v_create_rw(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t d,
                         f2v_model model, int32_t s, int32_t walk_length, float lr,
                         int32_t minibatch, uint64_t seed, f2v_precision precision,
                         uint32_t flags, void *stream, f2v_ctx **out)
{
    if (out) *out = nullptr;
    if (walk_length < 1 || walk_length > kMaxWalk)
        return fail(nullptr, F2V_EINVAL, "walk_length = %d, must be in [1, %d]", walk_length,
                    kMaxWalk);
    return create_impl(row_ptr, col_idx, n, d, model, s, walk_length, lr, minibatch, seed,
                       precision, flags, stream, out);
}

void f2v_destroy(f2v_ctx *ctx)
{
    if (!ctx) return;
    if (!ctx->failed) cudaStreamSynchronize(ctx->stream);
    release(ctx);
    delete ctx;
}

f2v_status f2v_epoch(f2v_ctx *ctx)
{
    F2V_CHECK_CTX(ctx);
    DeviceGuard g(ctx->device);
    return run_epoch(ctx);
}

f2v_status f2v_train(f2v_ctx *ctx, int32_t epochs)
{
    F2V_CHECK_CTX(ctx);
    if (epochs < 0) return fail(ctx, F2V_EINVAL, "epochs = %d < 0", epochs);
    DeviceGuard g(ctx->device);
    for (int32_t i = 0; i < epochs; ++i) {
        f2v_status st = run_epoch(ctx);
        if (st != F2V_OK) return st;
    }
    return F2V_OK;
}

f2v_status f2v_run_minibatches(f2v_ctx *ctx, int32_t count)
{
    F2V_CHECK_CTX(ctx);
    if (count < 0) return fail(ctx, F2V_EINVAL, "count = %d < 0", count);
    DeviceGuard g(ctx->device);
    const int M = num_minibatches(ctx);
    while (count > 0) {
        const int k0 = ctx->mb_pos;
        const int k1 = std::min(M, k0 + count);
        f2v_status st = run_range(ctx, k0, k1);
        if (st != F2V_OK) return st;
        advance(ctx, k1 - k0);
        count -= k1 - k0;
    }
    return F2V_OK;
}

f2v_status f2v_get_progress(const f2v_ctx *ctx, int32_t *epoch, int32_t *minibatch)
{
    if (!ctx || !epoch || !minibatch) return fail(nullptr, F2V_EINVAL, "null argument");
    *epoch = ctx->epoch;
    *minibatch = ctx->mb_pos;
    return F2V_OK;
}

f2v_status f2v_synchronize(f2v_ctx *ctx)
{
    F2V_CHECK_CTX(ctx);
    DeviceGuard g(ctx->device);
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    F2V_CUDA(ctx, cudaGetLastError());
    return check_device_error(ctx);
}

f2v_status f2v_get_embedding(f2v_ctx *ctx, float *out, size_t count)
{
    F2V_CHECK_CTX(ctx);
    if (!out) return fail(ctx, F2V_EINVAL, "out is NULL");
    const size_t want = (size_t)ctx->n * ctx->d;
    if (count != want) return fail(ctx, F2V_EINVAL, "count = %zu, expected n*d = %zu", count, want);
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    const float *src = ctx->precision == F2V_BF16 ? ctx->master : (const float *)ctx->z[ctx->cur];
    F2V_CUDA(ctx, cudaMemcpyAsync(out, src, want * sizeof(float), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

f2v_status f2v_get_embedding_device(f2v_ctx *ctx, float *dev_out, size_t count)
{
    F2V_CHECK_CTX(ctx);
    if (!dev_out) return fail(ctx, F2V_EINVAL, "dev_out is NULL");
    const size_t want = (size_t)ctx->n * ctx->d;
    if (count != want) return fail(ctx, F2V_EINVAL, "count = %zu, expected n*d = %zu", count, want);
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    const float *src = ctx->precision == F2V_BF16 ? ctx->master : (const float *)ctx->z[ctx->cur];
    F2V_CUDA(ctx, cudaMemcpyAsync(dev_out, src, want * sizeof(float), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return F2V_OK;
}

f2v_status f2v_set_embedding(f2v_ctx *ctx, const float *z, size_t count)
{
    F2V_CHECK_CTX(ctx);
    if (!z) return fail(ctx, F2V_EINVAL, "z is NULL");
    const size_t want = (size_t)ctx->n * ctx->d;
    if (count != want) return fail(ctx, F2V_EINVAL, "count = %zu, expected n*d = %zu", count, want);
    DeviceGuard g(ctx->device);
    if (ctx->precision == F2V_BF16) {
        F2V_CUDA(ctx, cudaMemcpyAsync(ctx->master, z, want * sizeof(float), cudaMemcpyHostToDevice,
                                      ctx->stream));
        const int blocks = (int)std::min<int64_t>(((int64_t)want + 255) / 256, 152 * 16);
        round_rows_kernel<__nv_bfloat16><<<blocks, 256, 0, ctx->stream>>>(
            (__nv_bfloat16 *)ctx->z[ctx->cur], ctx->master, (int64_t)want);
        ctx->launches++;
        F2V_CUDA(ctx, cudaGetLastError());
    } else {
        F2V_CUDA(ctx, cudaMemcpyAsync(ctx->z[ctx->cur], z, want * sizeof(float),
                                      cudaMemcpyHostToDevice, ctx->stream));
    }
    if (ctx->mb_pos > 0 && ctx->partition) {
        // mid-epoch: the epoch reads Z in its order, updated positions from z[2]
        const size_t rows = std::min<size_t>((size_t)ctx->mb_pos * ctx->b, (size_t)ctx->n);
        F2V_CUDA(ctx, launch_permute_rows((const float *)ctx->z[ctx->cur],
                                          (float *)ctx->z[ctx->cur ^ 1], ctx->perm, ctx->n,
                                          ctx->ld, false, ctx->stream));
        F2V_CUDA(ctx, launch_permute_rows((const float *)ctx->z[ctx->cur], (float *)ctx->z[2],
                                          ctx->perm, (int64_t)rows, ctx->ld, false, ctx->stream));
        ctx->launches += 2;
    } else if (ctx->mb_pos > 0) {   // mid-epoch: updated rows are read from the next buffer
        const size_t rows = std::min<size_t>((size_t)ctx->mb_pos * ctx->b, (size_t)ctx->n);
        F2V_CUDA(ctx, cudaMemcpyAsync(ctx->z[ctx->cur ^ 1], ctx->z[ctx->cur],
                                      rows * (size_t)ctx->ld * elem_size(ctx),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    }
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return F2V_OK;
}

f2v_status f2v_set_lr(f2v_ctx *ctx, float lr)
{
    F2V_CHECK_CTX(ctx);
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(ctx, F2V_EINVAL, "lr must be finite and > 0");
    ctx->lr = lr;
    return F2V_OK;
}

f2v_status f2v_set_schedule(f2v_ctx *ctx, f2v_schedule schedule, int32_t total_epochs)
{
    F2V_CHECK_CTX(ctx);
    if (schedule != F2V_LR_CONSTANT && schedule != F2V_LR_LINEAR)
        return fail(ctx, F2V_EINVAL, "unknown schedule %d", (int)schedule);
    if (schedule == F2V_LR_LINEAR && total_epochs < 1)
        return fail(ctx, F2V_EINVAL, "linear schedule needs total_epochs >= 1");
    ctx->schedule = schedule;
    ctx->total_epochs = total_epochs;
    return F2V_OK;
}

f2v_status f2v_set_epoch(f2v_ctx *ctx, int32_t epoch)
{
    F2V_CHECK_CTX(ctx);
    if (epoch < 0) return fail(ctx, F2V_EINVAL, "epoch = %d < 0", epoch);
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    // row flags name the epoch a row was written in; a counter that moves
    // (backwards, or to an epoch run before) must not meet stale flags
    if (ctx->row_flag)
        F2V_CUDA(ctx, cudaMemsetAsync(ctx->row_flag, 0, sizeof(int32_t) * (size_t)ctx->n,
                                      ctx->stream));
    ctx->mb_pos = 0;
    ctx->epoch = epoch;
    return F2V_OK;
}

f2v_status f2v_get_epoch(const f2v_ctx *ctx, int32_t *epoch)
{
    if (!ctx || !epoch) return fail(nullptr, F2V_EINVAL, "null argument");
    *epoch = ctx->epoch;
    return F2V_OK;
}

f2v_status f2v_set_stream(f2v_ctx *ctx, void *stream)
{
    F2V_CHECK_CTX(ctx);
    DeviceGuard g(ctx->device);
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->stream = (cudaStream_t)stream;
    return F2V_OK;
}

f2v_status f2v_eval_auc(f2v_ctx *ctx, const int32_t *pos_pairs, int64_t npos,
                        const int32_t *neg_pairs, int64_t nneg, double *auc)
{
    F2V_CHECK_CTX(ctx);
    if (!auc) return fail(ctx, F2V_EINVAL, "auc is NULL");
    if (npos < 1 || nneg < 1 || !pos_pairs || !neg_pairs)
        return fail(ctx, F2V_EINVAL, "need at least one positive and one negative pair");
    for (int64_t i = 0; i < 2 * npos; ++i)
        if (pos_pairs[i] < 0 || pos_pairs[i] >= ctx->n)
            return fail(ctx, F2V_EINVAL, "pos_pairs[%lld] out of range", (long long)i);
    for (int64_t i = 0; i < 2 * nneg; ++i)
        if (neg_pairs[i] < 0 || neg_pairs[i] >= ctx->n)
            return fail(ctx, F2V_EINVAL, "neg_pairs[%lld] out of range", (long long)i);
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    std::string err;
    const float *zf = ctx->precision == F2V_BF16 ? ctx->master : (const float *)ctx->z[ctx->cur];
    cudaError_t e = eval_auc_device(zf, nullptr, ctx->d, ctx->model, pos_pairs, npos, neg_pairs,
                                    nneg, ctx->stream, auc, &err);
    ctx->launches += 3;
    if (e == cudaErrorMemoryAllocation) return fail(ctx, F2V_ENOMEM, "eval_auc: %s", err.c_str());
    if (e != cudaSuccess) return fail(ctx, F2V_ECUDA, "eval_auc: %s", err.c_str());
    return F2V_OK;
}

f2v_status f2v_eval_loss(f2v_ctx *ctx, int32_t epoch, double *loss)
{
    F2V_CHECK_CTX(ctx);
    if (!loss) return fail(ctx, F2V_EINVAL, "loss is NULL");
    if (epoch < 0) return fail(ctx, F2V_EINVAL, "epoch < 0");
    if (ctx->model != F2V_TDIST && ctx->model != F2V_SIGMOID)
        return fail(ctx, F2V_EINVAL,
                    "eval_loss: the loss of Eq. 2 is defined for the t and sigmoid models only");
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    std::string err;
    const float *zf = ctx->precision == F2V_BF16 ? ctx->master : (const float *)ctx->z[ctx->cur];
    // the graph as given (with a random partition the kernels walk a relabelled copy)
    cudaError_t e = eval_loss_device(zf, ctx->d, ctx->model, ctx->row_ptr0, ctx->col_idx0, ctx->n,
                                     ctx->nnz, ctx->s, (uint32_t)epoch, (uint32_t)ctx->seed,
                                     (uint32_t)(ctx->seed >> 32), ctx->stream, loss, &err);
    ctx->launches += 2;
    if (e == cudaErrorMemoryAllocation) return fail(ctx, F2V_ENOMEM, "eval_loss: %s", err.c_str());
    if (e != cudaSuccess) return fail(ctx, F2V_ECUDA, "eval_loss: %s", err.c_str());
    return F2V_OK;
}

f2v_status f2v_debug_samples(f2v_ctx *ctx, int32_t epoch, int32_t *out, size_t count)
{
    F2V_CHECK_CTX(ctx);
    if (!out) return fail(ctx, F2V_EINVAL, "out is NULL");
    if (epoch < 0) return fail(ctx, F2V_EINVAL, "epoch < 0");
    const size_t want = (size_t)ctx->n * ctx->s;
    if (count != want) return fail(ctx, F2V_EINVAL, "count = %zu, expected n*s = %zu", count, want);
    if (want == 0) return F2V_OK;
    DeviceGuard g(ctx->device);
    int32_t *dbuf = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dbuf, want * sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return fail(ctx, F2V_ENOMEM, "debug_samples: %s", cudaGetErrorString(e));
    // shared samples under a random partition: a vertex's minibatch is its
    // position in that epoch's order
    int32_t *tperm = nullptr, *trank = nullptr;
    if (ctx->partition && ctx->shared) {
        // (the side stream may be building the next order with the scratch)
        if (ctx->xstream) F2V_CUDA(ctx, cudaStreamSynchronize(ctx->xstream));
        e = cudaMallocAsync((void **)&tperm, sizeof(int32_t) * (size_t)ctx->n, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void **)&trank, sizeof(int32_t) * (size_t)ctx->n, ctx->stream);
        if (e != cudaSuccess) return fail(ctx, F2V_ENOMEM, "debug_samples: %s", cudaGetErrorString(e));
        F2V_CUDA(ctx, launch_partition(ctx->n, (uint32_t)epoch, (uint32_t)ctx->seed,
                                       (uint32_t)(ctx->seed >> 32), ctx->pw, tperm, trank,
                                       ctx->stream));
        ctx->launches += 3;
    }
    const int blocks = (int)std::min<int64_t>(((int64_t)want + 255) / 256, 152 * 16);
    samples_kernel<<<blocks, 256, 0, ctx->stream>>>(dbuf, ctx->n, ctx->s,
                                                     ctx->shared ? ctx->b : 0, trank,
                                                     (uint32_t)epoch, (uint32_t)ctx->seed,
                                                     (uint32_t)(ctx->seed >> 32));
    if (tperm) F2V_CUDA(ctx, cudaFreeAsync(tperm, ctx->stream));
    if (trank) F2V_CUDA(ctx, cudaFreeAsync(trank, ctx->stream));
    ctx->launches++;
    F2V_CUDA(ctx, cudaGetLastError());
    F2V_CUDA(ctx, cudaMemcpyAsync(out, dbuf, want * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    F2V_CUDA(ctx, cudaFreeAsync(dbuf, ctx->stream));
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return F2V_OK;
}

f2v_status f2v_eval_link_lr(f2v_ctx *ctx, const int32_t *pos_pairs, int64_t npos,
                            const int32_t *neg_pairs, int64_t nneg, const uint8_t *train_mask,
                            double *accuracy, double *theta)
{
    F2V_CHECK_CTX(ctx);
    if (!accuracy || !train_mask) return fail(ctx, F2V_EINVAL, "null argument");
    if (npos < 0 || nneg < 0 || (npos > 0 && !pos_pairs) || (nneg > 0 && !neg_pairs))
        return fail(ctx, F2V_EINVAL, "bad pair lists");
    if (!pairs_in_range(pos_pairs, npos, ctx->n) || !pairs_in_range(neg_pairs, nneg, ctx->n))
        return fail(ctx, F2V_EINVAL, "a pair names a vertex out of range");
    if (lr_smem_bytes(ctx->d) > 227 * 1024)
        return fail(ctx, F2V_EINVAL, "link prediction needs d <= 150 (d = %d)", ctx->d);
    const int64_t total = npos + nneg;
    std::vector<int64_t> tr, te;
    for (int64_t i = 0; i < total; ++i) (train_mask[i] ? tr : te).push_back(i);
    if (tr.empty() || te.empty())
        return fail(ctx, F2V_EINVAL, "need at least one training and one test pair");
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    const float *zf = ctx->precision == F2V_BF16 ? ctx->master : (const float *)ctx->z[ctx->cur];
    const int D1 = ctx->d + 1;
    Scratch sc(ctx->stream);
    int32_t *dpos = nullptr, *dneg = nullptr;
    int64_t *dtr = nullptr, *dte = nullptr;
    double *dth = nullptr, *dg = nullptr, *dH = nullptr, *dstep = nullptr;
    unsigned long long *dcorrect = nullptr;
    cudaError_t e = sc.get(&dpos, 2 * (size_t)npos);
    if (e == cudaSuccess) e = sc.get(&dneg, 2 * (size_t)nneg);
    if (e == cudaSuccess) e = sc.get(&dtr, tr.size());
    if (e == cudaSuccess) e = sc.get(&dte, te.size());
    if (e == cudaSuccess) e = sc.get(&dth, (size_t)D1);
    if (e == cudaSuccess) e = sc.get(&dg, (size_t)D1);
    if (e == cudaSuccess) e = sc.get(&dH, (size_t)D1 * D1);
    if (e == cudaSuccess) e = sc.get(&dstep, 1);
    if (e == cudaSuccess) e = sc.get(&dcorrect, 1);
    if (e != cudaSuccess) return fail(ctx, F2V_ENOMEM, "eval_link_lr: %s", cudaGetErrorString(e));
    if (npos)
        F2V_CUDA(ctx, cudaMemcpyAsync(dpos, pos_pairs, sizeof(int32_t) * 2 * npos,
                                      cudaMemcpyHostToDevice, ctx->stream));
    if (nneg)
        F2V_CUDA(ctx, cudaMemcpyAsync(dneg, neg_pairs, sizeof(int32_t) * 2 * nneg,
                                      cudaMemcpyHostToDevice, ctx->stream));
    F2V_CUDA(ctx, cudaMemcpyAsync(dtr, tr.data(), sizeof(int64_t) * tr.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    F2V_CUDA(ctx, cudaMemcpyAsync(dte, te.data(), sizeof(int64_t) * te.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    F2V_CUDA(ctx, cudaMemsetAsync(dth, 0, sizeof(double) * D1, ctx->stream));
    for (int it = 0; it < 100; ++it) {   // Newton steps
        F2V_CUDA(ctx, cudaMemsetAsync(dg, 0, sizeof(double) * D1, ctx->stream));
        F2V_CUDA(ctx, cudaMemsetAsync(dH, 0, sizeof(double) * D1 * D1, ctx->stream));
        F2V_CUDA(ctx, launch_lr_newton(zf, ctx->d, dpos, npos, dneg, dtr, (int64_t)tr.size(), dth,
                                       dg, dH, ctx->stream));
        F2V_CUDA(ctx, launch_lr_solve(ctx->d, dH, dg, dth, dstep, ctx->stream));
        ctx->launches += 2;
        double step = 0.0;
        F2V_CUDA(ctx, cudaMemcpyAsync(&step, dstep, sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (!(step >= 1e-10)) break;      // converged (or not a number)
    }
    F2V_CUDA(ctx, cudaMemsetAsync(dcorrect, 0, sizeof(unsigned long long), ctx->stream));
    F2V_CUDA(ctx, launch_lr_accuracy(zf, ctx->d, dpos, npos, dneg, dte, (int64_t)te.size(), dth,
                                     dcorrect, ctx->stream));
    ctx->launches++;
    unsigned long long correct = 0;
    F2V_CUDA(ctx, cudaMemcpyAsync(&correct, dcorrect, sizeof(correct), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    if (theta)
        F2V_CUDA(ctx, cudaMemcpyAsync(theta, dth, sizeof(double) * D1, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *accuracy = (double)correct / (double)te.size();
    return F2V_OK;
}

f2v_status f2v_eval_kmeans(f2v_ctx *ctx, int32_t k, const int32_t *init, int32_t iters,
                           int32_t *labels, double *modularity, int32_t *rounds)
{
    F2V_CHECK_CTX(ctx);
    if (!init || !modularity) return fail(ctx, F2V_EINVAL, "null argument");
    if (k < 1 || k > 64) return fail(ctx, F2V_EINVAL, "k = %d, must be in [1, 64]", k);
    if (ctx->d > 256) return fail(ctx, F2V_EINVAL, "k-means needs d <= 256 (d = %d)", ctx->d);
    if (iters < 1) return fail(ctx, F2V_EINVAL, "iters = %d < 1", iters);
    for (int c = 0; c < k; ++c)
        if (init[c] < 0 || init[c] >= ctx->n)
            return fail(ctx, F2V_EINVAL, "init[%d] out of range", c);
    DeviceGuard g(ctx->device);
    f2v_status st = sync_current(ctx);
    if (st != F2V_OK) return st;
    const float *zf = ctx->precision == F2V_BF16 ? ctx->master : (const float *)ctx->z[ctx->cur];
    const int32_t n = ctx->n, d = ctx->d;
    Scratch sc(ctx->stream);
    int32_t *dinit = nullptr, *dlab = nullptr;
    double *dC = nullptr, *dsum = nullptr, *dq = nullptr;
    unsigned long long *dcnt = nullptr, *dchg = nullptr, *de = nullptr, *dD = nullptr;
    cudaError_t e = sc.get(&dinit, (size_t)k);
    if (e == cudaSuccess) e = sc.get(&dlab, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&dC, (size_t)k * d);
    if (e == cudaSuccess) e = sc.get(&dsum, (size_t)k * d);
    if (e == cudaSuccess) e = sc.get(&dq, 1);
    if (e == cudaSuccess) e = sc.get(&dcnt, (size_t)k);
    if (e == cudaSuccess) e = sc.get(&dchg, 1);
    if (e == cudaSuccess) e = sc.get(&de, (size_t)k);
    if (e == cudaSuccess) e = sc.get(&dD, (size_t)k);
    if (e != cudaSuccess) return fail(ctx, F2V_ENOMEM, "eval_kmeans: %s", cudaGetErrorString(e));
    F2V_CUDA(ctx, cudaMemcpyAsync(dinit, init, sizeof(int32_t) * k, cudaMemcpyHostToDevice,
                                  ctx->stream));
    F2V_CUDA(ctx, launch_km_init(zf, d, dinit, k, dC, ctx->stream));
    F2V_CUDA(ctx, cudaMemsetAsync(dlab, 0xFF, sizeof(int32_t) * n, ctx->stream));
    ctx->launches++;
    int it = 0;
    for (it = 1; it <= iters; ++it) {   // Lloyd rounds
        F2V_CUDA(ctx, cudaMemsetAsync(dsum, 0, sizeof(double) * k * d, ctx->stream));
        F2V_CUDA(ctx, cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long) * k, ctx->stream));
        F2V_CUDA(ctx, cudaMemsetAsync(dchg, 0, sizeof(unsigned long long), ctx->stream));
        F2V_CUDA(ctx, launch_km_assign(zf, n, d, dC, k, dlab, dsum, dcnt, dchg, ctx->stream));
        ctx->launches++;
        unsigned long long changed = 0;
        F2V_CUDA(ctx, cudaMemcpyAsync(&changed, dchg, sizeof(changed), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (changed == 0) break;
        F2V_CUDA(ctx, launch_km_update(k, d, dsum, dcnt, dC, ctx->stream));
        ctx->launches++;
    }
    F2V_CUDA(ctx, cudaMemsetAsync(de, 0, sizeof(unsigned long long) * k, ctx->stream));
    F2V_CUDA(ctx, cudaMemsetAsync(dD, 0, sizeof(unsigned long long) * k, ctx->stream));
    F2V_CUDA(ctx, launch_modularity(ctx->row_ptr0, ctx->col_idx0, n, ctx->nnz, dlab, k, de, dD,
                                    dq, ctx->stream));
    ctx->launches += 2;
    F2V_CUDA(ctx, cudaMemcpyAsync(modularity, dq, sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    if (labels)
        F2V_CUDA(ctx, cudaMemcpyAsync(labels, dlab, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (rounds) *rounds = std::min(it, iters);
    return F2V_OK;
}

f2v_status f2v_debug_wait(f2v_ctx *ctx, int32_t kind)
{
    F2V_CHECK_CTX(ctx);
    if (kind < 0 || kind > 3) return fail(ctx, F2V_EINVAL, "kind = %d, must be in [0, 3]", kind);
    DeviceGuard g(ctx->device);
    int32_t *cells = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&cells, 2 * sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return fail(ctx, F2V_ENOMEM, "debug_wait: %s", cudaGetErrorString(e));
    F2V_CUDA(ctx, cudaMemsetAsync(cells, 0, 2 * sizeof(int32_t), ctx->stream));
    F2V_CUDA(ctx, launch_wait_probe(cells, kind, ctx->err_word, ctx->stream));
    ctx->launches++;
    F2V_CUDA(ctx, cudaFreeAsync(cells, ctx->stream));
    return check_device_error(ctx);
}

f2v_status f2v_debug_walks(f2v_ctx *ctx, int32_t epoch, int32_t *out, size_t count)
{
    F2V_CHECK_CTX(ctx);
    if (!out) return fail(ctx, F2V_EINVAL, "out is NULL");
    if (epoch < 0) return fail(ctx, F2V_EINVAL, "epoch < 0");
    if (ctx->walk < 1) return fail(ctx, F2V_ESTATE, "the context has no walks (f2v_create_rw)");
    const size_t want = (size_t)ctx->n * (size_t)ctx->walk;
    if (count != want)
        return fail(ctx, F2V_EINVAL, "count = %zu, expected n*walk_length = %zu", count, want);
    DeviceGuard g(ctx->device);
    const size_t slots = (size_t)ctx->h_apair[(size_t)ctx->n];
    int32_t *list = nullptr, *dout = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&list, slots * sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dout, want * sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) {
        if (list) cudaFreeAsync(list, ctx->stream);
        return fail(ctx, F2V_ENOMEM, "debug_walks: %s", cudaGetErrorString(e));
    }
    // the list the epoch's force launches read, written by the same kernel
    F2V_CUDA(ctx, launch_partner_list(ctx, epoch, list, ctx->stream, true));
    F2V_CUDA(ctx, launch_extract_walks(ctx->apair0, ctx->row_ptr0, ctx->n, ctx->walk, list, dout,
                                       ctx->stream));
    ctx->launches++;
    F2V_CUDA(ctx, cudaMemcpyAsync(out, dout, want * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    F2V_CUDA(ctx, cudaFreeAsync(list, ctx->stream));
    F2V_CUDA(ctx, cudaFreeAsync(dout, ctx->stream));
    F2V_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return F2V_OK;
}

f2v_status f2v_pairs_per_epoch(const f2v_ctx *ctx, int64_t *pairs)
{
    if (!ctx || !pairs) return fail(nullptr, F2V_EINVAL, "null argument");
    *pairs = ctx->pairs;
    return F2V_OK;
}

f2v_status f2v_device_bytes(const f2v_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return fail(nullptr, F2V_EINVAL, "null argument");
    *bytes = ctx->device_bytes;
    return F2V_OK;
}

f2v_status f2v_launch_count(const f2v_ctx *ctx, int64_t *launches)
{
    if (!ctx || !launches) return fail(nullptr, F2V_EINVAL, "null argument");
    *launches = ctx->launches;
    return F2V_OK;
}

f2v_status f2v_set_kernel_timing(f2v_ctx *ctx, int32_t enable)
{
    F2V_CHECK_CTX(ctx);
    ctx->timing = enable != 0;
    return F2V_OK;
}

f2v_status f2v_read_kernel_timing(f2v_ctx *ctx, int64_t *launches, double *total_ms)
{
    F2V_CHECK_CTX(ctx);
    if (!launches || !total_ms) return fail(ctx, F2V_EINVAL, "null argument");
    DeviceGuard g(ctx->device);
    f2v_status st = collect_timing(ctx);
    if (st != F2V_OK) return st;
    *launches = ctx->timed_launches;
    *total_ms = ctx->timed_ms;
    ctx->timed_launches = 0;
    ctx->timed_ms = 0.0;
    return F2V_OK;
}

const char *f2v_last_error(const f2v_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

const char *f2v_last_error_global(void) { return g_last_error.c_str(); }

}  // extern "C"
