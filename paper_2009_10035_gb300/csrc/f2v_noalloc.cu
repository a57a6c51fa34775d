// f2v_noalloc.cu -- one minibatch of the force+update step on caller-owned
// device buffers, with no device allocation at all.
//
// Some callers cannot allocate device memory while they run this step: code
// that owns every byte of device memory through its own allocator or arena
// (and forbids libraries from calling cudaMalloc behind its back), code that
// must not stall on the driver's allocation path inside a latency budget, or
// code whose memory is planned ahead for the whole run.  f2v_create serves
// none of them, since a context allocates its buffers.  This entry point
// takes the graph and both embedding buffers from the caller and keeps its
// scratch (pair prefix, item table, partial sums of vertices split across
// items, arrival counters) in one fixed file-scope device array.
//
// The scratch array is kNoAllocScratchBytes (8 MiB).  Every device that
// loads this library holds it until the process exits.  All calls share it
// and it keeps the last call's contents: the counters that must start at
// zero are cleared at the start of each call, and two calls whose work
// overlaps on the GPU (different streams, or different host threads on one
// device) race on it and give wrong results.  The first call on a device
// looks up the array's device address (cudaGetSymbolAddress) with that
// device current; make that first call before any stream capture.  The
// address is kept for the life of the process: after a cudaDeviceReset (or
// anything else that re-creates the device's primary context) the kept
// address is stale, so this entry point must not be used on that device
// again.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <mutex>
#include <string>

#include "f2v.h"
#include "f2v_force.cuh"
#include "f2v_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kMaxDevices] = {};
thread_local std::string g_noalloc_error;

f2v_status noalloc_fail(f2v_status st, const char *msg)
{
    g_noalloc_error = msg;
    return st;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once
// per device).
f2v_status scratch_address(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(F2V_ECUDA, "f2v_minibatch_noalloc: no usable current device");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            g_noalloc_error = std::string("f2v_minibatch_noalloc: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e);
            return F2V_ECUDA;
        }
        g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_addr[dev];
    return F2V_OK;
}

// Exclusive prefix of the per-vertex pair counts c(u) = deg(u) + s (one empty
// pair if that is 0) over vertices [u_begin, u_begin + count), one block.
__global__ void noalloc_prefix_kernel(const int32_t *row_ptr, int s, int u_begin, int count,
                                      int64_t *prefix)
{
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int per = (count + blockDim.x - 1) / blockDim.x;
    const int lo = min(count, t * per), hi = min(count, lo + per);
    int64_t sum = 0;
    for (int i = lo; i < hi; ++i) {
        const int u = u_begin + i;
        int64_t c = (int64_t)(row_ptr[u + 1] - row_ptr[u]) + s;
        sum += c == 0 ? 1 : c;
    }
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    int64_t run = part[t];
    for (int i = lo; i < hi; ++i) {
        prefix[i] = run;
        const int u = u_begin + i;
        int64_t c = (int64_t)(row_ptr[u + 1] - row_ptr[u]) + s;
        run += c == 0 ? 1 : c;
    }
    if (hi == count && lo < hi) prefix[count] = run;
    if (count == 0 && t == 0) prefix[0] = 0;
}

// item_u0[i] = the vertex whose pairs contain pair i * C of the minibatch.
__global__ void noalloc_items_kernel(const int64_t *prefix, int mb_count, int C, int n_items,
                                     int u_begin, int32_t *item_u0)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_items;
         i += gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)i * C;
        int lo = 0, hi = mb_count - 1;          // last j with prefix[j] <= q
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= q) lo = mid; else hi = mid - 1;
        }
        item_u0[i] = u_begin + lo;
    }
}

}  // namespace

extern "C" const char *f2v_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" f2v_status f2v_minibatch_noalloc(const int32_t *row_ptr, const int32_t *col_idx,
                                            int32_t n, int32_t d, f2v_model model, int32_t s,
                                            float eta, uint64_t seed, int32_t epoch,
                                            int32_t mb_begin, int32_t mb_end,
                                            const float *z_cur, float *z_next, void *stream)
{
    using namespace f2v;
    g_noalloc_error.clear();
    if (!row_ptr || !col_idx || !z_cur || !z_next)
        return noalloc_fail(F2V_EINVAL, "f2v_minibatch_noalloc: a pointer is NULL");
    if (n < 1 || d < 1 || d > 1024 || s < 0 || s > 65534 || epoch < 0)
        return noalloc_fail(F2V_EINVAL, "f2v_minibatch_noalloc: n, d, s or epoch out of range");
    // The kernel reads and writes rows of Z with VEC-wide vector accesses
    // (16 bytes for most d, 8 for d = 2), and the CSR as 4-byte words.  The
    // buffers come from the caller's own allocator, so a misaligned pointer
    // is possible here; it would fault on the GPU, so it is refused first.
    const Shape sh = choose_shape(d);
    const uintptr_t zalign = (uintptr_t)(sh.VEC * sizeof(float));
    if (((uintptr_t)z_cur % zalign) != 0 || ((uintptr_t)z_next % zalign) != 0)
        return noalloc_fail(F2V_EINVAL,
                            "f2v_minibatch_noalloc: z_cur and z_next must be aligned to "
                            "16 bytes (8 for d = 2, 4 for d not in {2,4,8,...,1024})");
    if (((uintptr_t)row_ptr % 4) != 0 || ((uintptr_t)col_idx % 4) != 0)
        return noalloc_fail(F2V_EINVAL,
                            "f2v_minibatch_noalloc: row_ptr and col_idx must be 4-byte aligned");
    if (model < F2V_TDIST || model > F2V_FORCEATLAS)
        return noalloc_fail(F2V_EINVAL, "f2v_minibatch_noalloc: unknown model");
    if (!(eta > 0.f) || eta != eta || eta > 3.0e38f)
        return noalloc_fail(F2V_EINVAL, "f2v_minibatch_noalloc: eta must be finite and > 0");
    if (mb_begin < 0 || mb_end > n || mb_begin >= mb_end)
        return noalloc_fail(F2V_EINVAL, "f2v_minibatch_noalloc: need 0 <= mb_begin < mb_end <= n");
    cudaStream_t st = (cudaStream_t)stream;
    const int C = items_pairs(sh);
    const int mb_count = mb_end - mb_begin;
    // the kernel's decode window reads the pair prefix up to 32 vertices past
    // the minibatch
    const int win = std::min(n, mb_end + 32) - mb_begin;

    // fixed part of the scratch: pair prefix, final counters, error word
    size_t off = 0;
    const size_t off_prefix = off;
    off = align256(off + sizeof(int64_t) * ((size_t)win + 1));
    const size_t off_counter = off;
    off = align256(off + sizeof(int32_t) * (size_t)mb_count);
    const size_t off_err = off;
    off = align256(off + sizeof(int32_t));
    if (off > kNoAllocScratchBytes)
        return noalloc_fail(F2V_EINVAL,
                            "f2v_minibatch_noalloc: minibatch too large for the 8 MiB scratch");

    unsigned char *scratch = nullptr;
    f2v_status rc = scratch_address(&scratch);
    if (rc != F2V_OK) return rc;
    int64_t *prefix = reinterpret_cast<int64_t *>(scratch + off_prefix);

    noalloc_prefix_kernel<<<1, 1024, 0, st>>>(row_ptr, s, mb_begin, win, prefix);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(F2V_ECUDA, "f2v_minibatch_noalloc: prefix kernel launch failed");
    int64_t Pk = 0;
    e = cudaMemcpyAsync(&Pk, prefix + mb_count, sizeof Pk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return noalloc_fail(F2V_ECUDA, "f2v_minibatch_noalloc: reading the pair count failed");
    if (Pk < 1 || Pk >= (int64_t)INT32_MAX - C)
        return noalloc_fail(F2V_EINVAL, "f2v_minibatch_noalloc: pair count out of range");
    const int64_t n_items = (Pk + C - 1) / C;

    // variable part: item table, combine-tree slots and counters
    const size_t off_items = off;
    off = align256(off + sizeof(int32_t) * (size_t)n_items);
    size_t slot_rows = 0, unit_counters = 0;
    {
        int64_t units = n_items;
        int levels = 0;
        while (true) {
            slot_rows += 2 * (size_t)units;
            if (levels > 0) unit_counters += 2 * (size_t)units;
            levels++;
            if (units <= 1 || levels == kMaxLevels) break;
            units = (units + kFan - 1) / kFan;
        }
    }
    const size_t off_slots = off;
    off = align256(off + sizeof(float) * (size_t)d * slot_rows);
    const size_t off_ucnt = off;
    off = align256(off + sizeof(int32_t) * (unit_counters + 1));
    if (off > kNoAllocScratchBytes)
        return noalloc_fail(F2V_EINVAL,
                            "f2v_minibatch_noalloc: minibatch pairs x d too large for the 8 MiB "
                            "scratch");

    int32_t *counter = reinterpret_cast<int32_t *>(scratch + off_counter);
    int32_t *item_u0 = reinterpret_cast<int32_t *>(scratch + off_items);
    int32_t *ucnt = reinterpret_cast<int32_t *>(scratch + off_ucnt);
    // the arrival counters must start at zero
    e = cudaMemsetAsync(counter, 0, sizeof(int32_t) * (size_t)mb_count, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ucnt, 0, sizeof(int32_t) * (unit_counters + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + off_err, 0, sizeof(int32_t), st);
    if (e != cudaSuccess)
        return noalloc_fail(F2V_ECUDA, "f2v_minibatch_noalloc: clearing the counters failed");
    {
        const int blocks = (int)std::min<int64_t>((n_items + 255) / 256, 1024);
        noalloc_items_kernel<<<blocks, 256, 0, st>>>(prefix, mb_count, C, (int)n_items, mb_begin,
                                                     item_u0);
        if (cudaGetLastError() != cudaSuccess)
            return noalloc_fail(F2V_ECUDA, "f2v_minibatch_noalloc: item kernel launch failed");
    }

    ForceArgs<float> a{};
    a.row_ptr = row_ptr;
    a.col_idx = col_idx;
    a.apair = prefix - mb_begin;            // indexed by global vertex id
    a.item_u0 = item_u0;
    a.zcur = z_cur;
    a.znext = z_next;
    a.master = nullptr;
    a.slots = reinterpret_cast<float *>(scratch + off_slots);
    a.unit_cnt = ucnt;
    a.units0 = n_items;
    a.counter = counter - mb_begin;         // indexed by global vertex id
    a.P0 = 0;
    a.Pk = (int32_t)Pk;
    a.n_items = (int32_t)n_items;
    a.mb_begin = mb_begin;
    a.mb_end = mb_end;
    a.n = n; a.d = d; a.ld = d; a.s = s;
    a.C = C;
    a.epoch = (uint32_t)epoch;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.eta = eta;
    a.model = (int32_t)model;
    a.err = reinterpret_cast<int32_t *>(scratch + off_err);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = launch_force_fp32(sh, a, std::max(sms, 1) * 8, st);
    if (e != cudaSuccess)
        return noalloc_fail(F2V_ECUDA, "f2v_minibatch_noalloc: force kernel launch failed");
    return F2V_OK;
}
