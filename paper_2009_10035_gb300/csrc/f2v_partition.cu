// f2v_partition.cu -- a new random partition of V into minibatches every
// epoch (the partition step of Algorithm 1: random minibatches, no vertex
// in two of them), as an option.
//
// Epoch e orders the vertices by the key Philox4x32-10(key, ctr = (v, e, 0,
// 3)).x0, ties by id (a stable radix sort of (key, v)); minibatch k is the
// positions [k b, (k+1) b) of that order.  The epoch then runs on the graph
// relabelled into that order, so that every kernel keeps its contiguous
// minibatches: vertex perm[p] becomes p, each row keeps its neighbours in
// CSR order with their ids mapped through rank, the pair prefix and the
// chunk tables are rebuilt for the new order, and Z is gathered into it
// (and scattered back when the epoch ends).  Counters of samples and walks
// keep the original ids (the partner-list kernels take perm and rank), so a
// vertex draws the same samples and walks whatever its position.
#include <cuda_runtime.h>

#include <algorithm>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "f2v_device.cuh"
#include "f2v_internal.h"

namespace f2v {

namespace {

int grid_of(int64_t threads)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<int64_t>(
        1, std::min<int64_t>((threads + 255) / 256, (int64_t)std::max(sms, 1) * 16));
}

__global__ void part_keys_kernel(uint32_t *__restrict__ keys, int32_t *__restrict__ vals,
                                 int32_t n, uint32_t epoch, uint32_t key0, uint32_t key1)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = philox_x0((uint32_t)v, epoch, 0u, 3u, key0, key1);
        vals[v] = (int32_t)v;
    }
}

__global__ void part_rank_kernel(const int32_t *__restrict__ perm, int32_t *__restrict__ rank,
                                 int32_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        rank[perm[p]] = (int32_t)p;
}

// Degree and force-pair count of the vertex at each position (entry n is 0,
// so that exclusive scans of n + 1 entries give the prefixes).
__global__ void part_counts_kernel(const int32_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ perm, int32_t n, int32_t s,
                                   int32_t walk, int32_t *__restrict__ deg,
                                   int64_t *__restrict__ cnt)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (p == n) {
            deg[p] = 0;
            cnt[p] = 0;
            continue;
        }
        const int32_t u = perm[p];
        const int32_t du = row_ptr[u + 1] - row_ptr[u];
        int64_t c = (walk > 0 ? (du > 0 ? walk : 0) : du) + s;
        if (c == 0) c = 1;   // the empty pair
        deg[p] = du;
        cnt[p] = c;
    }
}

// Row p of the relabelled CSR: the neighbours of perm[p], in order, as ranks.
__global__ void part_cols_kernel(const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col_idx,
                                 const int32_t *__restrict__ perm, const int32_t *__restrict__ rank,
                                 const int32_t *__restrict__ row_ptr2, int32_t *__restrict__ col2,
                                 int32_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < n; p += nwarps) {
        const int32_t u = perm[p];
        const int32_t lo = row_ptr[u], deg = row_ptr[u + 1] - lo, out = row_ptr2[p];
        // eight gathers in flight per lane (a hub's row is one warp's)
        for (int32_t j0 = 0; j0 < deg; j0 += 32 * 8) {
            int32_t v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int32_t j = j0 + 32 * t + lane;
                v[t] = (j < deg) ? col_idx[lo + j] : 0;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = rank[v[t]];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int32_t j = j0 + 32 * t + lane;
                if (j < deg) col2[out + j] = v[t];
            }
        }
    }
}

// Chunk size and chunk count of every minibatch (entry M of nch is 0).
__global__ void part_sizes_kernel(const int64_t *__restrict__ apair, int32_t n, int32_t b,
                                  int32_t M, int64_t W, int32_t Cfix, int32_t *__restrict__ mb_C,
                                  int64_t *__restrict__ nch)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= M;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (k == M) {
            nch[k] = 0;
            continue;
        }
        const int64_t u0 = k * (int64_t)b, u1 = min((int64_t)n, u0 + b);
        const int64_t Pk = apair[u1] - apair[u0];
        int64_t C = Cfix;
        if (W > 0) {   // staged kernel: two chunks per warp, a multiple of 32 pairs
            C = (Pk + W - 1) / W;
            C = max((int64_t)32, ((C + 1) / 2 + 31) / 32 * 32);
        }
        mb_C[k] = (int32_t)C;
        nch[k] = (Pk + C - 1) / C;
    }
}

// Start vertex of every chunk: block k serves minibatch k.
__global__ void part_items_kernel(const int64_t *__restrict__ apair,
                                  const int64_t *__restrict__ mb_base,
                                  const int32_t *__restrict__ mb_C, int32_t n, int32_t b,
                                  int32_t *__restrict__ items)
{
    const int64_t k = blockIdx.x;
    const int64_t u0 = k * (int64_t)b, u1 = min((int64_t)n, u0 + b);
    const int64_t P0 = apair[u0], C = mb_C[k];
    const int64_t base = mb_base[k], nch = mb_base[k + 1] - base;
    for (int64_t i = threadIdx.x; i < nch; i += blockDim.x) {
        const int64_t q = P0 + i * C;
        int64_t lo = u0, hi = u1 - 1;   // the last u in [u0, u1) with apair[u] <= q
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (apair[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        items[base + i] = (int32_t)lo;
    }
}

// P0 of every minibatch and the end of the last (M + 1 entries).
__global__ void part_p0_kernel(const int64_t *__restrict__ apair, int32_t n, int32_t b, int32_t M,
                               int64_t *__restrict__ p0)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= M;
         k += (int64_t)gridDim.x * blockDim.x)
        p0[k] = apair[min((int64_t)n, k * (int64_t)b)];
}

// dst[p] = src[perm[p]] (gather) or dst[perm[p]] = src[p] (scatter), rows
// p < rows: one warp per row, consecutive lanes on consecutive elements.
__global__ void permute_rows_kernel(const float *__restrict__ src, float *__restrict__ dst,
                                    const int32_t *__restrict__ perm, int64_t rows, int32_t d,
                                    bool scatter)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < rows; p += nwarps) {
        const int64_t v = perm[p];
        const float *s = src + (scatter ? p : v) * d;
        float *t = dst + (scatter ? v : p) * d;
        for (int32_t j = lane; j < d; j += 32) t[j] = s[j];
    }
}

}  // namespace

size_t partition_temp_bytes(int32_t n, int32_t M)
{
    size_t a = 0, b = 0, c = 0, d = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, a, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                    (const int32_t *)nullptr, (int32_t *)nullptr, n);
    cub::DeviceScan::ExclusiveSum(nullptr, b, (const int32_t *)nullptr, (int32_t *)nullptr, n + 1);
    cub::DeviceScan::ExclusiveSum(nullptr, c, (const int64_t *)nullptr, (int64_t *)nullptr, n + 1);
    cub::DeviceScan::ExclusiveSum(nullptr, d, (const int64_t *)nullptr, (int64_t *)nullptr, M + 1);
    return std::max(std::max(a, b), std::max(c, d));
}

cudaError_t launch_partition(int32_t n, uint32_t epoch, uint32_t key0, uint32_t key1,
                             const PartitionScratch &w, int32_t *perm, int32_t *rank,
                             cudaStream_t st)
{
    part_keys_kernel<<<grid_of(n), 256, 0, st>>>(w.keys, w.vals, n, epoch, key0, key1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t bytes = w.temp_bytes;
    e = cub::DeviceRadixSort::SortPairs(w.temp, bytes, w.keys, w.keys2, w.vals, perm, n, 0, 32,
                                        st);
    if (e != cudaSuccess) return e;
    part_rank_kernel<<<grid_of(n), 256, 0, st>>>(perm, rank, n);
    return cudaGetLastError();
}

cudaError_t launch_relabel(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *perm,
                           const int32_t *rank, int32_t n, int32_t s, int32_t walk,
                           const PartitionScratch &w, int32_t *row_ptr2, int32_t *col_idx2,
                           int64_t *apair2, cudaStream_t st)
{
    part_counts_kernel<<<grid_of((int64_t)n + 1), 256, 0, st>>>(row_ptr, perm, n, s, walk, w.deg,
                                                                w.cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t bytes = w.temp_bytes;
    e = cub::DeviceScan::ExclusiveSum(w.temp, bytes, w.deg, row_ptr2, n + 1, st);
    if (e != cudaSuccess) return e;
    bytes = w.temp_bytes;
    e = cub::DeviceScan::ExclusiveSum(w.temp, bytes, w.cnt, apair2, n + 1, st);
    if (e != cudaSuccess) return e;
    part_cols_kernel<<<grid_of((int64_t)n * 32), 256, 0, st>>>(row_ptr, col_idx, perm, rank,
                                                               row_ptr2, col_idx2, n);
    return cudaGetLastError();
}

cudaError_t launch_mb_tables(const int64_t *apair2, int32_t n, int32_t b, int32_t M, int64_t W,
                             int32_t Cfix, const PartitionScratch &w, int32_t *mb_C,
                             int64_t *mb_base, int32_t *items, int64_t *mb_p0, cudaStream_t st)
{
    part_sizes_kernel<<<grid_of((int64_t)M + 1), 256, 0, st>>>(apair2, n, b, M, W, Cfix, mb_C,
                                                               w.nch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t bytes = w.temp_bytes;
    e = cub::DeviceScan::ExclusiveSum(w.temp, bytes, w.nch, mb_base, M + 1, st);
    if (e != cudaSuccess) return e;
    part_items_kernel<<<M, 256, 0, st>>>(apair2, mb_base, mb_C, n, b, items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    part_p0_kernel<<<grid_of((int64_t)M + 1), 256, 0, st>>>(apair2, n, b, M, mb_p0);
    return cudaGetLastError();
}

cudaError_t launch_permute_rows(const float *src, float *dst, const int32_t *perm, int64_t rows,
                                int32_t d, bool scatter, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    permute_rows_kernel<<<grid_of(rows * 32), 256, 0, st>>>(src, dst, perm, rows, d, scatter);
    return cudaGetLastError();
}

}  // namespace f2v
