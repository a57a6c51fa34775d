// f2v_expand.cu -- the per-epoch partner list of the staged force kernel
// (and of both kernels in the rForce2Vec form).
//
// Pair apair[u] + j of vertex u is its j-th neighbour for j < deg(u) and its
// negative sample k = j - deg(u) otherwise (Alg. 2's two loops, in order).
// Writing every pair's partner once per epoch lets the force kernel fetch a
// tile's partners with one coalesced load, instead of a dependent chain
// (row pointers, then column indices) and a Philox evaluation per sample.
// Samples follow the same counter layout as everywhere else:
// w = Philox4x32-10(key, ctr = (u, epoch, k, 0)).x0 mod n, or with shared
// samples (one set S_b per minibatch k = u / b) ctr = (k, epoch, j, 2).
// rForce2Vec (Algorithm 3) replaces the neighbours of u by the walk-length
// steps of a random walk from u (none if u has no neighbours); step i draws
// ctr = (u, epoch, i, 1), moves to that neighbour of the current vertex, and
// exerts no force where it lands on u; a walk stops at a vertex without
// out-neighbours.
#include <cuda_runtime.h>

#include <algorithm>

#include "f2v_device.cuh"
#include "f2v_internal.h"

namespace f2v {

namespace {

__global__ void expand_partners_kernel(const int32_t *__restrict__ row_ptr,
                                       const int32_t *__restrict__ col_idx,
                                       const int64_t *__restrict__ apair, int32_t n, int32_t s,
                                       int32_t shared_b, const int32_t *__restrict__ perm,
                                       const int32_t *__restrict__ rank, uint32_t epoch,
                                       uint32_t key0, uint32_t key1,
                                       int32_t *__restrict__ partner)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t base = apair[u];
        const int32_t r0 = row_ptr[u];
        const int32_t deg = row_ptr[u + 1] - r0;
        // eight loads in flight per lane before their stores (a hub's row is
        // one warp's: tens of thousands of entries)
        for (int32_t j0 = 0; j0 < deg; j0 += 32 * 8) {
            int32_t v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int32_t j = j0 + 32 * t + lane;
                v[t] = (j < deg) ? col_idx[r0 + j] : 0;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int32_t j = j0 + 32 * t + lane;
                if (j < deg) partner[base + j] = v[t];
            }
        }
        const int64_t uo = perm ? perm[u] : u;                // the original id
        const int64_t kb = shared_b > 0 ? u / shared_b : -1;   // u's minibatch
        for (int32_t k = lane; k < s; k += 32) {
            const uint32_t w = negative_sample(uo, kb, epoch, (uint32_t)k, n, key0, key1);
            partner[base + deg + k] =
                ((int64_t)w == uo) ? kPartnerNone : -2 - (rank ? rank[w] : (int32_t)w);
        }
        if (deg + s == 0 && lane == 0) partner[base] = kPartnerNone;   // the empty pair
    }
}

// Only the sample pairs of a list that already holds every vertex's
// neighbours (a list of another epoch of the same graph: the neighbour codes
// do not change between epochs, the samples do).  One thread per (vertex,
// sample): n * s codes instead of the whole list.
__global__ void refresh_samples_kernel(const int32_t *__restrict__ row_ptr,
                                       const int64_t *__restrict__ apair, int32_t n, int32_t s,
                                       int32_t shared_b, uint32_t epoch, uint32_t key0,
                                       uint32_t key1, int32_t *__restrict__ partner)
{
    const int64_t total = (int64_t)n * s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t u = t / s;
        const int32_t k = (int32_t)(t - u * s);
        const int32_t deg = row_ptr[u + 1] - row_ptr[u];
        const int64_t kb = shared_b > 0 ? u / shared_b : -1;   // u's minibatch
        const uint32_t w = negative_sample(u, kb, epoch, (uint32_t)k, n, key0, key1);
        partner[apair[u] + deg + k] = ((int64_t)w == u) ? kPartnerNone : -2 - (int32_t)w;
    }
}

// One thread per vertex u: the walk's steps are a chain of dependent reads
// (row pointers of w, then its column), so vertices, not steps, are spread
// over the lanes.
__global__ void expand_walks_kernel(const int32_t *__restrict__ row_ptr,
                                    const int32_t *__restrict__ col_idx,
                                    const int64_t *__restrict__ apair, int32_t n, int32_t s,
                                    int32_t walk, int32_t shared_b,
                                    const int32_t *__restrict__ perm,
                                    const int32_t *__restrict__ rank, uint32_t epoch,
                                    uint32_t key0, uint32_t key1, int32_t *__restrict__ partner)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += stride) {
        int64_t p = apair[u];
        const int64_t uo = perm ? perm[u] : u;                // the original id
        const bool has_walk = row_ptr[u + 1] > row_ptr[u];
        if (has_walk) {
            int32_t w = (int32_t)u;
            bool stopped = false;
            for (int32_t i = 0; i < walk; ++i) {
                int32_t code = kPartnerNone;
                if (!stopped) {
                    const int32_t lo = row_ptr[w];
                    const int32_t deg = row_ptr[w + 1] - lo;
                    if (deg == 0) {
                        stopped = true;
                    } else {
                        const uint32_t x = philox_x0((uint32_t)uo, epoch, (uint32_t)i, 1u, key0,
                                                     key1);
                        w = col_idx[lo + (int32_t)(x % (uint32_t)deg)];
                        code = ((int64_t)w == u) ? kPartnerNone : w;
                    }
                }
                partner[p++] = code;
            }
        }
        const int64_t kb = shared_b > 0 ? u / shared_b : -1;   // u's minibatch
        for (int32_t k = 0; k < s; ++k) {
            const uint32_t w = negative_sample(uo, kb, epoch, (uint32_t)k, n, key0, key1);
            partner[p++] = ((int64_t)w == uo) ? kPartnerNone : -2 - (rank ? rank[w] : (int32_t)w);
        }
        if (!has_walk && s == 0) partner[p] = kPartnerNone;   // the empty pair
    }
}

__global__ void extract_walks_kernel(const int64_t *__restrict__ apair,
                                     const int32_t *__restrict__ row_ptr, int32_t n, int32_t walk,
                                     const int32_t *__restrict__ partner, int32_t *__restrict__ out)
{
    const int64_t total = (int64_t)n * walk;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t u = t / walk, i = t - u * walk;
        out[t] = (row_ptr[u + 1] > row_ptr[u]) ? partner[apair[u] + i] : kPartnerNone;
    }
}

int grid_for(int64_t threads)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<int64_t>(
        1, std::min<int64_t>((threads + 255) / 256, (int64_t)std::max(sms, 1) * 16));
}

}  // namespace

cudaError_t launch_expand_walks(const int32_t *row_ptr, const int32_t *col_idx,
                                const int64_t *apair, int32_t n, int32_t s, int32_t walk,
                                int32_t shared_b, const int32_t *perm, const int32_t *rank,
                                uint32_t epoch, uint32_t key0, uint32_t key1, int32_t *partner,
                                cudaStream_t st)
{
    expand_walks_kernel<<<grid_for(n), 256, 0, st>>>(row_ptr, col_idx, apair, n, s, walk,
                                                     shared_b, perm, rank, epoch, key0, key1,
                                                     partner);
    return cudaGetLastError();
}

cudaError_t launch_extract_walks(const int64_t *apair, const int32_t *row_ptr, int32_t n,
                                 int32_t walk, const int32_t *partner, int32_t *out,
                                 cudaStream_t st)
{
    extract_walks_kernel<<<grid_for((int64_t)n * walk), 256, 0, st>>>(apair, row_ptr, n, walk,
                                                                      partner, out);
    return cudaGetLastError();
}

cudaError_t launch_refresh_samples(const int32_t *row_ptr, const int64_t *apair, int32_t n,
                                   int32_t s, int32_t shared_b, uint32_t epoch, uint32_t key0,
                                   uint32_t key1, int32_t *partner, cudaStream_t st)
{
    if (s == 0) return cudaSuccess;
    refresh_samples_kernel<<<grid_for((int64_t)n * s), 256, 0, st>>>(row_ptr, apair, n, s,
                                                                     shared_b, epoch, key0, key1,
                                                                     partner);
    return cudaGetLastError();
}

cudaError_t launch_expand_partners(const int32_t *row_ptr, const int32_t *col_idx,
                                   const int64_t *apair, int32_t n, int32_t s, int32_t shared_b,
                                   const int32_t *perm, const int32_t *rank, uint32_t epoch,
                                   uint32_t key0, uint32_t key1, int32_t *partner,
                                   cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t warps_needed = n;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((warps_needed + 7) / 8, (int64_t)std::max(sms, 1) * 16));
    expand_partners_kernel<<<blocks, 256, 0, st>>>(row_ptr, col_idx, apair, n, s, shared_b, perm,
                                                   rank, epoch, key0, key1, partner);
    return cudaGetLastError();
}

}  // namespace f2v
