// f2v_eval.cu -- held-out-edge link-prediction AUC and the loss of Eq. 2 on
// the device, both in FP64.
//
// Scores are FP64: z_u . z_v for the sigmoid model, -||z_u - z_v||^2 for the
// t model (both monotone in the model's similarity delta, Eq. 3 / Eq. 7).
// AUC is the Mann-Whitney statistic: negatives are radix-sorted, each positive
// counts the negatives below it (2 points) and equal to it (1 point) by
// binary search, and the integer counts are summed exactly in 64 bits.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cub/device/device_radix_sort.cuh>

#include <stdint.h>

#include <string>

#include "f2v_device.cuh"

namespace f2v {

namespace {

__global__ void score_kernel(const float *z, int d, int model, const int32_t *pairs, int64_t np,
                             double *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < np; i += nwarps) {
        const float *a = z + (int64_t)pairs[2 * i] * d;
        const float *b = z + (int64_t)pairs[2 * i + 1] * d;
        double acc = 0.0;
        for (int j = lane; j < d; j += 32) {
            if (model == 1) {
                acc += (double)a[j] * (double)b[j];
            } else {
                const double df = (double)a[j] - (double)b[j];
                acc += df * df;
            }
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
        if (lane == 0) out[i] = (model == 1) ? acc : -acc;
    }
}

__global__ void count_kernel(const double *pos, int64_t npos, const double *neg_sorted,
                             int64_t nneg, unsigned long long *total)
{
    unsigned long long local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npos;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double p = pos[i];
        int64_t lo = 0, hi = nneg;                   // first index with neg >= p
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (neg_sorted[m] < p) lo = m + 1; else hi = m;
        }
        int64_t lo2 = lo, hi2 = nneg;                // first index with neg > p
        while (lo2 < hi2) {
            const int64_t m = (lo2 + hi2) >> 1;
            if (neg_sorted[m] <= p) lo2 = m + 1; else hi2 = m;
        }
        local += 2ull * (unsigned long long)lo + (unsigned long long)(lo2 - lo);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) local += __shfl_xor_sync(0xffffffffu, local, m);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

// ---- loss of Eq. 2 --------------------------------------------------------

constexpr int kLossBlocks = 1024;    // fixed grid: the summation order does not
constexpr int kLossThreads = 256;    // depend on the device

// -log delta(z_u, z_x) of a neighbour (attractive) or -log(1 - delta) of a
// negative sample, from r = z_u . z_x (sigmoid model, delta of Eq. 3) or
// r = |z_u - z_x|^2 (t model, delta of Eq. 7, t^2 floored at 1e-8 in the
// repulsive term).  log(1 + e^y) is evaluated as max(y, 0) + log1p(e^-|y|),
// which is the same value without overflow.
__device__ __forceinline__ double pair_loss(int model, bool attractive, double r)
{
    if (model == 1) {
        const double y = attractive ? -r : r;   // -log sigma(r), -log(1 - sigma(r))
        return fmax(y, 0.0) + log1p(exp(-fabs(y)));
    }
    if (attractive) return log1p(r);            // -log 1/(1 + t^2)
    const double t2 = fmax(r, 1e-8);
    return log1p(1.0 / t2);                     // -log t^2/(1 + t^2)
}

// Pairs of the loss: CSR entry p < nnz is (u, col_idx[p]) with u the row
// holding p; p = nnz + u * s + k is negative sample k of u.  Each warp takes
// 32 consecutive pairs, decoded one per lane, and evaluates them in turn with
// its lanes striding over the d elements; lane j keeps pair j's term.  Each
// block writes the FP64 sum of its terms, reduced in a fixed order.
__global__ void __launch_bounds__(kLossThreads)
    loss_kernel(const float *z, int d, int model, const int32_t *row_ptr, const int32_t *col_idx,
                int n, int64_t nnz, int s, uint32_t epoch, uint32_t key0, uint32_t key1,
                double *partial)
{
    __shared__ double red[kLossThreads / 32];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = nnz + (int64_t)n * s;
    double acc = 0.0;
    for (int64_t base = warp * 32; base < total; base += nwarps * 32) {
        const int64_t p = base + lane;
        int u = -1, x = -1;
        if (p < nnz) {
            int lo = 0, hi = n - 1;                  // the row holding entry p
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int64_t)row_ptr[mid] <= p) lo = mid; else hi = mid - 1;
            }
            u = lo;
            x = col_idx[p];
        } else if (p < total) {
            const int64_t q = p - nnz;
            u = (int)(q / s);
            const uint32_t k = (uint32_t)(q - (int64_t)u * s);
            x = (int)(philox_x0((uint32_t)u, epoch, k, 0u, key0, key1) % (uint32_t)n);
            if (x == u) x = -1;                      // a sample equal to u adds nothing
        }
        const bool attr = p < nnz;
        for (int j = 0; j < 32; ++j) {
            const int uj = __shfl_sync(0xffffffffu, u, j);
            const int xj = __shfl_sync(0xffffffffu, x, j);
            if (uj < 0 || xj < 0) continue;          // warp-uniform
            const float *a = z + (int64_t)uj * d;
            const float *b = z + (int64_t)xj * d;
            double r = 0.0;
            for (int e = lane; e < d; e += 32) {
                const double ae = (double)a[e], be = (double)b[e];
                if (model == 1) {
                    r = fma(ae, be, r);
                } else {
                    const double df = ae - be;
                    r = fma(df, df, r);
                }
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) r += __shfl_xor_sync(0xffffffffu, r, m);
            if (lane == j) acc += pair_loss(model, attr, r);
        }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kLossThreads / 32; ++i) t += red[i];
        partial[blockIdx.x] = t;
    }
}

// out = sum of partial[0 .. count), in a fixed order (one block).
__global__ void sum_kernel(const double *partial, int count, double *out)
{
    __shared__ double red[kLossThreads];
    double t = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) t += partial[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

cudaError_t eval_loss_device(const float *z, int d, int model, const int32_t *row_ptr,
                             const int32_t *col_idx, int n, int64_t nnz, int s, uint32_t epoch,
                             uint32_t key0, uint32_t key1, cudaStream_t st, double *loss,
                             std::string *err)
{
    double *partial = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&partial, sizeof(double) * (kLossBlocks + 1), st);
    if (e != cudaSuccess) {
        *err = std::string("alloc: ") + cudaGetErrorString(e);
        return e;
    }
    loss_kernel<<<kLossBlocks, kLossThreads, 0, st>>>(z, d, model, row_ptr, col_idx, n, nnz, s,
                                                      epoch, key0, key1, partial);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        sum_kernel<<<1, kLossThreads, 0, st>>>(partial, kLossBlocks, partial + kLossBlocks);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(loss, partial + kLossBlocks, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) *err = std::string("loss kernels: ") + cudaGetErrorString(e);
    cudaFreeAsync(partial, st);
    cudaStreamSynchronize(st);
    return e;
}

cudaError_t eval_auc_device(const float *zf, const __nv_bfloat16 *, int d, int model,
                            const int32_t *pos, int64_t npos, const int32_t *neg, int64_t nneg,
                            cudaStream_t st, double *auc, std::string *err)
{
    int32_t *dpairs = nullptr;
    double *scores = nullptr, *sorted = nullptr;
    unsigned long long *total = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaSuccess;
    unsigned long long h_total = 0;
    const int64_t np = npos + nneg;
    auto check = [&](cudaError_t x, const char *what) {
        if (x != cudaSuccess && e == cudaSuccess) {
            e = x;
            *err = std::string(what) + ": " + cudaGetErrorString(x);
        }
        return e == cudaSuccess;
    };
    if (!check(cudaMallocAsync((void **)&dpairs, sizeof(int32_t) * 2 * np, st), "alloc pairs")) goto done;
    if (!check(cudaMallocAsync((void **)&scores, sizeof(double) * np, st), "alloc scores")) goto done;
    if (!check(cudaMallocAsync((void **)&sorted, sizeof(double) * nneg, st), "alloc sorted")) goto done;
    if (!check(cudaMallocAsync((void **)&total, sizeof(unsigned long long), st), "alloc total")) goto done;
    if (!check(cudaMemcpyAsync(dpairs, pos, sizeof(int32_t) * 2 * npos, cudaMemcpyHostToDevice, st), "copy pos")) goto done;
    if (!check(cudaMemcpyAsync(dpairs + 2 * npos, neg, sizeof(int32_t) * 2 * nneg, cudaMemcpyHostToDevice, st), "copy neg")) goto done;
    if (!check(cudaMemsetAsync(total, 0, sizeof(unsigned long long), st), "memset")) goto done;
    {
        const int blocks = (int)std::min<int64_t>((np * 32 + 255) / 256, 152 * 32);
        score_kernel<<<blocks, 256, 0, st>>>(zf, d, model, dpairs, np, scores);
        if (!check(cudaGetLastError(), "score kernel")) goto done;
    }
    if (!check(cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, scores + npos, sorted,
                                              (int)nneg, 0, 64, st), "sort size")) goto done;
    if (!check(cudaMallocAsync(&tmp, tmp_bytes, st), "alloc sort")) goto done;
    if (!check(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, scores + npos, sorted, (int)nneg,
                                              0, 64, st), "sort")) goto done;
    {
        const int blocks = (int)std::min<int64_t>((npos + 255) / 256, 152 * 16);
        count_kernel<<<blocks, 256, 0, st>>>(scores, npos, sorted, nneg, total);
        if (!check(cudaGetLastError(), "count kernel")) goto done;
    }
    if (!check(cudaMemcpyAsync(&h_total, total, sizeof h_total, cudaMemcpyDeviceToHost, st), "copy total")) goto done;
    if (!check(cudaStreamSynchronize(st), "sync")) goto done;
    *auc = (double)h_total / (2.0 * (double)npos * (double)nneg);
done:
    if (tmp) cudaFreeAsync(tmp, st);
    if (total) cudaFreeAsync(total, st);
    if (sorted) cudaFreeAsync(sorted, st);
    if (scores) cudaFreeAsync(scores, st);
    if (dpairs) cudaFreeAsync(dpairs, st);
    cudaStreamSynchronize(st);
    return e;
}

}  // namespace f2v
