// f2v_eval.cu -- held-out-edge link-prediction AUC on the device.
//
// Scores are FP64: z_u . z_v for the sigmoid model, -||z_u - z_v||^2 for the
// t model (both monotone in the model's similarity delta, Eq. 3 / Eq. 7).
// AUC is the Mann-Whitney statistic: negatives are radix-sorted, each positive
// counts the negatives below it (2 points) and equal to it (1 point) by
// binary search, and the integer counts are summed exactly in 64 bits.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cub/device/device_radix_sort.cuh>

#include <string>

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

}  // namespace

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
