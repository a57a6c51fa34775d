// f2v_downstream.cu -- the downstream evaluations of Sec. IV, in FP64 on the
// device: link prediction (Hadamard features of a pair, an L2-regularised
// logistic regression fitted by Newton's method, accuracy on held-out pairs)
// and clustering (Lloyd's k-means on the rows of Z, scored by modularity).
//
// Logistic regression.  theta = (w, b) minimises
//   sum_i log(1 + exp(-s_i (w . x_i + b))) + |w|^2 / 2,   s_i = 2 y_i - 1,
// x_i = z_u * z_v.  Each Newton step needs g = sum (p_i - y_i) a_i + (w, 0)
// and H = sum p_i (1 - p_i) a_i a_i^T + diag(1, .., 1, 0), a_i = (x_i, 1):
// every block keeps a partial H (D1 x D1, D1 = d + 1 <= 129) in shared
// memory over the pairs it takes, staging 16 pairs' a_i at a time, then adds
// it into the global sums; one block then solves H step = g by Cholesky.
//
// k-means.  A warp per vertex finds the nearest centre (FP64 squared
// distances, the lowest index on a tie); centre sums and counts are added up
// with FP64 atomics; a centre whose cluster is empty is kept.
#include <cuda_runtime.h>

#include <algorithm>

#include "f2v_internal.h"

namespace f2v {

namespace {

constexpr int kLrTile = 16;       // pairs staged per step
constexpr int kLrThreads = 512;

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(sms, 1);
}

__device__ __forceinline__ double sigmoid_d(double t) { return 0.5 * (1.0 + tanh(0.5 * t)); }

// Pair i of the combined list: pos pairs (label 1) first, then neg pairs.
__device__ __forceinline__ void pair_of(const int32_t *pos, int64_t npos, const int32_t *neg,
                                        int64_t i, int32_t &u, int32_t &v, double &y)
{
    if (i < npos) {
        u = pos[2 * i];
        v = pos[2 * i + 1];
        y = 1.0;
    } else {
        u = neg[2 * (i - npos)];
        v = neg[2 * (i - npos) + 1];
        y = 0.0;
    }
}

__global__ void __launch_bounds__(kLrThreads) lr_newton_kernel(
    const float *__restrict__ z, int32_t d, const int32_t *__restrict__ pos, int64_t npos,
    const int32_t *__restrict__ neg, const int64_t *__restrict__ idx, int64_t m,
    const double *__restrict__ theta, double *__restrict__ g_out, double *__restrict__ h_out)
{
    extern __shared__ double sm[];
    const int D1 = d + 1;
    double *H = sm;                              // D1 * D1
    double *A = H + D1 * D1;                     // kLrTile * D1: sqrt(p (1 - p)) a_i
    double *R = A + kLrTile * D1;                // kLrTile * D1: (p - y) a_i
    for (int e = threadIdx.x; e < D1 * D1; e += blockDim.x) H[e] = 0.0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double gacc = 0.0;                           // thread t < D1 keeps g[t]
    for (int64_t t0 = (int64_t)blockIdx.x * kLrTile; t0 < m; t0 += (int64_t)gridDim.x * kLrTile) {
        __syncthreads();
        for (int t = warp; t < kLrTile; t += nw) {
            const int64_t i = t0 + t;
            double s = 0.0, y = 0.0;
            int32_t u = 0, v = 0;
            const bool live = i < m;
            if (live) {
                pair_of(pos, npos, neg, idx[i], u, v, y);
                for (int j = lane; j < d; j += 32)
                    s += (double)z[(int64_t)u * d + j] * (double)z[(int64_t)v * d + j] * theta[j];
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const double p = sigmoid_d(s + theta[d]);
            const double sw = live ? sqrt(p * (1.0 - p)) : 0.0;
            const double r = live ? p - y : 0.0;
            for (int j = lane; j < D1; j += 32) {
                const double a = (j < d && live)
                                     ? (double)z[(int64_t)u * d + j] * (double)z[(int64_t)v * d + j]
                                     : (live ? 1.0 : 0.0);
                A[t * D1 + j] = sw * a;
                R[t * D1 + j] = r * a;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < D1 * D1; e += blockDim.x) {
            const int r = e / D1, c = e - r * D1;
            double acc = 0.0;
#pragma unroll 4
            for (int t = 0; t < kLrTile; ++t) acc += A[t * D1 + r] * A[t * D1 + c];
            H[e] += acc;
        }
        if (threadIdx.x < D1) {
            for (int t = 0; t < kLrTile; ++t) gacc += R[t * D1 + threadIdx.x];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < D1 * D1; e += blockDim.x) atomicAdd(&h_out[e], H[e]);
    if (threadIdx.x < D1) atomicAdd(&g_out[threadIdx.x], gacc);
}

// One block: adds the penalty, solves H step = g (Cholesky), theta -= step,
// and writes max |step| to *step_max.
__global__ void lr_solve_kernel(int32_t d, double *__restrict__ H, double *__restrict__ g,
                                double *__restrict__ theta, double *__restrict__ step_max)
{
    const int D1 = d + 1;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        H[j * D1 + j] += 1.0;
        g[j] += theta[j];
    }
    __syncthreads();
    // in-place Cholesky, lower triangle: H = L L^T
    for (int k = 0; k < D1; ++k) {
        if (threadIdx.x == 0) {
            double s = H[k * D1 + k];
            for (int j = 0; j < k; ++j) s -= H[k * D1 + j] * H[k * D1 + j];
            H[k * D1 + k] = sqrt(s);
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < D1; i += blockDim.x) {
            double s = H[i * D1 + k];
            for (int j = 0; j < k; ++j) s -= H[i * D1 + j] * H[k * D1 + j];
            H[i * D1 + k] = s / H[k * D1 + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // L y = g, then L^T x = y (x overwrites g)
        for (int i = 0; i < D1; ++i) {
            double s = g[i];
            for (int j = 0; j < i; ++j) s -= H[i * D1 + j] * g[j];
            g[i] = s / H[i * D1 + i];
        }
        double mx = 0.0;
        for (int i = D1 - 1; i >= 0; --i) {
            double s = g[i];
            for (int j = i + 1; j < D1; ++j) s -= H[j * D1 + i] * g[j];
            g[i] = s / H[i * D1 + i];
            theta[i] -= g[i];
            mx = fmax(mx, fabs(g[i]));
        }
        *step_max = mx;
    }
}

__global__ void lr_accuracy_kernel(const float *__restrict__ z, int32_t d,
                                   const int32_t *__restrict__ pos, int64_t npos,
                                   const int32_t *__restrict__ neg, const int64_t *__restrict__ idx,
                                   int64_t m, const double *__restrict__ theta,
                                   unsigned long long *__restrict__ correct)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mine = 0;
    for (int64_t i = warp; i < m; i += nwarps) {
        int32_t u, v;
        double y;
        pair_of(pos, npos, neg, idx[i], u, v, y);
        double s = 0.0;
        for (int j = lane; j < d; j += 32)
            s += (double)z[(int64_t)u * d + j] * (double)z[(int64_t)v * d + j] * theta[j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && ((s + theta[d] > 0.0) == (y > 0.5))) ++mine;
    }
    if (lane == 0 && mine) atomicAdd(correct, mine);
}

// ---- k-means ----------------------------------------------------------

__global__ void km_init_kernel(const float *__restrict__ z, int32_t d, const int32_t *__restrict__ init,
                               int32_t k, double *__restrict__ C)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)k * d;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / d, j = t - c * d;
        C[t] = (double)z[(int64_t)init[c] * d + j];
    }
}

__global__ void km_assign_kernel(const float *__restrict__ z, int32_t n, int32_t d,
                                 const double *__restrict__ C, int32_t k,
                                 int32_t *__restrict__ labels, double *__restrict__ sums,
                                 unsigned long long *__restrict__ counts,
                                 unsigned long long *__restrict__ changed)
{
    extern __shared__ double Cs[];               // k * d
    for (int t = threadIdx.x; t < k * d; t += blockDim.x) Cs[t] = C[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long moved = 0;
    for (int64_t u = warp; u < n; u += nwarps) {
        double best = 0.0;
        int bc = 0;
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int j = lane; j < d; j += 32) {
                const double df = (double)z[u * d + j] - Cs[c * d + j];
                s += df * df;
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (c == 0 || s < best) {          // strict: the lowest index on a tie
                best = s;
                bc = c;
            }
        }
        if (lane == 0) {
            if (labels[u] != bc) ++moved;
            labels[u] = bc;
            atomicAdd(&counts[bc], 1ull);
        }
        for (int j = lane; j < d; j += 32) atomicAdd(&sums[(int64_t)bc * d + j], (double)z[u * d + j]);
    }
    if (lane == 0 && moved) atomicAdd(changed, moved);
}

__global__ void km_update_kernel(int32_t k, int32_t d, const double *__restrict__ sums,
                                 const unsigned long long *__restrict__ counts,
                                 double *__restrict__ C)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)k * d;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / d;
        if (counts[c] > 0) C[t] = sums[t] / (double)counts[c];   // empty: the centre stays
    }
}

// e[c]: CSR entries with both ends in cluster c; D[c]: summed degree of c.
__global__ void modularity_counts_kernel(const int32_t *__restrict__ row_ptr,
                                         const int32_t *__restrict__ col_idx, int32_t n,
                                         const int32_t *__restrict__ labels,
                                         unsigned long long *__restrict__ e,
                                         unsigned long long *__restrict__ D)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int32_t lo = row_ptr[u], hi = row_ptr[u + 1], lu = labels[u];
        unsigned long long inside = 0;
        for (int32_t q = lo + lane; q < hi; q += 32) inside += (labels[col_idx[q]] == lu);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) inside += __shfl_xor_sync(0xffffffffu, inside, o);
        if (lane == 0) {
            if (inside) atomicAdd(&e[lu], inside);
            if (hi > lo) atomicAdd(&D[lu], (unsigned long long)(hi - lo));
        }
    }
}

__global__ void modularity_kernel(int32_t k, int64_t nnz, const unsigned long long *__restrict__ e,
                                  const unsigned long long *__restrict__ D, double *__restrict__ q)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        if (nnz > 0)
            for (int c = 0; c < k; ++c) {
                const double f = (double)D[c] / (double)nnz;
                s += (double)e[c] / (double)nnz - f * f;
            }
        *q = s;
    }
}

}  // namespace

size_t lr_smem_bytes(int32_t d)
{
    const size_t D1 = (size_t)d + 1;
    return sizeof(double) * (D1 * D1 + 2 * kLrTile * D1);
}

cudaError_t launch_lr_newton(const float *z, int32_t d, const int32_t *pos, int64_t npos,
                             const int32_t *neg, const int64_t *idx, int64_t m,
                             const double *theta, double *g, double *H, cudaStream_t st)
{
    const size_t smem = lr_smem_bytes(d);
    cudaError_t e = cudaFuncSetAttribute(lr_newton_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (m + kLrTile - 1) / kLrTile;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sm_count()));
    lr_newton_kernel<<<blocks, kLrThreads, smem, st>>>(z, d, pos, npos, neg, idx, m, theta, g, H);
    return cudaGetLastError();
}

cudaError_t launch_lr_solve(int32_t d, double *H, double *g, double *theta, double *step_max,
                            cudaStream_t st)
{
    lr_solve_kernel<<<1, 256, 0, st>>>(d, H, g, theta, step_max);
    return cudaGetLastError();
}

cudaError_t launch_lr_accuracy(const float *z, int32_t d, const int32_t *pos, int64_t npos,
                               const int32_t *neg, const int64_t *idx, int64_t m,
                               const double *theta, unsigned long long *correct, cudaStream_t st)
{
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((m * 32 + 255) / 256, (int64_t)sm_count() * 16));
    lr_accuracy_kernel<<<blocks, 256, 0, st>>>(z, d, pos, npos, neg, idx, m, theta, correct);
    return cudaGetLastError();
}

cudaError_t launch_km_init(const float *z, int32_t d, const int32_t *init, int32_t k, double *C,
                           cudaStream_t st)
{
    km_init_kernel<<<std::max(1, (k * d + 255) / 256), 256, 0, st>>>(z, d, init, k, C);
    return cudaGetLastError();
}

cudaError_t launch_km_assign(const float *z, int32_t n, int32_t d, const double *C, int32_t k,
                             int32_t *labels, double *sums, unsigned long long *counts,
                             unsigned long long *changed, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)k * d;
    cudaError_t e = cudaFuncSetAttribute(km_assign_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)n * 32 + 255) / 256, (int64_t)sm_count() * 4));
    km_assign_kernel<<<blocks, 256, smem, st>>>(z, n, d, C, k, labels, sums, counts, changed);
    return cudaGetLastError();
}

cudaError_t launch_km_update(int32_t k, int32_t d, const double *sums,
                             const unsigned long long *counts, double *C, cudaStream_t st)
{
    km_update_kernel<<<std::max(1, (k * d + 255) / 256), 256, 0, st>>>(k, d, sums, counts, C);
    return cudaGetLastError();
}

cudaError_t launch_modularity(const int32_t *row_ptr, const int32_t *col_idx, int32_t n,
                              int64_t nnz, const int32_t *labels, int32_t k,
                              unsigned long long *e, unsigned long long *D, double *q,
                              cudaStream_t st)
{
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)n * 32 + 255) / 256, (int64_t)sm_count() * 16));
    modularity_counts_kernel<<<blocks, 256, 0, st>>>(row_ptr, col_idx, n, labels, e, D);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    modularity_kernel<<<1, 32, 0, st>>>(k, nnz, e, D, q);
    return cudaGetLastError();
}

}  // namespace f2v
