// f2v_device.cuh -- device helpers of libf2v: the Philox4x32-10 generator,
// row loads/stores for FP32 and BF16 storage, and small group reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace f2v {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies by
// 0xD2511F53 and 0xCD9E8D57, with the key advanced by the Weyl increments
// 0x9E3779B9 and 0xBB67AE85 between rounds.  Returns word 0 of the output.
__device__ __forceinline__ uint32_t philox_x0(uint32_t c0, uint32_t c1, uint32_t c2,
                                              uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
        const uint32_t lo_a = 0xD2511F53u * c0;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo_b = 0xCD9E8D57u * c2;
        c0 = hi_b ^ c1 ^ k0;
        c1 = lo_b;
        c2 = hi_a ^ c3 ^ k1;
        c3 = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// Z0[i][j] = (Philox(ctr=(i, j, 0xFFFF, 0)).x0 >> 8) * 2^-24 - 0.5: a multiple
// of 2^-24 in [-0.5, 0.5), exact in FP32 (the initial embedding, uniform as
// the paper's random start).
// Negative sample k of vertex u in epoch `epoch`: its own draw
// Philox(ctr = (u, epoch, k, 0)).x0 mod n, or, with kb >= 0 (one set S_b
// per minibatch, Alg. 1's sampling step read literally), the draw of minibatch kb,
// Philox(ctr = (kb, epoch, k, 2)).x0 mod n.
__device__ __forceinline__ uint32_t negative_sample(int64_t u, int64_t kb, uint32_t epoch,
                                                    uint32_t k, int32_t n, uint32_t key0,
                                                    uint32_t key1)
{
    const uint32_t x = (kb >= 0) ? philox_x0((uint32_t)kb, epoch, k, 2u, key0, key1)
                                 : philox_x0((uint32_t)u, epoch, k, 0u, key0, key1);
    return x % (uint32_t)n;
}

__device__ __forceinline__ float z0_value(uint32_t i, uint32_t j, uint32_t k0, uint32_t k1)
{
    const uint32_t x = philox_x0(i, j, 0xFFFFu, 0u, k0, k1);
    return (float)(x >> 8) * 5.9604644775390625e-8f - 0.5f;   // 2^-24
}

// BF16 -> FP32 is exact: a BF16 value is the upper 16 bits of the FP32 value
// with the same bits.  Widening by shift and mask keeps the conversion on the
// integer ALUs, which issue at the FMA rate (a conversion instruction per
// element would run at a fraction of it and, with two conversions per element
// per tile, bound the BF16 kernels).
__device__ __forceinline__ void bf16x2_to_float(unsigned int w, float *x)
{
    x[0] = __uint_as_float(w << 16);
    x[1] = __uint_as_float(w & 0xFFFF0000u);
}

// Row element loads: VEC consecutive elements starting at p, widened to FP32.
template <int VEC>
__device__ __forceinline__ void load_vec(const float *p, float *x)
{
    if constexpr (VEC == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else if constexpr (VEC == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        x[0] = t.x; x[1] = t.y;
    } else {
        x[0] = __ldg(p);
    }
}

template <int VEC>
__device__ __forceinline__ void load_vec(const __nv_bfloat16 *p, float *x)
{
    if constexpr (VEC == 4) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        bf16x2_to_float(t.x, x);
        bf16x2_to_float(t.y, x + 2);
    } else if constexpr (VEC == 2) {
        const unsigned int t = __ldg(reinterpret_cast<const unsigned int *>(p));
        bf16x2_to_float(t, x);
    } else {
        x[0] = __uint_as_float((unsigned int)__ldg(reinterpret_cast<const unsigned short *>(p)) << 16);
    }
}

// Loads through L2 only (for data written by other blocks of the same launch).
template <int VEC>
__device__ __forceinline__ void load_vec_cg(const float *p, float *x)
{
    if constexpr (VEC == 4) {
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else if constexpr (VEC == 2) {
        const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
        x[0] = t.x; x[1] = t.y;
    } else {
        x[0] = __ldcg(p);
    }
}

template <int VEC>
__device__ __forceinline__ void load_vec_cg(const __nv_bfloat16 *p, float *x)
{
    if constexpr (VEC == 4) {
        const uint2 t = __ldcg(reinterpret_cast<const uint2 *>(p));
        bf16x2_to_float(t.x, x);
        bf16x2_to_float(t.y, x + 2);
    } else if constexpr (VEC == 2) {
        const unsigned int t = __ldcg(reinterpret_cast<const unsigned int *>(p));
        bf16x2_to_float(t, x);
    } else {
        const unsigned short t = __ldcg(reinterpret_cast<const unsigned short *>(p));
        x[0] = __uint_as_float((unsigned int)t << 16);
    }
}

template <int VEC>
__device__ __forceinline__ void store_vec(float *p, const float *x)
{
    if constexpr (VEC == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else if constexpr (VEC == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    } else {
        p[0] = x[0];
    }
}

template <int VEC>
__device__ __forceinline__ void store_vec_cg(float *p, const float *x)
{
    if constexpr (VEC == 4) {
        __stcg(reinterpret_cast<float4 *>(p), make_float4(x[0], x[1], x[2], x[3]));
    } else if constexpr (VEC == 2) {
        __stcg(reinterpret_cast<float2 *>(p), make_float2(x[0], x[1]));
    } else {
        __stcg(p, x[0]);
    }
}

// BF16 stores round to nearest even.
template <int VEC>
__device__ __forceinline__ void store_vec(__nv_bfloat16 *p, const float *x)
{
    if constexpr (VEC == 4) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(x[0], x[1]);
        const __nv_bfloat162 b = __floats2bfloat162_rn(x[2], x[3]);
        uint2 t;
        t.x = *reinterpret_cast<const unsigned int *>(&a);
        t.y = *reinterpret_cast<const unsigned int *>(&b);
        *reinterpret_cast<uint2 *>(p) = t;
    } else if constexpr (VEC == 2) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(x[0], x[1]);
        *reinterpret_cast<__nv_bfloat162 *>(p) = a;
    } else {
        p[0] = __float2bfloat16_rn(x[0]);
    }
}

// Shared-memory vector loads, widened to FP32.
template <int VEC>
__device__ __forceinline__ void load_vec_smem(const float *p, float *x)
{
    if constexpr (VEC == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else if constexpr (VEC == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        x[0] = t.x; x[1] = t.y;
    } else {
        x[0] = p[0];
    }
}

template <int VEC>
__device__ __forceinline__ void load_vec_smem(const __nv_bfloat16 *p, float *x)
{
    if constexpr (VEC == 4) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        bf16x2_to_float(t.x, x);
        bf16x2_to_float(t.y, x + 2);
    } else if constexpr (VEC == 2) {
        const unsigned int t = *reinterpret_cast<const unsigned int *>(p);
        bf16x2_to_float(t, x);
    } else {
        x[0] = __uint_as_float((unsigned int)*reinterpret_cast<const unsigned short *>(p) << 16);
    }
}

// Packed FP32 pairs (sm_100 family): one instruction for two elements, each
// rounded as its scalar counterpart (fmaf, subtraction) would be.
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rd, {%0, %1};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rd;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

__device__ __forceinline__ void sub2(float &d0, float &d1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// x - o for the two BF16 elements packed in w (low half first), each widened
// exactly and the difference rounded once: the mixed-precision subtraction
// of the sm_100 family, one instruction per element with no separate widening.
__device__ __forceinline__ void sub_bf16x2_f32(float &d0, float &d1, unsigned int w, float o0,
                                               float o1)
{
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "sub.rn.f32.bf16 %0, lo, %3;\n\tsub.rn.f32.bf16 %1, hi, %4;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "r"(w), "f"(o0), "f"(o1));
}

// Waits between warps of one launch are bounded: about a second at 2 GHz.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait until *p >= target (acquire); false on time-out.
__device__ __forceinline__ bool wait_at_least(const int32_t *p, int target)
{
    if (ld_acquire(p) >= target) return true;
    const long long t0 = clock64();
    while (ld_acquire(p) < target) {
        if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(64);
    }
    return true;
}

// Bounded wait until *p == target (acquire); false on time-out.
__device__ __forceinline__ bool wait_equal(const int32_t *p, int target)
{
    if (ld_acquire(p) == target) return true;
    const long long t0 = clock64();
    while (ld_acquire(p) != target) {
        if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(32);
    }
    return true;
}

}  // namespace f2v

