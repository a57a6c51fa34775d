// f2v_bulk.cuh -- the force+update kernel for row sizes d = 32 * EPL
// (EPL = 2, 4, 8), with partner rows staged in shared memory by TMA bulk
// copies instead of register gathers.
//
// One warp walks one contiguous chunk of the minibatch's pair sequence (the
// same pair order as the register kernel: neighbours in CSR order, then the
// s negative samples).  Per tile of at most 32 pairs spanning at most 8
// vertices:
//   decode  lane t finds pair t's vertex and partner (col_idx or Philox);
//   stage   lane t issues one cp.async.bulk copy of its partner row into the
//           warp's shared buffer, lanes j < 8 copy the tile's own rows, all
//           completing on one mbarrier; the next tile is decoded while the
//           copies are in flight;
//   reduce  each lane forms the partial dot product / squared distance of
//           all 32 rows over its EPL elements, and a transpose-reduction
//           (31 shuffles) leaves lane r with row r's full sum;
//   force   lane r turns its sum into the scalar of Eq. 5/6 or Eq. 8/9;
//   update  rows are accumulated per vertex in registers; a vertex that
//           ends is written (z_u - eta g, Eq. 10) or, if it began in an
//           earlier chunk or runs into a later one, passed up the ordered
//           combine tree of f2v_internal.h with chunks as level-0 units.
// Waits on the mbarrier are bounded: after about a second the kernel records
// an error code, waits (bounded again) for its copies, and stops.
#pragma once

#include <climits>

#include "f2v_device.cuh"
#include "f2v_force.cuh"
#include "f2v_internal.h"

namespace f2v {

constexpr int kOwnSlots = 8;            // distinct vertices per tile at most

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global -> shared bulk copy (TMA), completion counted on `bar` in bytes.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait (about a second at 2 GHz); false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) return false;
    }
    return true;
}

// Per-warp shared-memory layout.
template <int D, typename Ts>
struct BulkLayout {
    static constexpr int ROWB = D * (int)sizeof(Ts);      // partner row bytes
    static constexpr int OWNB = D * 4;                    // own row bytes (FP32)
    static constexpr int ROWS_OFF = 0;
    static constexpr int OWN_OFF = ROWS_OFF + 32 * ROWB;
    static constexpr int COEF_OFF = OWN_OFF + kOwnSlots * OWNB;    // float[32]
    static constexpr int VERT_OFF = COEF_OFF + 32 * 4;             // int[32]: vertex - u_tile
    static constexpr int VEND_OFF = VERT_OFF + 32 * 4;             // int[32]: vertex end
    static constexpr int KIND_OFF = VEND_OFF + 32 * 4;             // int[32]
    static constexpr int BAR_OFF = KIND_OFF + 32 * 4;              // uint64
    static constexpr int BYTES = ((BAR_OFF + 8 + 127) / 128) * 128;
};

// Lane-parallel decode of the tile starting at pair q (local), within the
// chunk ending at q_end, whose first pair lies in vertex u.
struct Tile {
    int q, n, u;          // first pair, pairs in the tile, vertex of the first pair
    int nverts;           // distinct vertices in the tile (<= kOwnSlots)
    int u_next;           // vertex holding pair q + n
    int first_lo;         // start of vertex u (local pair index)
    // per lane (pair q + lane)
    int pu, nb, kind, p_hi;
};

template <typename Ts>
__device__ __forceinline__ Tile decode_tile(const ForceArgs<Ts> &a, int q, int q_end, int u,
                                            int lane)
{
    Tile t;
    t.q = q;
    t.u = u;
    const int uu = u + lane;
    int A_hi = INT_MAX, rp_lo = 0, rp_hi = 0;
    if (uu < a.n) {
        const int64_t ah = __ldg(&a.apair[uu + 1]) - a.P0;
        A_hi = ah > INT_MAX ? INT_MAX : (int)ah;
        rp_lo = __ldg(&a.row_ptr[uu]);
        rp_hi = __ldg(&a.row_ptr[uu + 1]);
    }
    const int A_up = __shfl_up_sync(0xffffffffu, A_hi, 1);
    const int A_lo = (lane == 0) ? (int)(__ldg(&a.apair[u]) - a.P0) : A_up;
    t.first_lo = __shfl_sync(0xffffffffu, A_lo, 0);
    // at most 32 pairs, at most kOwnSlots vertices, not past the chunk
    const int end8 = __shfl_sync(0xffffffffu, A_hi, kOwnSlots - 1);
    t.n = min(32, min(q_end - q, end8 - q));
    const int pos = A_hi - q;                         // >= 1
    const unsigned bit = (pos < 32) ? (1u << pos) : 0u;
    const unsigned ends = __reduce_or_sync(0xffffffffu, bit);
    const int off = __popc(ends & ((2u << lane) - 1u));
    t.pu = u + off;
    const int pA_lo = __shfl_sync(0xffffffffu, A_lo, off);
    t.p_hi = __shfl_sync(0xffffffffu, A_hi, off);
    const int prp_lo = __shfl_sync(0xffffffffu, rp_lo, off);
    const int prp_hi = __shfl_sync(0xffffffffu, rp_hi, off);
    t.nb = t.pu;
    t.kind = KIND_NONE;
    if (lane < t.n) {
        const int j = q + lane - pA_lo;
        const int deg = prp_hi - prp_lo;
        if (j < deg) {
            t.nb = __ldg(&a.col_idx[prp_lo + j]);
            t.kind = KIND_ATTR;
        } else if (j - deg < a.s) {
            const uint32_t x0 =
                philox_x0((uint32_t)t.pu, a.epoch, (uint32_t)(j - deg), 0u, a.key0, a.key1);
            t.nb = (int)(x0 % (uint32_t)a.n);
            t.kind = (t.nb == t.pu) ? KIND_NONE : KIND_REP;
        }
    }
    t.nverts = __shfl_sync(0xffffffffu, off, t.n - 1) + 1;
    t.u_next = u + __popc(__ballot_sync(0xffffffffu, pos <= t.n));
    return t;
}

template <int D, typename Ts>
__global__ void __launch_bounds__(D <= 64 ? 512 : 320) force_bulk_kernel(const ForceArgs<Ts> a)
{
    using Lay = BulkLayout<D, Ts>;
    constexpr int EPL = D / 32;                     // elements per lane
    constexpr int VEC = EPL >= 4 ? 4 : EPL;
    constexpr int NV = EPL / VEC;
    constexpr int L = 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    unsigned char *wsm = smem_raw + (size_t)warp * Lay::BYTES;
    Ts *rows = reinterpret_cast<Ts *>(wsm + Lay::ROWS_OFF);
    float *own = reinterpret_cast<float *>(wsm + Lay::OWN_OFF);
    float *coefs = reinterpret_cast<float *>(wsm + Lay::COEF_OFF);
    int *vert = reinterpret_cast<int *>(wsm + Lay::VERT_OFF);
    int *vends = reinterpret_cast<int *>(wsm + Lay::VEND_OFF);
    int *kinds = reinterpret_cast<int *>(wsm + Lay::KIND_OFF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(wsm + Lay::BAR_OFF);
    const bool tdist = (a.model == 0);

    // zero the staging buffers once, so rows that are never copied are finite
    {
        float4 *zb = reinterpret_cast<float4 *>(wsm + Lay::ROWS_OFF);
        const int n16 = (Lay::COEF_OFF - Lay::ROWS_OFF) / 16;
        for (int i = lane; i < n16; i += 32) zb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    __syncwarp();
    uint32_t phase = 0;

    for (int chunk = blockIdx.x * warps + warp; chunk < a.n_items; chunk += gridDim.x * warps) {
        const int q_begin = chunk * a.C;
        const int q_end = min(q_begin + a.C, a.Pk);
        const int u0 = __ldg(&a.item_u0[chunk]);
        Tile t = decode_tile(a, q_begin, q_end, u0, lane);
        int ucur = -1, vbeg = 0, vend = 0;
        float zu[EPL], g[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) { zu[e] = 0.f; g[e] = 0.f; }

        while (true) {
            // ---- stage the tile: partner rows and own rows, one mbarrier --
            const int myvert = (lane < t.n) ? t.pu - t.u : 0;
            vert[lane] = myvert;
            vends[lane] = t.p_hi;
            const bool has_row = (lane < t.n) && (t.kind != KIND_NONE);
            const bool has_own = lane < t.nverts;
            const uint32_t bytes =
                (uint32_t)__popc(__ballot_sync(0xffffffffu, has_row)) * Lay::ROWB +
                (uint32_t)t.nverts * Lay::OWNB;
            // rows where a new vertex segment begins
            const int prev_vert = __shfl_up_sync(0xffffffffu, myvert, 1);
            const unsigned seg_starts =
                __ballot_sync(0xffffffffu, lane < t.n && (lane == 0 || prev_vert != myvert));
            fence_proxy_async_smem();
            __syncwarp();
            if (has_row) {
                const Ts *src = ((t.nb < a.mb_begin) ? a.znext : a.zcur) + (int64_t)t.nb * a.ld;
                bulk_copy_g2s(rows + lane * D, src, Lay::ROWB, bar);
            }
            if (has_own) {
                const int w = t.u + lane;
                const float *src = (sizeof(Ts) == 2) ? a.master + (int64_t)w * a.ld
                                                     : reinterpret_cast<const float *>(a.zcur) +
                                                           (int64_t)w * a.ld;
                bulk_copy_g2s(own + lane * D, src, Lay::OWNB, bar);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
            const int tn = t.n, tu = t.u, tq = t.q, first_lo = t.first_lo;
            const int tkind = (lane < t.n) ? t.kind : KIND_NONE;

            // ---- decode the next tile while the copies are in flight ------
            const int q_next = tq + tn;
            const bool more = q_next < q_end;
            if (more) t = decode_tile(a, q_next, q_end, t.u_next, lane);

            if (!mbar_wait_bounded(bar, phase)) {
                if (lane == 0) atomicExch(a.err, 1);
                mbar_wait_bounded(bar, phase);      // let the copies land before leaving
                return;
            }
            phase ^= 1u;
            __syncwarp();

            // ---- reduce: partial sums of all 32 rows (rows past the tile and
            // rows without a copy hold finite stale data and are discarded),
            // then a transpose-reduction leaves row r's sum in lane r.
            float p[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int j = vert[r];
                float x[EPL], o[EPL];
#pragma unroll
                for (int i = 0; i < NV; ++i) {
                    const int e0 = (i * L + lane) * VEC;
                    load_vec_smem<VEC>(rows + r * D + e0, x + i * VEC);
                    load_vec_smem<VEC>(own + j * D + e0, o + i * VEC);
                }
                float acc = 0.f;
                if (tdist) {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        const float df = o[e] - x[e];
                        acc = fmaf(df, df, acc);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) acc = fmaf(o[e], x[e], acc);
                }
                p[r] = acc;
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                const bool upper = (lane & m) != 0;
#pragma unroll
                for (int i = 0; i < m; ++i) {
                    const float send = upper ? p[i] : p[i + m];
                    const float keep = upper ? p[i + m] : p[i];
                    p[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                }
            }
            // ---- force: lane r turns row r's sum into its pair's scalar -----
            {
                const float sdot = p[0];
                float coef = 0.f;
                if (tkind != KIND_NONE) {
                    if (tdist) {
                        if (tkind == KIND_ATTR) {
                            coef = 2.f / (1.f + sdot);                 // Eq. 8 / t
                        } else {
                            const float q2 = fmaxf(sdot, kT2Floor);
                            coef = -2.f / (q2 * (1.f + q2));           // Eq. 9 / t
                        }
                    } else {
                        coef = (tkind == KIND_ATTR) ? -1.f / (1.f + expf(sdot))   // Eq. 5
                                                    : 1.f / (1.f + expf(-sdot));  // Eq. 6
                    }
                }
                coefs[lane] = coef;              // 0 for pairs without a force
            }
            __syncwarp();

            // ---- accumulate each vertex segment; finish vertices that end ---
            unsigned starts = seg_starts;
            while (starts) {
                const int rs = __ffs(starts) - 1;
                starts &= starts - 1;
                const int re = starts ? __ffs(starts) - 1 : tn;
                const int j = vert[rs];
                if (tu + j != ucur) {
                    if (ucur >= 0)
                        finish_vertex<32, VEC, NV, true>(a, 0xffffffffu, lane, chunk, ucur, vbeg,
                                                         vend, zu, g);
                    vbeg = (ucur >= 0) ? vend : first_lo;
                    ucur = tu + j;
                    vend = vends[rs];
#pragma unroll
                    for (int i = 0; i < NV; ++i)
                        load_vec_smem<VEC>(own + j * D + (i * L + lane) * VEC, zu + i * VEC);
#pragma unroll
                    for (int e = 0; e < EPL; ++e) g[e] = 0.f;
                }
                for (int r0 = rs; r0 < re; r0 += 4) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = min(r0 + i, 31);
                        const float c = (r0 + i < re) ? coefs[r] : 0.f;
                        float x[EPL];
#pragma unroll
                        for (int k = 0; k < NV; ++k)
                            load_vec_smem<VEC>(rows + r * D + (k * L + lane) * VEC, x + k * VEC);
                        if (tdist) {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) g[e] = fmaf(c, zu[e] - x[e], g[e]);
                        } else {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) g[e] = fmaf(c, x[e], g[e]);
                        }
                    }
                }
            }
            __syncwarp();
            if (!more) break;
        }
        if (ucur >= 0)
            finish_vertex<32, VEC, NV, true>(a, 0xffffffffu, lane, chunk, ucur, vbeg, vend, zu, g);
    }
}

constexpr int kBulkSmemBudget = 220 * 1024;

template <int D, typename Ts>
int bulk_warps()
{
    const int w = kBulkSmemBudget / BulkLayout<D, Ts>::BYTES;
    const int cap = (D <= 64 ? 512 : 320) / 32;       // the kernel's launch bound
    return w > cap ? cap : w;
}

template <typename Ts>
bool bulk_config_t(int d, int *warps, int *smem)
{
    switch (d) {
        case 64: *warps = bulk_warps<64, Ts>(); *smem = *warps * BulkLayout<64, Ts>::BYTES; return true;
        case 128: *warps = bulk_warps<128, Ts>(); *smem = *warps * BulkLayout<128, Ts>::BYTES; return true;
        case 256: *warps = bulk_warps<256, Ts>(); *smem = *warps * BulkLayout<256, Ts>::BYTES; return true;
        default: return false;
    }
}

template <int D, typename Ts>
cudaError_t launch_bulk_d(const ForceArgs<Ts> &a, int blocks, int warps, int smem,
                          cudaStream_t st)
{
    static bool attr_set = false;          // per instantiation; set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(force_bulk_kernel<D, Ts>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    force_bulk_kernel<D, Ts><<<blocks, warps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename Ts>
cudaError_t launch_bulk_t(int d, const ForceArgs<Ts> &a, int blocks, int warps, int smem,
                          cudaStream_t st)
{
    switch (d) {
        case 64: return launch_bulk_d<64, Ts>(a, blocks, warps, smem, st);
        case 128: return launch_bulk_d<128, Ts>(a, blocks, warps, smem, st);
        case 256: return launch_bulk_d<256, Ts>(a, blocks, warps, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace f2v
