// f2v_bulk.cuh -- the persistent force+update kernel for row sizes
// d = 32 * EPL (EPL = 2, 4, 8), with partner rows staged in shared memory by
// TMA bulk copies.  One launch runs a range of minibatches of one epoch.
//
// Work.  Minibatch k's pair sequence (neighbours of each vertex in CSR
// order, then its s negative samples) is cut into chunks of C_k pairs (about
// two per warp); a free warp takes the next unclaimed chunk of the oldest
// minibatch that has one left, so warps flow from one minibatch into the next
// without a grid-wide barrier, and a slow chunk holds up no warp but its own.
// With FP32 rows and chunks of at most 512 pairs, a block claims a group of
// 16 consecutive chunks at a time and its warps take them in order from a
// shared-memory queue (BlockQueue below).
// Per tile of at most 32 pairs spanning at most kOwnSlots (4) vertices:
//   decode  lane t finds pair t's vertex and partner (the epoch's partner list);
//   stage   TMA gather4 copies bring the tile's partner rows and own rows
//           into the warp's shared buffers, completing on one mbarrier; the
//           next tile (possibly of the next chunk) is decoded while the
//           copies are in flight;
//   reduce  each lane forms the partial dot product / squared distance of
//           all 32 rows over its EPL elements, and a transpose-reduction
//           (31 shuffles) leaves lane r with row r's full sum;
//   force   lane r turns its sum into the scalar of Eq. 5/6 or Eq. 8/9;
//   update  rows are accumulated per vertex in registers; a vertex that
//           ends is written (z_u - eta g, Eq. 10) or, if it spans several
//           chunks, passed up the ordered combine tree of f2v_internal.h.
//
// Ordering between minibatches (synchronous SGD, Sec. III-B).  A partner row
// v of an earlier minibatch is read from the next buffer only after its
// flag row_flag[v] equals epoch + 1, which its writer releases after the row
// is stored.  A warp holds one chunk at a time and waits only for rows of
// older minibatches, whose chunks were all claimed by running warps, so the
// oldest unfinished chunk always progresses (no block needs to wait for a
// block that is not resident).  The combine-tree scratch is a ring of `ring`
// regions; before it starts a chunk of minibatch k a warp waits until
// minibatch k - ring is complete.
//
// Every wait is bounded (about a second at 2 GHz): on expiry the kernel
// records an error code (1 mbarrier, 2 row flag, 3 ring), lets its own copies
// land, and returns; the host reports F2V_ETIMEOUT.
#pragma once

#include <algorithm>
#include <climits>

#include "f2v_device.cuh"
#include "f2v_force.cuh"
#include "f2v_internal.h"

namespace f2v {

constexpr int kOwnSlots = 4;                 // distinct vertices per tile at most
// A tile finishes at most kOwnSlots + 1 vertices (the one it continues, the
// ones it holds, and at a chunk's end its last).
constexpr int kMaxPub = kOwnSlots + 1;
// own rows arrive by tile::gather4 copies of four rows each into a buffer of
// kOwnSlots rows, so the buffer must hold whole copies
static_assert(kOwnSlots % 4 == 0 && kOwnSlots <= 8, "kOwnSlots: a multiple of 4, at most 8");

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

// TMA tile::gather4: rows r0..r3 (each one box = one whole row) of the 2-D
// tensor behind `map` into consecutive rows at dst, completing on `bar`.
__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *map, int r0, int r1,
                                            int r2, int r3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1),
          "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}


__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_relaxed_gpu(int32_t *p, int32_t v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A lane's part of a pair's reduced scalar over its EPL elements: the squared
// distance (tdist) or the dot product of its own-row and partner slices.
// PACKED: as two interleaved partial sums (even and odd elements) added at the
// end, with packed instructions; else one sequential sum.  (Packed halves the
// instructions but holds more registers: it is faster for BF16 rows, which
// also widen each element; for FP32 rows it made the kernel spill or run
// slower.)
template <int EPL, bool TDIST, bool PACKED>
__device__ __forceinline__ float lane_reduce(const float *o, const float *x)
{
    if (!PACKED) {
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            if (TDIST) {
                const float df = o[e] - x[e];
                acc = fmaf(df, df, acc);
            } else {
                acc = fmaf(o[e], x[e], acc);
            }
        }
        return acc;
    }
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int e = 0; e < EPL; e += 2) {
        if (TDIST) {
            float d0, d1;
            sub2(d0, d1, o[e], o[e + 1], x[e], x[e + 1]);
            fma2(s0, s1, d0, d1, d0, d1);
        } else {
            fma2(s0, s1, o[e], o[e + 1], x[e], x[e + 1]);
        }
    }
    return s0 + s1;
}

// The squared distance of a lane's EPL elements of an own row (FP32) and a
// BF16 partner row (EPL / 2 packed words), as two interleaved partial sums.
// Each difference is x - o rounded once, the negation of o - x rounded
// once, so the sums equal lane_reduce's on the widened row.
template <int EPL>
__device__ __forceinline__ float lane_dist_bf16(const float *o, const unsigned int *w)
{
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int e = 0; e < EPL; e += 2) {
        float d0, d1;
        sub_bf16x2_f32(d0, d1, w[e / 2], o[e], o[e + 1]);
        fma2(s0, s1, d0, d1, d0, d1);
    }
    return s0 + s1;
}

// A lane's EPL / 2 packed words of a BF16 row in shared memory.
template <int VEC>
__device__ __forceinline__ void load_words_smem(const __nv_bfloat16 *p, unsigned int *w)
{
    if constexpr (VEC == 4) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        w[0] = t.x;
        w[1] = t.y;
    } else {
        w[0] = *reinterpret_cast<const unsigned int *>(p);
    }
}

// acc += c * x, element by element.
template <int EPL>
__device__ __forceinline__ void lane_axpy(float *acc, float c, const float *x)
{
#pragma unroll
    for (int e = 0; e < EPL; e += 2) fma2(acc[e], acc[e + 1], c, c, x[e], x[e + 1]);
}

// Bounded wait on an mbarrier phase; false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
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
    static constexpr int BAR_OFF = VEND_OFF + 32 * 4;              // uint64
    // the tile's finished vertices whose flags are pending (kMaxPub ids)
    static constexpr int PEND_OFF = BAR_OFF + 8;
    static constexpr int BYTES = ((PEND_OFF + 4 * kMaxPub + 127) / 128) * 128;
};

// One chunk of one minibatch.
struct Chunk {
    int idx;               // chunk index within the minibatch
    int k;                 // minibatch
    int mb_begin;          // its first vertex
    int64_t P0;            // its first pair (global index)
    int q_begin, q_end;    // the chunk's pairs, local to the minibatch
    int C;                 // pairs per chunk in this minibatch
    int u0;                // vertex holding pair q_begin
};

// Per-warp claims (the BF16 instantiations): the next unclaimed chunk of the
// first minibatch >= k of the launch that has one left (mb_next[k] counts the
// chunks handed out); false if none.  Whichever warp is free takes the next
// chunk, so a slow chunk delays its own minibatch only, not every later one.
template <typename Ts>
__device__ __forceinline__ bool find_chunk(const EpochArgs<Ts> &a, int lane, int k, Chunk &c)
{
    for (; k < a.k_end; ++k) {
        const int64_t base = __ldg(&a.mb_item_base[k]);
        const int64_t nch = __ldg(&a.mb_item_base[k + 1]) - base;
        int w = 0;
        if (lane == 0) w = atomicAdd(&a.mb_next[k], 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w < nch) {
            c.idx = w;
            c.k = k;
            c.mb_begin = k * a.b;
            const int mb_end = min(a.f.n, c.mb_begin + a.b);
            c.P0 = __ldg(&a.f.apair[c.mb_begin]);
            const int Pk = (int)(__ldg(&a.f.apair[mb_end]) - c.P0);
            c.C = __ldg(&a.mb_C[k]);
            c.q_begin = w * c.C;
            c.q_end = min(c.q_begin + c.C, Pk);
            c.u0 = __ldg(&a.items[base + w]);
            return true;
        }
    }
    return false;
}

// Group claims (the FP32 instantiations).  Chunks are handed out in groups.
// A group is the kFan consecutive chunks
// of a minibatch that form one level-1 unit of the combine tree, and all of a
// group's chunks are walked by the warps of one block: a vertex cut by a chunk
// boundary inside a group is combined by warps of that block alone, so those
// arrivals synchronise at block scope (no wait for stores to reach L2).
// A block takes the next unclaimed group of the oldest minibatch that has one
// left (per-minibatch counters, mb_next); its warps take the group's chunks in
// order as they become free, so a slow chunk delays its own minibatch only.
//
// The block's queue lives in shared memory: a 64-bit word holds the current
// group's sequence number (high half) and the tickets handed out for it (low
// half), so one atomic add gives a warp both; ticket t < n is chunk t of the
// group.  The warp that draws the first ticket past the end installs the next
// group (under a lock): it claims one from the minibatch counters, writes its
// record into a small ring indexed by sequence number, then starts the new
// sequence.  A record carries its sequence number; a warp that finds another
// there (the ring wrapped while it held a ticket, which needs eight installs
// within a few instructions) reports an error instead of losing the chunk.
constexpr int kGroupRing = 8;
struct BlockQueue {
    unsigned long long word;       // sequence << 32 | tickets handed out
    int lock;
    int pad;
    int4 rec[kGroupRing];          // sequence s: {minibatch, first chunk, chunks (-1: none left), s}
};
constexpr int kQueueBytes = 256;
static_assert(sizeof(BlockQueue) <= kQueueBytes, "queue area");

// The next unclaimed group of the first minibatch >= k of the launch, as a
// record of sequence `seq` (lane 0 only).
template <typename Ts>
__device__ __forceinline__ int4 claim_group(const EpochArgs<Ts> &a, int k, unsigned seq)
{
    for (; k < a.k_end; ++k) {
        const int64_t base = __ldg(&a.mb_item_base[k]);
        const int nch = (int)(__ldg(&a.mb_item_base[k + 1]) - base);
        const int g = atomicAdd(&a.mb_next[k], 1);
        if (g * kFan < nch) return make_int4(k, g * kFan, min(kFan, nch - g * kFan), (int)seq);
    }
    return make_int4(a.k_end, 0, -1, (int)seq);
}

__device__ __forceinline__ int4 load_rec(const BlockQueue *q, unsigned seq)
{
    const volatile int *r = reinterpret_cast<const volatile int *>(&q->rec[seq % kGroupRing]);
    return make_int4(r[0], r[1], r[2], r[3]);
}

// Takes the block's next chunk; false if none is left (or, after setting the
// error word, if the queue failed).
template <typename Ts>
__device__ __forceinline__ bool next_chunk(const EpochArgs<Ts> &a, int lane, BlockQueue *q,
                                           Chunk &c)
{
    int k = 0, idx = -1;                           // idx: -1 no more work, -2 error
    if (lane == 0) {
        const long long t0 = clock64();
        while (true) {
            const unsigned long long old = atomicAdd(&q->word, 1ull);
            const unsigned seq = (unsigned)(old >> 32), t = (unsigned)old;
            const int4 r = load_rec(q, seq);
            if (r.w != (int)seq) { idx = -2; break; }
            if (r.z < 0) break;                    // every group is taken
            if ((int)t < r.z) { k = r.x; idx = r.y + (int)t; break; }
            // the group is used up: one warp installs the next one
            if (atomicCAS(&q->lock, 0, 1) == 0) {
                if ((unsigned)(atomicAdd(&q->word, 0ull) >> 32) == seq) {
                    const int4 nr = claim_group(a, r.x, seq + 1);
                    volatile int *w = reinterpret_cast<volatile int *>(&q->rec[(seq + 1) % kGroupRing]);
                    w[0] = nr.x; w[1] = nr.y; w[2] = nr.z; w[3] = nr.w;
                    __threadfence_block();
                    atomicExch(&q->word, (unsigned long long)(seq + 1) << 32);
                }
                __threadfence_block();
                atomicExch(&q->lock, 0);
            } else {
                const volatile unsigned long long *wv = &q->word;
                while ((unsigned)(*wv >> 32) == seq) {
                    if (clock64() - t0 > kWaitCycles) break;
                }
            }
            if (clock64() - t0 > kWaitCycles) { idx = -2; break; }
        }
    }
    idx = __shfl_sync(0xffffffffu, idx, 0);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (idx < 0) {
        if (idx == -2 && lane == 0) atomicExch(a.f.err, 3);
        return false;
    }
    c.idx = idx;
    c.k = k;
    c.mb_begin = k * a.b;
    const int mb_end = min(a.f.n, c.mb_begin + a.b);
    c.P0 = __ldg(&a.f.apair[c.mb_begin]);
    const int Pk = (int)(__ldg(&a.f.apair[mb_end]) - c.P0);
    c.C = __ldg(&a.mb_C[k]);
    c.q_begin = idx * c.C;
    c.q_end = min(c.q_begin + c.C, Pk);
    c.u0 = __ldg(&a.items[__ldg(&a.mb_item_base[k]) + idx]);
    return true;
}

// Lane-parallel decode of the tile starting at pair q (local to the chunk's
// minibatch), within the chunk, whose first pair lies in vertex u.
struct Tile {
    int q, n, u;          // first pair, pairs in the tile, vertex of the first pair
    int nverts;           // distinct vertices in the tile (<= kOwnSlots)
    int u_next;           // vertex holding pair q + n
    int first_lo;         // start of vertex u (local pair index)
    // per lane (pair q + lane)
    int pu, nb, kind, p_hi;
    bool ready;           // partner row may be read now
};

template <typename Ts>
__device__ __forceinline__ Tile decode_tile(const EpochArgs<Ts> &a, const Chunk &ch, int q,
                                            int u, int lane)
{
    Tile t;
    t.q = q;
    t.u = u;
    const int q_end = ch.q_end;
    const int uu = u + lane;
    // two independent loads per lane: the end of vertex u + lane, and the
    // partner code of pair q + lane
    int A_hi = INT_MAX;
    if (uu < a.f.n) {
        const int64_t ah = __ldg(&a.f.apair[uu + 1]) - ch.P0;
        A_hi = ah > INT_MAX ? INT_MAX : (int)ah;
    }
    const int code = (q + lane < q_end) ? __ldg(&a.partner[ch.P0 + q + lane]) : kPartnerNone;
    const int A_up = __shfl_up_sync(0xffffffffu, A_hi, 1);
    const int A_lo = (lane == 0) ? (int)(__ldg(&a.f.apair[u]) - ch.P0) : A_up;
    t.first_lo = __shfl_sync(0xffffffffu, A_lo, 0);
    // at most 32 pairs, at most kOwnSlots vertices, not past the chunk
    const int end8 = __shfl_sync(0xffffffffu, A_hi, kOwnSlots - 1);
    t.n = min(32, min(q_end - q, end8 - q));
    const int pos = A_hi - q;                         // >= 1
    const unsigned bit = (pos < 32) ? (1u << pos) : 0u;
    const unsigned ends = __reduce_or_sync(0xffffffffu, bit);
    const int off = __popc(ends & ((2u << lane) - 1u));
    t.pu = u + off;
    t.p_hi = __shfl_sync(0xffffffffu, A_hi, off);
    t.nb = t.pu;
    t.kind = KIND_NONE;
    t.ready = true;
    if (lane < t.n) {
        if (code >= 0) {
            t.nb = code;
            t.kind = KIND_ATTR;
        } else if (code != kPartnerNone) {
            t.nb = -2 - code;
            t.kind = KIND_REP;
        }
        // a row of an earlier minibatch: readable once its writer released it
        if (t.kind != KIND_NONE && t.nb < ch.mb_begin)
            t.ready = ld_acquire(&a.row_flag[t.nb]) == (int)a.f.epoch + 1;
    }
    t.nverts = __shfl_sync(0xffffffffu, off, t.n - 1) + 1;
    t.u_next = u + __popc(__ballot_sync(0xffffffffu, pos <= t.n));
    return t;
}

// Finishing vertices.  A vertex whose pairs all lie in the tile's chunk gets
// its new row stored at once, but its flag is set only after the tile: one
// release fence then covers every row the tile stored, and the flags (and the
// chunk's completion count) follow with relaxed stores.  A release fence
// waits for the warp's stores to reach L2, which costs about as much as a
// tile's arithmetic, so one per tile instead of one per vertex pays.  A vertex
// split across chunks arrives at its combine-tree counter at once: the
// arrival decides which part completes the vertex, and delaying it delays
// every later minibatch that reads the row.

// The part of vertex u (local pairs [vbeg, vend)) summed in g over level-0
// unit `unit0` goes up the ordered combine tree of f2v_internal.h.  Level-0
// units are chunks and level-1 units are the groups one block walks, so the
// parts that meet at a level-0 counter all come from this block: that arrival
// is released and acquired at block scope.  Higher levels join parts of
// several blocks with GPU-scope acquire-release arrivals.  Returns true if
// this warp completed the vertex and stored its row (the flag is then set
// with the tile's).
template <int VEC, int NV, int MODEL, typename Ts>
__device__ __forceinline__ bool finish_split(const ForceArgs<Ts> &a, const FinishCtx &fc,
                                             int lane, int unit0, int u, int vbeg, int vend,
                                             const float *zu, float *g)
{
    constexpr int E = VEC * NV;
    int64_t fu = vbeg / fc.C, lu = (vend - 1) / fc.C;
    int64_t unit = unit0, unit_pairs = fc.C, units = a.units0;
    float *slot_base = fc.slots;
    int32_t *cnt_base = fc.unit_cnt;
    for (int lvl = 0; lvl + 1 < kMaxLevels; ++lvl) {
        store_row_cg<32, VEC, NV, true>(slot_base + unit_slot(unit, vbeg, unit_pairs) * a.ld,
                                        lane, a.d, g);
        const int64_t parent = unit / kFan;
        const int64_t pfu = fu / kFan, plu = lu / kFan;
        const int64_t c0 = max(fu, parent * kFan);
        const int64_t c1 = min(lu, parent * kFan + (kFan - 1));
        const bool top = (pfu == plu);
        const int64_t punits = (units + kFan - 1) / kFan;
        int32_t *cnt = top ? &a.counter[u] : &cnt_base[unit_slot(parent, vbeg, unit_pairs * kFan)];
        __syncwarp();
        int prior = 0;
        if (lane == 0) {
            if (lvl == 0) {
                asm volatile("fence.acq_rel.cta;" ::: "memory");
                asm volatile("atom.relaxed.cta.global.add.s32 %0, [%1], 1;"
                             : "=r"(prior)
                             : "l"(cnt)
                             : "memory");
            } else {
                asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;"
                             : "=r"(prior)
                             : "l"(cnt)
                             : "memory");
            }
        }
        prior = __shfl_sync(0xffffffffu, prior, 0);
        if (prior != (int)(c1 - c0)) return false;     // a sibling completes it
        if (lvl == 0 && lane == 0) asm volatile("fence.acq_rel.cta;" ::: "memory");
        __syncwarp();                                   // the other lanes read after the acquire
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = 0.f;
        for (int64_t c = c0; c <= c1; c += 4) {         // children in order
            float part[4][E];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c + k <= c1)
                    load_row_cg<32, VEC, NV, true>(
                        slot_base + unit_slot(c + k, vbeg, unit_pairs) * a.ld, lane, a.d, part[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c + k <= c1) {
#pragma unroll
                    for (int e = 0; e < E; ++e) g[e] += part[k][e];
                }
        }
        if (lane == 0) *cnt = 0;
        if (top) {
            const FinishCtx quiet{fc.C, fc.slots, fc.unit_cnt, nullptr, 0};
            write_row<32, VEC, NV, true, MODEL>(a, quiet, 0xffffffffu, u, lane, zu, g);
            return true;
        }
        slot_base += 2 * units * a.ld;
        cnt_base += 2 * punits;
        unit = parent;
        fu = pfu;
        lu = plu;
        units = punits;
        unit_pairs *= kFan;
    }
    return false;
}

// Vertex u (local pairs [vbeg, vend), summed in g over level-0 unit
// `unit0`) ends: if the unit held all its pairs, store z_u - eta g (Eq. 10)
// and list u for its flag; else pass its part up the combine tree, listing u
// if that completed it.
// GROUPS: the chunks of each level-1 unit are walked by one block (group
// claims), so level-0 arrivals synchronise at block scope (finish_split);
// else every arrival is GPU-scope (finish_vertex, which also sets the flag of
// a row it completes).
template <int VEC, int NV, int MODEL, bool GROUPS, typename Ts>
__device__ __forceinline__ void finish_store(const ForceArgs<Ts> &a, const FinishCtx &fc, int lane,
                                             int unit0, int u, int vbeg, int vend,
                                             const float *zu, float *g, int *pend, int &npub,
                                             bool groups)
{
    bool written = true;
    if (vbeg / fc.C == (vend - 1) / fc.C) {
        const FinishCtx quiet{fc.C, fc.slots, fc.unit_cnt, nullptr, 0};
        write_row<32, VEC, NV, true, MODEL>(a, quiet, 0xffffffffu, u, lane, zu, g);
    } else if (GROUPS && groups) {
        written = finish_split<VEC, NV, MODEL>(a, fc, lane, unit0, u, vbeg, vend, zu, g);
    } else {
        finish_vertex<32, VEC, NV, true, MODEL>(a, fc, 0xffffffffu, lane, unit0, u, vbeg, vend,
                                                zu, g);
        written = false;
    }
    if (written) {
        if (lane == 0) pend[npub] = u;
        ++npub;
    }
}

template <int D, typename Ts, int MODEL, bool GROUPS>
__global__ void __launch_bounds__((D <= 64) ? 512 : 384)
    force_bulk_kernel(const __grid_constant__ EpochArgs<Ts> a,
                      const __grid_constant__ CUtensorMap zmap,
                      const __grid_constant__ CUtensorMap mmap)
{
    using Lay = BulkLayout<D, Ts>;
    constexpr int EPL = D / 32;                     // elements per lane
    constexpr int VEC = EPL >= 4 ? 4 : EPL;
    constexpr int NV = EPL / VEC;
    constexpr int L = 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *wsm = smem_raw + (size_t)warp * Lay::BYTES;
    Ts *rows = reinterpret_cast<Ts *>(wsm + Lay::ROWS_OFF);
    float *own = reinterpret_cast<float *>(wsm + Lay::OWN_OFF);
    float *coefs = reinterpret_cast<float *>(wsm + Lay::COEF_OFF);
    int *vert = reinterpret_cast<int *>(wsm + Lay::VERT_OFF);
    int *vends = reinterpret_cast<int *>(wsm + Lay::VEND_OFF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(wsm + Lay::BAR_OFF);
    int *pend = reinterpret_cast<int *>(wsm + Lay::PEND_OFF);
    // the force model class, fixed per instantiation: every model but the
    // sigmoid reduces a squared distance and accumulates c (z_u - x)
    constexpr bool tdist = (MODEL != 1);
    constexpr bool kPackReduce = (sizeof(Ts) == 2);
    // BF16 rows, distance models: widening and subtraction in one instruction
    constexpr bool kMixedSub = (sizeof(Ts) == 2) && tdist && (VEC >= 2);
    // GROUPS: group claims with block-scope level-0 combining (the host
    // picks the instantiation, see launch_bulk_d)
    constexpr bool kGroups = GROUPS;
    constexpr bool groups = GROUPS;
    const int model = model_of<MODEL>(a.f.model);
    const int flag_value = (int)a.f.epoch + 1;
    // Where a tile's flags are published: at the end of its iteration, or
    // (kPublishAtTop) at the top of the next one.  Only the loop's back edge
    // lies between the two, so they publish at the same moment; the code
    // differs.  At the top, the sigmoid instantiation with group claims fits
    // its registers without spilling (R-MAT 20, d = 128, b = 4096: 4.27 ->
    // 3.91 ms per launch); the t model runs 0.8% faster with the publish at
    // the end.
    constexpr bool kPublishAtTop = (MODEL == 1) && GROUPS;
    int npend = 0;                 // kPublishAtTop: the last tile's pending flags,
    bool pend_chunk = false;       // whether it ended its chunk,
    int pend_k = 0;                // and the chunk's minibatch
    auto publish_pending = [&]() {
        if (npend > 0 || pend_chunk) {
            __syncwarp();
            fence_acq_rel_gpu();
            if (lane < npend) st_relaxed_gpu(&a.row_flag[pend[lane]], flag_value);
            if (pend_chunk && lane == 0)
                asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(&a.mb_done[pend_k])
                             : "memory");
            npend = 0;
            pend_chunk = false;
        }
    };

    // zero the staging buffers once, so rows that are never copied are finite
    {
        float4 *zb = reinterpret_cast<float4 *>(wsm + Lay::ROWS_OFF);
        const int n16 = (Lay::COEF_OFF - Lay::ROWS_OFF) / 16;
        for (int i = lane; i < n16; i += 32) zb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    // the block's group queue: no group yet (the first ticket installs one)
    BlockQueue *queue = reinterpret_cast<BlockQueue *>(smem_raw + (size_t)(blockDim.x >> 5) * Lay::BYTES);
    if (threadIdx.x == 0) {
        queue->word = 0ull;
        queue->lock = 0;
        queue->rec[0] = make_int4(a.k_begin, 0, 0, 0);
    }
    __syncthreads();
    uint32_t phase = 0;

    Chunk ch;
    if (!(groups ? next_chunk(a, lane, queue, ch) : find_chunk(a, lane, a.k_begin, ch))) return;
    Tile t = decode_tile(a, ch, ch.q_begin, ch.u0, lane);
    bool chunk_start = true;
    int ring_known = a.k_begin - 1;    // minibatches up to this one are known complete
    int ucur = -1, vbeg = 0, vend = 0;
    float zu[EPL], g[EPL];
    // t model: the sum of c * (z_u - x) is kept as the sum of -c * x plus
    // z_u times the sum of c (one multiply-add per element instead of a
    // subtract and a multiply-add); it is folded in before the vertex's
    // gradient leaves the warp
    float csum = 0.f;
#pragma unroll
    for (int e = 0; e < EPL; ++e) { zu[e] = 0.f; g[e] = 0.f; }

    while (true) {
        if constexpr (kPublishAtTop) publish_pending();
        // ---- minibatch entry: the scratch region must be free ------------
        if (chunk_start) {
            chunk_start = false;
            // (a warp's chunks come in minibatch order, so a region seen free
            // for one chunk stays free for the warp's later chunks)
            if (ch.k - a.ring >= a.k_begin && ch.k - a.ring > ring_known) {
                const int kk = ch.k - a.ring;
                ring_known = kk;
                const int target =
                    (int)(__ldg(&a.mb_item_base[kk + 1]) - __ldg(&a.mb_item_base[kk]));
                int ok = 1;
                if (lane == 0) ok = wait_at_least(&a.mb_done[kk], target);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    if (lane == 0) atomicExch(a.f.err, 3);
                    return;
                }
            }
        }
        // ---- rows of earlier minibatches: wait until written ------------
        const bool has_row = (lane < t.n) && (t.kind != KIND_NONE);
        if (__any_sync(0xffffffffu, has_row && !t.ready)) {
            int ok = 1;
            if (has_row && !t.ready) ok = wait_equal(&a.row_flag[t.nb], flag_value);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicExch(a.f.err, 2);
                return;
            }
        }
        // rows written in this launch are read through the async proxy next
        if (__any_sync(0xffffffffu, has_row && t.nb < ch.mb_begin)) fence_proxy_async_global();

        // ---- stage the tile: partner rows and own rows, one mbarrier -----
        const int myvert = (lane < t.n) ? t.pu - t.u : 0;
        vert[lane] = myvert;
        vends[lane] = t.p_hi;
        // map row of each lane's partner (a finite stand-in where there is none)
        const int prow = has_row ? t.nb + ((t.nb < ch.mb_begin) ? a.znext_row0 : a.zcur_row0)
                                 : a.zcur_row0 + t.u;
        const int ngroups = (t.n + 3) >> 2;          // gather4 loads of partner rows
        const int nown = (t.nverts + 3) >> 2;        // gather4 loads of own rows (<= 2)
        const uint32_t bytes = (uint32_t)ngroups * 4u * Lay::ROWB + (uint32_t)nown * 4u * Lay::OWNB;
        int r4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) r4[i] = __shfl_sync(0xffffffffu, prow, (4 * lane + i) & 31);
        // rows where a new vertex segment begins
        const int prev_vert = __shfl_up_sync(0xffffffffu, myvert, 1);
        const unsigned seg_starts =
            __ballot_sync(0xffffffffu, lane < t.n && (lane == 0 || prev_vert != myvert));
        // The copies below overwrite the buffers the previous tile was read
        // from.  No proxy fence is needed for that: a warp issues in order,
        // and every shared-memory read of the previous tile fed an arithmetic
        // instruction issued before this point, so it had returned its value.
        __syncwarp();
        if (lane < ngroups) {
            tma_gather4(rows + 4 * lane * D, &zmap, r4[0], r4[1], r4[2], r4[3], bar);
        } else if (lane >= 8 && lane < 8 + nown) {
            int o4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                o4[i] = a.own_row0 + t.u + min(4 * (lane - 8) + i, t.nverts - 1);
            tma_gather4(own + 4 * (lane - 8) * D, &mmap, o4[0], o4[1], o4[2], o4[3], bar);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
        const int tn = t.n, tu = t.u, tq = t.q, first_lo = t.first_lo;
        const int tkind = (lane < t.n) ? t.kind : KIND_NONE;
        const Chunk cur = ch;

        // ---- decode the next tile (maybe of the next minibatch) ----------
        const int q_next = tq + tn;
        const bool last_of_chunk = q_next >= cur.q_end;
        bool more = true;
        if (!last_of_chunk) {
            t = decode_tile(a, cur, q_next, t.u_next, lane);
        } else if (groups ? next_chunk(a, lane, queue, ch) : find_chunk(a, lane, cur.k, ch)) {
            t = decode_tile(a, ch, ch.q_begin, ch.u0, lane);
        } else {
            more = false;
        }

        if (!mbar_wait_bounded(bar, phase)) {
            if (lane == 0) atomicExch(a.f.err, 1);
            mbar_wait_bounded(bar, phase);      // let the copies land before leaving
            return;
        }
        phase ^= 1u;
        __syncwarp();

        // ---- reduce: partial sums of all 32 rows (rows past the tile and
        // rows without a copy hold finite stale data and are discarded),
        // then a transpose-reduction leaves row r's sum in lane r.
        // A full tile of one vertex (most pairs live in such tiles) takes a
        // path without per-row vertex lookups or predicates.
        const bool single = (tn == 32) && (seg_starts == 1u);
        float p[32];
        if (single) {
            float o[EPL];
#pragma unroll
            for (int i = 0; i < NV; ++i)
                load_vec_smem<VEC>(own + (i * L + lane) * VEC, o + i * VEC);
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                if constexpr (kMixedSub) {
                    unsigned int w[EPL / 2];
#pragma unroll
                    for (int i = 0; i < NV; ++i)
                        load_words_smem<VEC>(reinterpret_cast<const __nv_bfloat16 *>(rows) + r * D +
                                                 (i * L + lane) * VEC,
                                             w + i * (VEC / 2));
                    p[r] = lane_dist_bf16<EPL>(o, w);
                } else {
                    float x[EPL];
#pragma unroll
                    for (int i = 0; i < NV; ++i)
                        load_vec_smem<VEC>(rows + r * D + (i * L + lane) * VEC, x + i * VEC);
                    p[r] = lane_reduce<EPL, tdist, kPackReduce>(o, x);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int j = vert[r];
                float o[EPL];
                if constexpr (kMixedSub) {
                    unsigned int w[EPL / 2];
#pragma unroll
                    for (int i = 0; i < NV; ++i) {
                        const int e0 = (i * L + lane) * VEC;
                        load_words_smem<VEC>(reinterpret_cast<const __nv_bfloat16 *>(rows) + r * D + e0,
                                             w + i * (VEC / 2));
                        load_vec_smem<VEC>(own + j * D + e0, o + i * VEC);
                    }
                    p[r] = lane_dist_bf16<EPL>(o, w);
                } else {
                    float x[EPL];
#pragma unroll
                    for (int i = 0; i < NV; ++i) {
                        const int e0 = (i * L + lane) * VEC;
                        load_vec_smem<VEC>(rows + r * D + e0, x + i * VEC);
                        load_vec_smem<VEC>(own + j * D + e0, o + i * VEC);
                    }
                    p[r] = lane_reduce<EPL, tdist, kPackReduce>(o, x);
                }
            }
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
        // ---- force: lane r turns row r's sum into its pair's scalar -------
        {
            const float sdot = p[0];
            float coef = 0.f;
            if (tkind != KIND_NONE) coef = pair_coef(model, tkind, sdot);   // Eq. 5/6, 8/9, Table "diffmodels"
            coefs[lane] = coef;              // 0 for pairs without a force
        }
        __syncwarp();

        // ---- accumulate each vertex segment; finish vertices that end -----
        const int ring_slot = cur.k % a.ring;
        const FinishCtx fc{cur.C, a.slots + (int64_t)ring_slot * a.slot_stride,
                           a.unit_cnt + (int64_t)ring_slot * a.cnt_stride, a.row_flag,
                           flag_value};
        int npub = 0;                  // this tile's rows whose flags are pending
        unsigned starts = seg_starts;
        while (starts) {
            const int rs = __ffs(starts) - 1;
            starts &= starts - 1;
            const int re = starts ? __ffs(starts) - 1 : tn;
            const int j = vert[rs];
            if (tu + j != ucur) {
                if (ucur >= 0) {
                    if (tdist) {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) g[e] = fmaf(csum, zu[e], g[e]);
                    }
                    finish_store<VEC, NV, MODEL, kGroups>(a.f, fc, lane, cur.idx, ucur, vbeg,
                                                          vend, zu, g, pend, npub, groups);
                }
                csum = 0.f;
                vbeg = (ucur >= 0) ? vend : first_lo;
                ucur = tu + j;
                vend = vends[rs];
#pragma unroll
                for (int i = 0; i < NV; ++i)
                    load_vec_smem<VEC>(own + j * D + (i * L + lane) * VEC, zu + i * VEC);
#pragma unroll
                for (int e = 0; e < EPL; ++e) g[e] = 0.f;
            }
            // two accumulators (even and odd rows of each group of four) keep
            // two independent FMA chains per element; added in a fixed order
            float g2[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) g2[e] = 0.f;
            if (single) {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const float c = coefs[r];
                    float x[EPL];
#pragma unroll
                    for (int k = 0; k < NV; ++k)
                        load_vec_smem<VEC>(rows + r * D + (k * L + lane) * VEC, x + k * VEC);
                    float *acc = (r & 1) ? g2 : g;
                    if (tdist) csum += c;
                    lane_axpy<EPL>(acc, tdist ? -c : c, x);
                }
            } else {
                for (int r0 = rs; r0 < re; r0 += 4) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = min(r0 + i, 31);
                        const float c = (r0 + i < re) ? coefs[r] : 0.f;
                        float x[EPL];
#pragma unroll
                        for (int k = 0; k < NV; ++k)
                            load_vec_smem<VEC>(rows + r * D + (k * L + lane) * VEC, x + k * VEC);
                        float *acc = (i & 1) ? g2 : g;
                        if (tdist) csum += c;
                        lane_axpy<EPL>(acc, tdist ? -c : c, x);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < EPL; ++e) g[e] += g2[e];
        }
        if (last_of_chunk) {
            // the chunk's last vertex, then the chunk counts as done
            if (tdist) {
#pragma unroll
                for (int e = 0; e < EPL; ++e) g[e] = fmaf(csum, zu[e], g[e]);
            }
            csum = 0.f;
            finish_store<VEC, NV, MODEL, kGroups>(a.f, fc, lane, cur.idx, ucur, vbeg, vend, zu,
                                                  g, pend, npub, groups);
            ucur = -1;
            chunk_start = true;
        }
        // ---- publish: one release fence for everything the tile stored ---
        if constexpr (kPublishAtTop) {
            npend = npub;
            pend_chunk = last_of_chunk;
            pend_k = cur.k;
        } else if (npub > 0 || last_of_chunk) {
            __syncwarp();
            fence_acq_rel_gpu();
            if (lane < npub) st_relaxed_gpu(&a.row_flag[pend[lane]], flag_value);
            // the chunk is done: its rows, its tree parts and any tree sums it
            // made (with their counter resets) precede the fence
            if (last_of_chunk && lane == 0)
                asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(&a.mb_done[cur.k])
                             : "memory");
        }
        __syncwarp();
        if (!more) break;
    }
    if constexpr (kPublishAtTop) publish_pending();
}

constexpr int kBulkSmemBudget = 227 * 1024;   // the most shared memory one block may take

template <int D, typename Ts>
int bulk_warps()
{
    const int w = (kBulkSmemBudget - kQueueBytes) / BulkLayout<D, Ts>::BYTES;
    // the kernel's launch bound: 16 warps at d = 64, else 12 (FP32 rows at
    // d = 128: 18.5 KB of staging per warp, 222 KB per block).  BF16 rows at
    // d = 128 would fit 16 warps, but 12 with 168 registers each measured
    // faster (fewer, longer chunks; no spills)
    const int cap = ((D <= 64) ? 512 : 384) / 32;
    return w > cap ? cap : w;
}

template <typename Ts>
bool bulk_config_t(int d, int *warps, int *smem)
{
    switch (d) {
        case 64: *warps = bulk_warps<64, Ts>(); *smem = *warps * BulkLayout<64, Ts>::BYTES + kQueueBytes; return true;
        case 128: *warps = bulk_warps<128, Ts>(); *smem = *warps * BulkLayout<128, Ts>::BYTES + kQueueBytes; return true;
        case 256: *warps = bulk_warps<256, Ts>(); *smem = *warps * BulkLayout<256, Ts>::BYTES + kQueueBytes; return true;
        default: return false;
    }
}

// Blocks of `warps` warps that fit on one SM at once (0 if none).
template <int D, typename Ts, int MODEL, bool GROUPS>
int bulk_resident_g(int warps, int smem)
{
    if (cudaFuncSetAttribute(force_bulk_kernel<D, Ts, MODEL, GROUPS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks,
                                                      force_bulk_kernel<D, Ts, MODEL, GROUPS>,
                                                      warps * 32, smem) != cudaSuccess)
        return 0;
    return blocks;
}

// Group claims are instantiated for FP32 rows only (BF16 rows measured 2-5%
// slower with them).
template <typename Ts>
constexpr bool bulk_has_groups()
{
    return sizeof(Ts) == 4;
}

template <int D, typename Ts, int MODEL>
int bulk_resident_d(int warps, int smem)
{
    int r = bulk_resident_g<D, Ts, MODEL, false>(warps, smem);
    if constexpr (bulk_has_groups<Ts>()) r = std::min(r, bulk_resident_g<D, Ts, MODEL, true>(warps, smem));
    return r;
}

template <int D, typename Ts, int MODEL, bool GROUPS>
cudaError_t launch_bulk_g(const EpochArgs<Ts> &a, const CUtensorMap &zmap, const CUtensorMap &mmap,
                          int blocks, int warps, int smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(force_bulk_kernel<D, Ts, MODEL, GROUPS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // Warps wait on rows and chunks that other blocks produce; a cooperative
    // launch places every block at once (or fails) so that no wait can be
    // on a block that has not started.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)(warps * 32));
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, force_bulk_kernel<D, Ts, MODEL, GROUPS>, a, zmap, mmap);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Group claims (FP32 rows) pay off for small chunks (R-MAT 20, b = 4096,
// 64-pair chunks: 4.26 -> 3.97 ms) and cost for large ones (one minibatch
// of the whole graph, chunks of ~9,600 pairs: 2.6 -> 3.4 ms, the last chunks
// of a block's group leaving most of its warps idle); the host sets a.groups
// from the launch's chunk sizes.
template <int D, typename Ts, int MODEL>
cudaError_t launch_bulk_d(const EpochArgs<Ts> &a, const CUtensorMap &zmap, const CUtensorMap &mmap,
                          int blocks, int warps, int smem, cudaStream_t st)
{
    if constexpr (bulk_has_groups<Ts>()) {
        if (a.groups) return launch_bulk_g<D, Ts, MODEL, true>(a, zmap, mmap, blocks, warps, smem, st);
    }
    return launch_bulk_g<D, Ts, MODEL, false>(a, zmap, mmap, blocks, warps, smem, st);
}

template <int D, typename Ts>
cudaError_t launch_bulk_m(int model, const EpochArgs<Ts> &a, const CUtensorMap &zmap,
                          const CUtensorMap &mmap, int blocks, int warps, int smem,
                          cudaStream_t st)
{
    if (model == 0) return launch_bulk_d<D, Ts, 0>(a, zmap, mmap, blocks, warps, smem, st);
    if (model == 1) return launch_bulk_d<D, Ts, 1>(a, zmap, mmap, blocks, warps, smem, st);
    return launch_bulk_d<D, Ts, kModelOther>(a, zmap, mmap, blocks, warps, smem, st);
}

template <typename Ts>
cudaError_t launch_bulk_t(int d, int model, const EpochArgs<Ts> &a, const CUtensorMap &zmap,
                          const CUtensorMap &mmap, int blocks, int warps, int smem,
                          cudaStream_t st)
{
    switch (d) {
        case 64: return launch_bulk_m<64, Ts>(model, a, zmap, mmap, blocks, warps, smem, st);
        case 128: return launch_bulk_m<128, Ts>(model, a, zmap, mmap, blocks, warps, smem, st);
        case 256: return launch_bulk_m<256, Ts>(model, a, zmap, mmap, blocks, warps, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

// Blocks per SM: the smallest of the model classes' (they differ only in code).
template <int D, typename Ts>
int bulk_resident_m(int warps, int smem)
{
    return std::min(std::min(bulk_resident_d<D, Ts, 0>(warps, smem),
                             bulk_resident_d<D, Ts, 1>(warps, smem)),
                    bulk_resident_d<D, Ts, kModelOther>(warps, smem));
}

template <typename Ts>
int bulk_resident_t(int d, int warps, int smem)
{
    switch (d) {
        case 64: return bulk_resident_m<64, Ts>(warps, smem);
        case 128: return bulk_resident_m<128, Ts>(warps, smem);
        case 256: return bulk_resident_m<256, Ts>(warps, smem);
        default: return 0;
    }
}

}  // namespace f2v
