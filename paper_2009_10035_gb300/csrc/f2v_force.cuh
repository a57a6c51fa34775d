// f2v_force.cuh -- the fused SDDMM + SpMM force kernel and SGD update of one
// minibatch (Algorithm 2 followed by the update step of Algorithm 1, Eq. 10).
//
// Work decomposition.  The minibatch's force pairs (neighbours of each u in
// CSR order, then its s negative samples) form one flat sequence; it is cut
// into items of C pairs, so every group of lanes gets the same amount of
// gathering regardless of degree skew (the degree-balanced partition of
// Sec. III-D, at pair granularity).  A group of L lanes walks its item in
// tiles of L pairs:
//   1. decode -- lane t finds the vertex and the partner of pair t of the
//      tile from a window of L consecutive vertices (pair prefix, row
//      pointers), reading the partner from col_idx (attractive) or drawing it
//      with Philox (repulsive), or, in the rForce2Vec form, reading its code
//      from the epoch's expanded partner list;
//   2. gather -- the group fetches the partner rows, U at a time, each lane
//      a VEC-wide vector of NV slices (128-bit loads for FP32 rows of d >= 4);
//   3. force -- the dot product (sigmoid) or squared distance (the other
//      models) is reduced with xor shuffles inside the group, turned into the
//      scalar of Eq. 5/6, Eq. 8/9 or Table "diffmodels" (pair_coef), and the
//      scaled row is accumulated in FP32 registers (the SpMM half);
//   4. update -- when a vertex's pairs end, z_u - eta * g is written to the
//      next buffer, directly if the item held all its pairs, else through the
//      ordered combine tree described in f2v_internal.h.
// Pair positions inside a launch are 32-bit offsets from the minibatch's
// first pair.  The own row of the next vertex is fetched while the current
// one is being summed, since vertices of an item are consecutive ids.
#pragma once

#include <climits>

#include "f2v_device.cuh"
#include "f2v_internal.h"

namespace f2v {

constexpr int kBlock = 256;
constexpr int KIND_NONE = 0;   // no force (self sample, or the empty pair)
constexpr int KIND_ATTR = 1;   // neighbour: attractive force
constexpr int KIND_REP = 2;    // negative sample: repulsive force
constexpr float kT2Floor = 1e-8f;
constexpr float kSigmoidBound = 4.f;

// Force models (f2v_model): 0 t-distribution, 1 sigmoid, 2 Fruchterman-
// Reingold, 3 LinLog, 4 ForceAtlas.  Kernels are instantiated per model
// class: MODEL = 0 (t), 1 (sigmoid), 2 (FR, LinLog or ForceAtlas, chosen by
// ForceArgs::model at run time; they share every loop and differ only in the
// attraction scalar), or -1 (everything read at run time).
constexpr int kModelOther = 2;

// The model a kernel instantiation computes.
template <int MODEL>
__device__ __forceinline__ int model_of(int rt_model)
{
    return (MODEL == 0 || MODEL == 1) ? MODEL : rt_model;
}

// Force scalar c of one pair from its reduced scalar r: the dot product
// z_u . z_x for the sigmoid model (term c z_x), the squared distance
// q = |z_u - z_x|^2 for the others (term c (z_u - z_x)):
//   t model, Eq. 8/9 times the unit vector:      2/(1+q),  -2/(q(1+q))
//   FR, LinLog, ForceAtlas, minus the force of Table "diffmodels" times the
//   unit vector:  t = sqrt(q), log(1+t)/t, 1;    -1/q
// (q floored at 1e-8 in the repulsive terms).
__device__ __forceinline__ float pair_coef(int model, int kind, float r)
{
    if (model == 1)
        return (kind == KIND_ATTR) ? -1.f / (1.f + expf(r))     // Eq. 5
                                   : 1.f / (1.f + expf(-r));    // Eq. 6
    if (kind == KIND_ATTR) {
        if (model == 0) return 2.f / (1.f + r);                  // Eq. 8 / t
        const float t = sqrtf(r);
        if (model == 2) return t;                                // FR: t^2 / t
        if (model == 3) return t > 0.f ? log1pf(t) / t : 1.f;    // LinLog
        return 1.f;                                              // ForceAtlas: t / t
    }
    const float q2 = fmaxf(r, kT2Floor);
    return (model == 0) ? -2.f / (q2 * (1.f + q2))               // Eq. 9 / t
                        : -1.f / q2;                             // (1/t) / t
}

template <int L, int VEC, int NV>
struct ShapeTraits {
    static constexpr int E = VEC * NV;                       // elements per lane
    static constexpr int U0 = (32 / E) < 1 ? 1 : (32 / E);  // rows in flight
    static constexpr int U1 = U0 > 8 ? 8 : U0;
    static constexpr int U = U1 > L ? L : U1;
};

// Element index of lane `gl`'s slot (i, c).
template <int L, int VEC>
__device__ __forceinline__ int elem_index(int gl, int i, int c)
{
    return (i * L + gl) * VEC + c;
}

template <int L, int VEC, int NV, bool EXACT, typename Ts>
__device__ __forceinline__ void load_row(const Ts *row, int gl, int d, float *x)
{
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e0 = elem_index<L, VEC>(gl, i, 0);
        if (EXACT || e0 < d) {
            load_vec<VEC>(row + e0, x + i * VEC);
        } else {
#pragma unroll
            for (int c = 0; c < VEC; ++c) x[i * VEC + c] = 0.f;
        }
    }
}

template <int L, int VEC, int NV, bool EXACT, typename Ts>
__device__ __forceinline__ void load_row_cg(const Ts *row, int gl, int d, float *x)
{
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e0 = elem_index<L, VEC>(gl, i, 0);
        if (EXACT || e0 < d) {
            load_vec_cg<VEC>(row + e0, x + i * VEC);
        } else {
#pragma unroll
            for (int c = 0; c < VEC; ++c) x[i * VEC + c] = 0.f;
        }
    }
}

template <int L, int VEC, int NV, bool EXACT>
__device__ __forceinline__ void store_row_cg(float *row, int gl, int d, const float *x)
{
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e0 = elem_index<L, VEC>(gl, i, 0);
        if (EXACT || e0 < d) store_vec_cg<VEC>(row + e0, x + i * VEC);
    }
}

// Own row of u: the FP32 master in the BF16 form, else the current buffer.
template <int L, int VEC, int NV, bool EXACT, typename Ts>
__device__ __forceinline__ void load_own_row(const ForceArgs<Ts> &a, int u, int gl, float *x)
{
    if constexpr (sizeof(Ts) == 2)
        load_row_cg<L, VEC, NV, EXACT>(a.master + (int64_t)u * a.ld, gl, a.d, x);
    else
        load_row<L, VEC, NV, EXACT>(a.zcur + (int64_t)u * a.ld, gl, a.d, x);
}

// Where a finished vertex's partial sums and row go, for one minibatch.
struct FinishCtx {
    int C;                     // pairs per level-0 unit (item or chunk)
    float *slots;              // combine-tree slots of this minibatch
    int32_t *unit_cnt;         // combine-tree counters of this minibatch
    int32_t *row_flag;         // if not null: row_flag[u] = flag_value once row u is written
    int32_t flag_value;
};

// Marks row u as written.  The group's lanes stored the row; the warp
// barrier orders their stores before lane 0's release store of the flag,
// and release is cumulative, so a reader that acquires the flag sees the
// whole row.  (A reader that then reads the row through the async proxy
// issues the proxy fence itself.)
__device__ __forceinline__ void publish_row(int32_t *flag, int u, int32_t value, unsigned gmask,
                                            int gl)
{
    __syncwarp(gmask);
    if (gl == 0)
        asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flag + u), "r"(value)
                     : "memory");
}

// z_u <- z_u - eta * g (Eq. 10) into the next buffer (and the master).
// MODEL: the force model when the caller fixes it at compile time (0 t,
// 1 sigmoid), else -1 (read from a.model).
template <int L, int VEC, int NV, bool EXACT, int MODEL = -1, typename Ts>
__device__ __forceinline__ void write_row(const ForceArgs<Ts> &a, const FinishCtx &fc,
                                          unsigned gmask, int u, int gl, const float *zu,
                                          const float *g)
{
    constexpr int E = VEC * NV;
    float z[E];
#pragma unroll
    for (int e = 0; e < E; ++e) z[e] = fmaf(-a.eta, g[e], zu[e]);
    // every model but t: coordinates bounded to [-4, 4] (their forces do
    // not vanish with distance; without a bound the summed gradients of a
    // high-degree vertex make Alg. 1 diverge)
    if (MODEL > 0 || (MODEL < 0 && a.model != 0)) {
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = fminf(fmaxf(z[e], -kSigmoidBound), kSigmoidBound);
    }
    Ts *dst = a.znext + (int64_t)u * a.ld;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e0 = elem_index<L, VEC>(gl, i, 0);
        if (EXACT || e0 < a.d) {
            store_vec<VEC>(dst + e0, z + i * VEC);
            if constexpr (sizeof(Ts) == 2)
                store_vec<VEC>(a.master + (int64_t)u * a.ld + e0, z + i * VEC);
        }
    }
    if (fc.row_flag) publish_row(fc.row_flag, u, fc.flag_value, gmask, gl);
}

// Slot of vertex u (pairs [lb, le) of the minibatch) in level-`lvl` unit j:
// 2j if u holds the unit's first pair, else 2j+1 (u then holds its last).
__device__ __forceinline__ int64_t unit_slot(int64_t j, int lb, int64_t unit_pairs)
{
    return ((int64_t)lb <= j * unit_pairs) ? 2 * j : 2 * j + 1;
}

// Finishes vertex u, whose local pairs are [vbeg, vend) and whose pairs in
// level-0 unit `unit0` are summed in g: writes z_u - eta * g if the unit held
// all of them, else passes the part up the ordered combine tree (g is
// clobbered).
template <int L, int VEC, int NV, bool EXACT, int MODEL = -1, typename Ts>
__device__ __forceinline__ void finish_vertex(const ForceArgs<Ts> &a, const FinishCtx &fc,
                                              unsigned gmask, int gl, int unit0, int u, int vbeg,
                                              int vend, const float *zu, float *g)
{
    constexpr int E = VEC * NV;
    int64_t fu = vbeg / fc.C, lu = (vend - 1) / fc.C;
    if (fu == lu) {
        write_row<L, VEC, NV, EXACT, MODEL>(a, fc, gmask, u, gl, zu, g);
        return;
    }
    int64_t unit = unit0, unit_pairs = fc.C, units = a.units0;
    float *slot_base = fc.slots;
    int32_t *cnt_base = fc.unit_cnt;
    for (int lvl = 0; lvl + 1 < kMaxLevels; ++lvl) {
        store_row_cg<L, VEC, NV, EXACT>(slot_base + unit_slot(unit, vbeg, unit_pairs) * a.ld,
                                        gl, a.d, g);
        const int64_t parent = unit / kFan;
        const int64_t pfu = fu / kFan, plu = lu / kFan;
        const int64_t c0 = max(fu, parent * kFan);
        const int64_t c1 = min(lu, parent * kFan + (kFan - 1));
        const bool top = (pfu == plu);
        const int64_t punits = (units + kFan - 1) / kFan;
        int32_t *cnt = top ? &a.counter[u]
                           : &cnt_base[unit_slot(parent, vbeg, unit_pairs * kFan)];
        // arrive: the group's slot stores, ordered by the warp barrier, are
        // released by lane 0's acq_rel increment; the last arrival acquires
        // every sibling's release through the same counter
        __syncwarp(gmask);
        int prior = 0;
        if (gl == 0)
            asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;"
                         : "=r"(prior)
                         : "l"(cnt)
                         : "memory");
        prior = __shfl_sync(gmask, prior, 0, L);
        if (prior != (int)(c1 - c0)) return;      // a sibling completes it
        __syncwarp(gmask);                         // the other lanes read after the acquire
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = 0.f;
        for (int64_t c = c0; c <= c1; c += 4) {    // children in order
            float part[4][E];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c + k <= c1)
                    load_row_cg<L, VEC, NV, EXACT>(
                        slot_base + unit_slot(c + k, vbeg, unit_pairs) * a.ld, gl, a.d, part[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c + k <= c1) {
#pragma unroll
                    for (int e = 0; e < E; ++e) g[e] += part[k][e];
                }
        }
        if (gl == 0) *cnt = 0;
        if (top) {
            write_row<L, VEC, NV, EXACT, MODEL>(a, fc, gmask, u, gl, zu, g);
            return;
        }
        slot_base += 2 * units * a.ld;
        cnt_base += 2 * punits;
        unit = parent;
        fu = pfu;
        lu = plu;
        units = punits;
        unit_pairs *= kFan;
    }
}

// A pair's partner from its code in an expanded partner list (rForce2Vec);
// a code without a force leaves nb and kind as they are (kind KIND_NONE).
__device__ __forceinline__ void decode_code(int code, int &nb, int &kind)
{
    if (code >= 0) {
        nb = code;
        kind = KIND_ATTR;
    } else if (code != kPartnerNone) {
        nb = -2 - code;
        kind = KIND_REP;
    }
}

// Partner row v: from the next buffer if an earlier minibatch of this epoch
// wrote it, else from the current one.  Rows written earlier in the same
// launch (COHERENT: the batched kernel) are read through L2 only, since L1 is
// not coherent with other SMs' stores; rows of earlier launches may take the
// read-only path.
template <int L, int VEC, int NV, bool EXACT, bool COHERENT, typename Ts>
__device__ __forceinline__ void load_partner(const ForceArgs<Ts> &a, int v, int gl, float *x)
{
    if (v < a.mb_begin) {
        if constexpr (COHERENT)
            load_row_cg<L, VEC, NV, EXACT>(a.znext + (int64_t)v * a.ld, gl, a.d, x);
        else
            load_row<L, VEC, NV, EXACT>(a.znext + (int64_t)v * a.ld, gl, a.d, x);
    } else {
        load_row<L, VEC, NV, EXACT>(a.zcur + (int64_t)v * a.ld, gl, a.d, x);
    }
}

// One item walked by a single lane (rows of d <= 4 elements).  A lane has no
// partners to share a row with, so instead of one pair per step it takes up
// to T pairs of the current vertex at once: their partner codes (column
// indices or Philox draws) and then their rows are all in flight together.
// The gradient adds the pairs in order, as the group walk does.
template <int VEC, int NV, bool EXACT, bool COHERENT, int MODEL, typename Ts>
__device__ __forceinline__ void force_item_lane(const ForceArgs<Ts> &a, const FinishCtx &fc,
                                                int item, unsigned gmask)
{
    constexpr int E = VEC * NV;
    constexpr int T = 8;
    const int model = model_of<MODEL>(a.model);
    const bool dist = (model != 1);       // squared distance, else dot product
    const int q_begin = item * a.C;
    const int q_end = min(q_begin + a.C, a.Pk);
    int u = __ldg(&a.item_u0[item]);
    float zu[E], g[E];
    load_own_row<1, VEC, NV, EXACT>(a, u, 0, zu);
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = 0.f;
    int vbeg = (int)(__ldg(&a.apair[u]) - a.P0);
    int vend = (int)(__ldg(&a.apair[u + 1]) - a.P0);
    int rp_lo = __ldg(&a.row_ptr[u]);
    int deg = __ldg(&a.row_ptr[u + 1]) - rp_lo;
    int q = q_begin;
    while (true) {
        // pairs q .. q + n - 1, all of vertex u
        const int n = min(T, min(vend, q_end) - q);
        int nb[T], kd[T];
#pragma unroll
        for (int i = 0; i < T; ++i) {
            nb[i] = u;
            kd[i] = KIND_NONE;
            if (i < n && a.partner) {
                decode_code(__ldg(&a.partner[a.P0 + q + i]), nb[i], kd[i]);
            } else if (i < n) {
                const int j = q + i - vbeg;
                if (j < deg) {
                    nb[i] = __ldg(&a.col_idx[rp_lo + j]);
                    kd[i] = KIND_ATTR;
                } else if (j - deg < a.s) {
                    const uint32_t x0 = philox_x0((uint32_t)u, a.epoch, (uint32_t)(j - deg), 0u,
                                                  a.key0, a.key1);
                    nb[i] = (int)(x0 % (uint32_t)a.n);
                    kd[i] = (nb[i] == u) ? KIND_NONE : KIND_REP;
                }
            }
        }
        float zv[T][E];
#pragma unroll
        for (int i = 0; i < T; ++i)
            if (kd[i] != KIND_NONE) load_partner<1, VEC, NV, EXACT, COHERENT>(a, nb[i], 0, zv[i]);
#pragma unroll
        for (int i = 0; i < T; ++i) {
            if (kd[i] == KIND_NONE) continue;
            float part = 0.f;
            if (dist) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const float df = zu[e] - zv[i][e];
                    part = fmaf(df, df, part);
                }
                const float coef = pair_coef(model, kd[i], part);
#pragma unroll
                for (int e = 0; e < E; ++e) g[e] = fmaf(coef, zu[e] - zv[i][e], g[e]);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) part = fmaf(zu[e], zv[i][e], part);
                const float coef = pair_coef(1, kd[i], part);
#pragma unroll
                for (int e = 0; e < E; ++e) g[e] = fmaf(coef, zv[i][e], g[e]);
            }
        }
        q += n;
        if (q < vend && q < q_end) continue;
        // the vertex's pairs in this item end here
        finish_vertex<1, VEC, NV, EXACT, MODEL>(a, fc, gmask, 0, item, u, vbeg, vend, zu, g);
        if (q >= q_end) break;
        ++u;
        load_own_row<1, VEC, NV, EXACT>(a, u, 0, zu);
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = 0.f;
        vbeg = vend;
        vend = (int)(__ldg(&a.apair[u + 1]) - a.P0);
        rp_lo = __ldg(&a.row_ptr[u]);
        deg = __ldg(&a.row_ptr[u + 1]) - rp_lo;
    }
}

// One item (C consecutive pairs of the minibatch) walked by a group of L
// lanes: lane gl of the group, gmask the group's lanes; U partner rows in
// flight at a time.
template <int L, int VEC, int NV, bool EXACT, bool COHERENT, int MODEL = -1,
          int U = ShapeTraits<L, VEC, NV>::U, typename Ts>
__device__ __forceinline__ void force_item(const ForceArgs<Ts> &a, const FinishCtx &fc, int item,
                                           int gl, unsigned gmask)
{
    constexpr int E = VEC * NV;
    if constexpr (L == 1) {
        force_item_lane<VEC, NV, EXACT, COHERENT, MODEL>(a, fc, item, gmask);
        return;
    }
    // the force model: fixed per instantiation when MODEL is 0 or 1
    const int model = model_of<MODEL>(a.model);
    const bool dist = (model != 1);       // squared distance, else dot product
    const int q_begin = item * a.C;
    const int q_end = min(q_begin + a.C, a.Pk);
    int u = __ldg(&a.item_u0[item]);       // vertex holding pair q_begin

    // own rows: the item's first vertex now, the next one ahead of need
    int ucur = u;
    float zu[E], zn[E], g[E];
    load_own_row<L, VEC, NV, EXACT>(a, ucur, gl, zu);
    if (ucur + 1 < a.mb_end) load_own_row<L, VEC, NV, EXACT>(a, ucur + 1, gl, zn);
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = 0.f;
    int vbeg = 0, vend = 0;

    // decoded tile (lane gl <-> pair q + gl)
    int q = q_begin - L;
    int r = 0, ntile = 0, next_u = u;
    int pu = u, nb = u, kind = KIND_NONE, pA_hi = 0;
    for (;;) {
        if (r == ntile) {
            // ---- 1. decode the next tile -------------------------------
            q += L;
            u = next_u;
            if (q < q_end) {
                const int uu = u + gl;
                int A_hi = INT_MAX;
                int rp_lo = 0, rp_hi = 0;
                if (uu < a.n) {
                    const int64_t ah = __ldg(&a.apair[uu + 1]) - a.P0;
                    A_hi = ah > INT_MAX ? INT_MAX : (int)ah;
                    rp_lo = __ldg(&a.row_ptr[uu]);
                    rp_hi = __ldg(&a.row_ptr[uu + 1]);
                }
                const int A_up = __shfl_up_sync(gmask, A_hi, 1, L);
                const int A_lo = (gl == 0) ? (int)(__ldg(&a.apair[u]) - a.P0) : A_up;
                const int pos = A_hi - q;             // >= 1: vertex uu ends after q
                const unsigned bit = (pos < L) ? (1u << pos) : 0u;
                const unsigned ends = __reduce_or_sync(gmask, bit);
                const int off = __popc(ends & ((2u << gl) - 1u));
                pu = u + off;                         // vertex of this lane's pair
                const int pA_lo = __shfl_sync(gmask, A_lo, off, L);
                pA_hi = __shfl_sync(gmask, A_hi, off, L);
                const int prp_lo = __shfl_sync(gmask, rp_lo, off, L);
                const int prp_hi = __shfl_sync(gmask, rp_hi, off, L);
                nb = pu;
                kind = KIND_NONE;
                if (q + gl < q_end && a.partner) {
                    decode_code(__ldg(&a.partner[a.P0 + q + gl]), nb, kind);
                } else if (q + gl < q_end) {
                    const int j = q + gl - pA_lo;
                    const int deg = prp_hi - prp_lo;
                    if (j < deg) {
                        nb = __ldg(&a.col_idx[prp_lo + j]);
                        kind = KIND_ATTR;
                    } else if (j - deg < a.s) {
                        const uint32_t x0 = philox_x0((uint32_t)pu, a.epoch,
                                                      (uint32_t)(j - deg), 0u, a.key0, a.key1);
                        nb = (int)(x0 % (uint32_t)a.n);
                        kind = (nb == pu) ? KIND_NONE : KIND_REP;
                    }
                }
                if (q == q_begin) {
                    vbeg = __shfl_sync(gmask, A_lo, 0, L);
                    vend = __shfl_sync(gmask, A_hi, 0, L);
                }
                next_u = u + __popc(__ballot_sync(gmask, pos <= L) & gmask);
                ntile = min(L, q_end - q);
                r = 0;
            }
        }
        // vertex of the next pair; -1 once the item is done
        const int w = (q < q_end) ? __shfl_sync(gmask, pu, r, L) : -1;
        if (w != ucur) {
            // ---- 4. update: the only place a vertex is finished ------
            finish_vertex<L, VEC, NV, EXACT, MODEL>(a, fc, gmask, gl, item, ucur, vbeg, vend, zu,
                                                    g);
            if (w < 0) break;
            // next vertex: always ucur + 1, its own row already fetched
            ucur = w;
            vbeg = vend;
            vend = __shfl_sync(gmask, pA_hi, r, L);
#pragma unroll
            for (int e = 0; e < E; ++e) { zu[e] = zn[e]; g[e] = 0.f; }
            if (ucur + 1 < a.mb_end && vend < q_end)
                load_own_row<L, VEC, NV, EXACT>(a, ucur + 1, gl, zn);
        }
        // ---- 2-3. gather and accumulate this vertex's pairs of the tile
        const int seg_end = min(ntile, vend - q);
        for (int r0 = r; r0 < seg_end; r0 += U) {
            float zv[U][E];
            int kr[U];
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const int ri = min(r0 + i, L - 1);
                const int v = __shfl_sync(gmask, nb, ri, L);
                kr[i] = __shfl_sync(gmask, kind, ri, L);
                if (r0 + i >= seg_end) kr[i] = KIND_NONE;
                if (kr[i] != KIND_NONE)
                    load_partner<L, VEC, NV, EXACT, COHERENT>(a, v, gl, zv[i]);
            }
            // the U rows in phases, so that their independent work overlaps:
            // partial sums, the group reductions level by level, the force
            // scalars; then the accumulation, in row order
            float part[U];
#pragma unroll
            for (int i = 0; i < U; ++i) {
                part[i] = 0.f;
                if (dist) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const float df = zu[e] - zv[i][e];
                        part[i] = fmaf(df, df, part[i]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) part[i] = fmaf(zu[e], zv[i][e], part[i]);
                }
            }
#pragma unroll
            for (int m = L / 2; m >= 1; m >>= 1) {
#pragma unroll
                for (int i = 0; i < U; ++i) part[i] += __shfl_xor_sync(gmask, part[i], m, L);
            }
            // lane i of the group turns row i's sum into its scalar once (after
            // the butterfly every lane holds the same sum, bit for bit) and the
            // group shares the U scalars
            float my_part = part[0];
            int my_kind = kr[0];
#pragma unroll
            for (int i = 1; i < U; ++i)
                if (gl == i) {
                    my_part = part[i];
                    my_kind = kr[i];
                }
            const float my_coef = (my_kind != KIND_NONE) ? pair_coef(model, my_kind, my_part) : 0.f;
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const float coef = __shfl_sync(gmask, my_coef, i, L);
                if (kr[i] == KIND_NONE) continue;     // (its row was not loaded)
                if (dist) {
#pragma unroll
                    for (int e = 0; e < E; ++e) g[e] = fmaf(coef, zu[e] - zv[i][e], g[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) g[e] = fmaf(coef, zv[i][e], g[e]);
                }
            }
        }
        r = seg_end;
    }
}

template <int L, int VEC, int NV, bool EXACT, int MODEL, typename Ts>
__global__ void __launch_bounds__(kBlock) force_kernel(const ForceArgs<Ts> a)
{
    constexpr int G = 32 / L;
    static_assert(L >= 1 && L <= 32 && (L & (L - 1)) == 0, "L must be a power of two");

    const int lane = threadIdx.x & 31;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (grp * L));
    const int warps = blockDim.x >> 5;
    const int gid = (blockIdx.x * warps + (threadIdx.x >> 5)) * G + grp;
    const int ngroups = gridDim.x * warps * G;
    const FinishCtx fc{a.C, a.slots, a.unit_cnt, nullptr, 0};
    for (int item = gid; item < a.n_items; item += ngroups)
        force_item<L, VEC, NV, EXACT, false, MODEL>(a, fc, item, gl, gmask);
}

template <int L, int VEC, int NV, bool EXACT, typename Ts>
cudaError_t launch_shape(const ForceArgs<Ts> &a, int blocks_cap, cudaStream_t st)
{
    constexpr int G = 32 / L;
    const int64_t groups_per_block = (kBlock / 32) * G;
    int64_t blocks = (a.n_items + groups_per_block - 1) / groups_per_block;
    if (blocks_cap > 0 && blocks > blocks_cap) blocks = blocks_cap;
    if (blocks < 1) blocks = 1;
    if (a.model == 0)
        force_kernel<L, VEC, NV, EXACT, 0, Ts><<<(unsigned)blocks, kBlock, 0, st>>>(a);
    else if (a.model == 1)
        force_kernel<L, VEC, NV, EXACT, 1, Ts><<<(unsigned)blocks, kBlock, 0, st>>>(a);
    else
        force_kernel<L, VEC, NV, EXACT, kModelOther, Ts><<<(unsigned)blocks, kBlock, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename Ts>
cudaError_t launch_force_any(const Shape &sh, const ForceArgs<Ts> &a, int blocks_cap,
                             cudaStream_t st)
{
    if (sh.exact) {
        switch (sh.L * 100 + sh.VEC * 10 + sh.NV) {
            case 121: return launch_shape<1, 2, 1, true>(a, blocks_cap, st);
            case 141: return launch_shape<1, 4, 1, true>(a, blocks_cap, st);
            case 241: return launch_shape<2, 4, 1, true>(a, blocks_cap, st);
            case 441: return launch_shape<4, 4, 1, true>(a, blocks_cap, st);
            case 841: return launch_shape<8, 4, 1, true>(a, blocks_cap, st);
            case 1641: return launch_shape<16, 4, 1, true>(a, blocks_cap, st);
            case 3241: return launch_shape<32, 4, 1, true>(a, blocks_cap, st);
            case 3242: return launch_shape<32, 4, 2, true>(a, blocks_cap, st);
            case 3244: return launch_shape<32, 4, 4, true>(a, blocks_cap, st);
            case 3248: return launch_shape<32, 4, 8, true>(a, blocks_cap, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sh.NV) {
        case 1: return launch_shape<32, 1, 1, false>(a, blocks_cap, st);
        case 2: return launch_shape<32, 1, 2, false>(a, blocks_cap, st);
        case 4: return launch_shape<32, 1, 4, false>(a, blocks_cap, st);
        case 8: return launch_shape<32, 1, 8, false>(a, blocks_cap, st);
        case 16: return launch_shape<32, 1, 16, false>(a, blocks_cap, st);
        case 32: return launch_shape<32, 1, 32, false>(a, blocks_cap, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace f2v
