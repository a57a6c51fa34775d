/*
 * sbm.c -- seeded stochastic-block-model graphs, many at once (input
 * generation only; nothing of the embedding method).
 *
 * Graph g has n[g] vertices in B[g] near-equal blocks (block J holds ids
 * [floor(J n / B), floor((J+1) n / B))); an undirected edge {u, v}, u < v,
 * is present with probability p_in if u and v share a block and p_out
 * otherwise, independently.  Edges are drawn row by row over the upper
 * triangle by geometric skipping (the gap to the next present pair is
 * floor(log U / log(1 - p)), U uniform in (0, 1]), so the cost is linear in
 * the number of edges.  Every graph draws from its own xoshiro256** stream
 * seeded by splitmix64 from (seed, g), so the output does not depend on how
 * graphs are spread over threads.
 *
 * The result is the symmetric CSR of every graph, rows sorted, no
 * self-loops, no duplicates, concatenated: graph g's n[g] + 1 row pointers
 * (starting at 0) follow graph g - 1's, and its column indices (local ids)
 * follow graph g - 1's.
 *
 *   h = f2v_sbm_begin(G, n, B, p_in, p_out, seed, nnz_out)   draws the edges,
 *       writes nnz_out[g] (entries of graph g's CSR, both directions);
 *   f2v_sbm_finish(h, row_ptr, col_idx)   writes the CSRs and frees h.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    int32_t *upper;      /* upper-triangle neighbours, row by row */
    int32_t *up_cnt;     /* per row */
    int64_t m;           /* upper edges */
} sbm_graph;

typedef struct {
    int32_t G;
    sbm_graph *g;
} sbm_batch;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xoshiro_next(uint64_t s[4])
{
    const uint64_t r = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return r;
}

/* uniform in (0, 1] with 53 random bits */
static double unif(uint64_t s[4]) { return ((double)(xoshiro_next(s) >> 11) + 1.0) * 0x1.0p-53; }

static int draw_graph(sbm_graph *gr, int32_t n, int32_t B, double p_in, double p_out,
                      uint64_t seed, int32_t g)
{
    uint64_t sm = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(g + 1));
    uint64_t s[4];
    for (int i = 0; i < 4; ++i) s[i] = splitmix64(&sm);
    if (B < 1) B = 1;
    if (B > n) B = n;
    gr->n = n;
    gr->m = 0;
    gr->up_cnt = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int64_t cap = 1024;
    gr->upper = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (!gr->up_cnt || !gr->upper) return -1;
    const double lq_in = (p_in > 0 && p_in < 1) ? log1p(-p_in) : 0.0;
    const double lq_out = (p_out > 0 && p_out < 1) ? log1p(-p_out) : 0.0;
    int32_t I = 0;
    for (int32_t u = 0; u < n; ++u) {
        while ((int64_t)(I + 1) * n / B <= u) ++I;
        for (int32_t J = I; J < B; ++J) {
            const int64_t start = (int64_t)J * n / B, end = (int64_t)(J + 1) * n / B;
            const int64_t lo = (u + 1 > start) ? u + 1 : start;
            if (lo >= end) continue;
            const double p = (J == I) ? p_in : p_out;
            const double lq = (J == I) ? lq_in : lq_out;
            if (p <= 0) continue;
            int64_t v = lo - 1;
            for (;;) {
                if (p >= 1) {
                    v += 1;
                } else {
                    const double gap = floor(log(unif(s)) / lq);
                    if (gap >= (double)(end - v)) break;
                    v += 1 + (int64_t)gap;
                }
                if (v >= end) break;
                if (gr->m == cap) {
                    cap *= 2;
                    int32_t *nu = (int32_t *)realloc(gr->upper, (size_t)cap * sizeof(int32_t));
                    if (!nu) return -1;
                    gr->upper = nu;
                }
                gr->upper[gr->m++] = (int32_t)v;
                gr->up_cnt[u] += 1;
            }
        }
    }
    return 0;
}

void *f2v_sbm_begin(int32_t G, const int32_t *n, const int32_t *B, double p_in, double p_out,
                    uint64_t seed, int64_t *nnz_out)
{
    sbm_batch *h = (sbm_batch *)calloc(1, sizeof(sbm_batch));
    if (!h) return NULL;
    h->G = G;
    h->g = (sbm_graph *)calloc((size_t)G, sizeof(sbm_graph));
    if (!h->g) {
        free(h);
        return NULL;
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t g = 0; g < G; ++g) {
        if (draw_graph(&h->g[g], n[g], B[g], p_in, p_out, seed, g) != 0) bad |= 1;
        nnz_out[g] = 2 * h->g[g].m;
    }
    if (bad) {
        for (int32_t g = 0; g < G; ++g) {
            free(h->g[g].upper);
            free(h->g[g].up_cnt);
        }
        free(h->g);
        free(h);
        return NULL;
    }
    return h;
}

void f2v_sbm_finish(void *handle, int32_t *row_ptr, int32_t *col_idx)
{
    sbm_batch *h = (sbm_batch *)handle;
    const int32_t G = h->G;
    int64_t *roff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)G + 1));
    int64_t *coff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)G + 1));
    roff[0] = 0;
    coff[0] = 0;
    for (int32_t g = 0; g < G; ++g) {
        roff[g + 1] = roff[g] + h->g[g].n + 1;
        coff[g + 1] = coff[g] + 2 * h->g[g].m;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t g = 0; g < G; ++g) {
        sbm_graph *gr = &h->g[g];
        const int32_t n = gr->n;
        int32_t *rp = row_ptr + roff[g];
        int32_t *ci = col_idx + coff[g];
        /* degree = upper count + lower count */
        memset(rp, 0, sizeof(int32_t) * ((size_t)n + 1));
        for (int32_t u = 0; u < n; ++u) rp[u + 1] += gr->up_cnt[u];
        for (int64_t e = 0; e < gr->m; ++e) rp[gr->upper[e] + 1] += 1;
        for (int32_t u = 0; u < n; ++u) rp[u + 1] += rp[u];
        int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        memcpy(pos, rp, sizeof(int32_t) * (size_t)n);
        /* rows in ascending u: row u already holds its lower neighbours
           (appended while earlier rows were walked), then gets its upper
           ones; each upper neighbour v gets u appended, in ascending u */
        int64_t e = 0;
        for (int32_t u = 0; u < n; ++u) {
            for (int32_t k = 0; k < gr->up_cnt[u]; ++k, ++e) {
                const int32_t v = gr->upper[e];
                ci[pos[u]++] = v;
                ci[pos[v]++] = u;
            }
        }
        free(pos);
        free(gr->upper);
        free(gr->up_cnt);
    }
    free(roff);
    free(coff);
    free(h->g);
    free(h);
}
