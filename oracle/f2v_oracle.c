/*
 * f2v_oracle.c -- plain FP64 CPU oracle for Force2Vec's minibatch force
 * computation and SGD update (Rahman, Sujon, Azad, "Force2Vec: Parallel
 * force-directed graph embedding", arXiv:2009.10035).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header or constant table with the CUDA library; the two meet only at
 * the seeded graphs the tests hand to both.
 *
 * What each function follows:
 *   orc_philox4x32_10   Philox4x32-10, the published counter-based generator
 *                       (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
 *                       two-multiply S-box with a Weyl key schedule.
 *   orc_init_value      random initial embedding (Sec. III-C, "Initialization
 *                       and hyper parameters"), uniform in [-0.5, 0.5).
 *   orc_sample          uniform negative sample for vertex u (Sec. III-C,
 *                       negative sampling; one set of s samples per vertex as
 *                       in the complexity paragraph of Sec. III-C).
 *   orc_sample_shared   Alg. 1's sampling step read literally: one set S_b of s
 *                       samples per minibatch, used by every vertex of it
 *                       (Sec. III-C, the paragraph after Alg. 1).
 *   attractive_grad,    per-pair gradients: sigmoid model Eq. 5 / Eq. 6,
 *   repulsive_grad      t-distribution model Eq. 8 / Eq. 9, each times the
 *                       unit vector of Sec. III-B for the t model; the
 *                       Fruchterman-Reingold, LinLog and ForceAtlas models
 *                       of Table "diffmodels" (Sec. III-A, "Other
 *                       force-directed models"), also along the unit vector.
 *   orc_grad_minibatch  Algorithm 2 (GradMinibatch).
 *   orc_walk            Algorithm 3 (GenWalk): the random-walk neighbourhood
 *                       of rForce2Vec (Sec. III-C, its rForce2Vec paragraph).
 *   orc_train           Algorithm 1 with the update of Eq. 10.
 *   orc_loss_vertex     Eq. 2 with delta from Eq. 3 (sigmoid) or Eq. 7 (t).
 *   orc_auc             Mann-Whitney AUC of held-out edges (evaluation).
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *   - Synchronous minibatch SGD (Sec. III-B): every gradient of a minibatch is
 *     computed from Z as it stood when the minibatch began; the minibatch's
 *     rows are then updated; the next minibatch sees those updates.
 *   - Minibatch k holds vertex ids [k*b, min((k+1)*b, n)) in id order; or,
 *     as an option, the positions [k*b, min((k+1)*b, n)) of a random
 *     permutation drawn anew each epoch (the partition step of Alg. 1: random
 *     minibatches, no vertex in two of them): vertices sorted by Philox(key, ctr=(v, e, 0, 3)).x0,
 *     ties by id (orc_partition).  Shared samples then belong to the
 *     minibatch index k.
 *   - Only z_u for u in the minibatch is updated (the update step of Algorithm 1).
 *   - Negative sample k of vertex u in epoch e is
 *       w = Philox(key=(seed lo, seed hi), ctr=(u, e, k, 0)).x0 mod n,
 *     with no neighbour rejection; w == u contributes nothing.
 *   - Z0[i][j] = (Philox(key, ctr=(i, j, 0xFFFF, 0)).x0 >> 8) * 2^-24 - 0.5,
 *     exact in FP32 and FP64.  Sample counters use ctr[2] = k < s <= 0xFFFE,
 *     so the two streams never meet.
 *   - t model: t^2 is clamped to at least 1e-8 in the repulsive term only.
 *   - Learning-rate schedule: constant, or eta_e = eta0 * (1 - e/E) for a
 *     linearly decayed run of E epochs.
 *   - rForce2Vec (Alg. 3): N(u) is the sequence of the k vertices a walk of
 *     k steps from u reaches, repeats included, one attractive pair each (the
 *     paper's O(nkd) attractive cost; read as a set, the loop of Alg. 3
 *     would not end on a component of fewer than k + 1 vertices).  Step i
 *     (0-based) of the walk from u in epoch e moves from w to
 *       col_idx[row_ptr[w] + Philox(key, ctr=(u, e, i, 1)).x0 mod deg(w)].
 *     A step that lands on u adds no force (as a sample equal to u); a walk
 *     that reaches a vertex without out-neighbours (only in a CSR that is not
 *     symmetric) stops there; a vertex without neighbours has no walk.  The
 *     walk's pairs come first, then the s negative samples.
 *   - Table "diffmodels" (FR, LinLog, ForceAtlas) lists each model's force
 *     on u along the unit vector (z_u - z_x)/t, t = |z_u - z_x|: negative
 *     for the attraction toward a neighbour, positive for the repulsion
 *     from a sample.  Eq. 10 steps against the gradient, so the per-pair
 *     gradient is minus that force times the unit vector:
 *       FR         attractive  t^2 (z_u - z_v)/t = t (z_u - z_v)
 *       LinLog     attractive  log(1 + t) (z_u - z_v)/t
 *       ForceAtlas attractive  (z_u - z_v)
 *       all three  repulsive   -(1/t) (z_u - z_w)/t = -(z_u - z_w)/t^2,
 *     with t^2 floored at 1e-8 as in the t model.  (Read as gradients, the
 *     listed signs would push neighbours apart and pull samples together.)
 *     Their forces grow (FR, LinLog, ForceAtlas attraction) or stay finite
 *     with distance, so like the sigmoid model they take the coordinate
 *     bound below.
 *   - Shared samples (Alg. 1's sampling step read literally, an option): sample j of
 *     minibatch k in epoch e is Philox(key, ctr=(k, e, j, 2)).x0 mod n for
 *     every vertex of the minibatch; a sample equal to u adds no force.
 *   - Sigmoid (and FR, LinLog, ForceAtlas) models: after each update every
 *     coordinate of z_u is clamped to
 *     [-4, 4].  The paper is silent on divergence; without a bound, Alg. 1 at
 *     eta = 0.02 with the summed gradients of Alg. 2 diverges on graphs with
 *     high-degree vertices even in FP64 (max |z| grows ~1e5-fold per epoch on
 *     an R-MAT scale-20 graph), leaving FP32's range after seven epochs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TDIST 0
#define ORC_SIGMOID 1
#define ORC_FR 2           /* Fruchterman-Reingold (Table "diffmodels") */
#define ORC_LINLOG 3
#define ORC_FORCEATLAS 4

#define ORC_T2_FLOOR 1e-8
#define ORC_SIGMOID_BOUND 4.0

/* OpenMP thread count used by the parallel loops (n <= 0: leave as is). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    const uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;  /* golden ratio */
            k[1] += 0xBB67AE85u;  /* sqrt(3) - 1 */
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

static uint32_t philox_x0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ------------------------------------------------------------------ */
/* Initial embedding and negative samples                              */
/* ------------------------------------------------------------------ */

double orc_init_value(uint64_t seed, uint32_t i, uint32_t j)
{
    const uint32_t x = philox_x0(seed, i, j, 0xFFFFu, 0u);
    return ldexp((double)(x >> 8), -24) - 0.5;
}

void orc_init_embedding(int64_t n, int32_t d, uint64_t seed, double *Z)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < d; ++j)
            Z[i * d + j] = orc_init_value(seed, (uint32_t)i, (uint32_t)j);
}

uint32_t orc_sample(uint64_t seed, uint32_t u, uint32_t epoch, uint32_t k, uint32_t n)
{
    return philox_x0(seed, u, epoch, k, 0u) % n;
}

uint32_t orc_sample_shared(uint64_t seed, uint32_t k, uint32_t epoch, uint32_t j, uint32_t n)
{
    return philox_x0(seed, k, epoch, j, 2u) % n;
}

void orc_samples(uint64_t seed, int64_t n, int32_t s, int32_t epoch, int32_t *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u)
        for (int32_t k = 0; k < s; ++k)
            out[u * s + k] = (int32_t)orc_sample(seed, (uint32_t)u, (uint32_t)epoch,
                                                 (uint32_t)k, (uint32_t)n);
}

/*
 * Algorithm 3 (GenWalk) for vertex u in epoch e: out[i] is the vertex step i
 * reaches, or -1 once the walk has stopped (no neighbours to move to).
 */
void orc_walk(uint64_t seed, const int32_t *row_ptr, const int32_t *col_idx, int64_t u,
              int32_t epoch, int32_t k, int32_t *out)
{
    int64_t w = u;                      /* w <- u */
    int stopped = 0;
    for (int32_t i = 0; i < k; ++i) {   /* while |N(u)| < k */
        out[i] = -1;
        if (stopped) continue;
        const int32_t lo = row_ptr[w];
        const int32_t deg = row_ptr[w + 1] - lo;
        if (deg == 0) {
            stopped = 1;
            continue;
        }
        /* w_next <- a random neighbour of w; N(u) <- N(u) + {w_next}; w <- w_next */
        const uint32_t x = philox_x0(seed, (uint32_t)u, (uint32_t)epoch, (uint32_t)i, 1u);
        w = col_idx[lo + (int32_t)(x % (uint32_t)deg)];
        out[i] = (int32_t)w;
    }
}

/* ------------------------------------------------------------------ */
/* Per-pair gradient terms (added into g)                              */
/* ------------------------------------------------------------------ */

static double sigma(double x) { return 1.0 / (1.0 + exp(-x)); }

static double dot(const double *a, const double *b, int32_t d)
{
    double acc = 0.0;
    for (int32_t j = 0; j < d; ++j) acc += a[j] * b[j];
    return acc;
}

static double dist(const double *a, const double *b, int32_t d)
{
    double acc = 0.0;
    for (int32_t j = 0; j < d; ++j) acc += (a[j] - b[j]) * (a[j] - b[j]);
    return sqrt(acc);
}

/*
 * Error scale of the tests (only when gabs is not NULL): for each pair the
 * term is c(r) * x_j, where r is a reduced scalar (dot product or squared
 * distance), c the force coefficient and x the partner row (sigmoid) or the
 * difference z_u - z_v (t model).  Evaluated in finite precision, r carries
 * an error proportional to r_abs (the same reduction over absolute values),
 * so the term's first-order error is proportional to
 *     (|c| + |dc/dr| * r_abs) * |x_j|,
 * which is what gabs accumulates.
 */
static void add_scale(double *gabs, const double *x, int32_t d, double c, double dc, double r_abs)
{
    if (!gabs) return;
    const double w = fabs(c) + fabs(dc) * r_abs;
    for (int32_t j = 0; j < d; ++j) gabs[j] += w * fabs(x[j]);
}

static double dot_abs(const double *a, const double *b, int32_t d)
{
    double acc = 0.0;
    for (int32_t j = 0; j < d; ++j) acc += fabs(a[j] * b[j]);
    return acc;
}

/* attractive: grad of f_a(u,v) with respect to z_u */
static void attractive_grad(int model, const double *zu, const double *zv, int32_t d, double *g,
                            double *gabs)
{
    if (model == ORC_SIGMOID) {
        /* Eq. 5: -(1 - sigma(z_u . z_v)) z_v */
        const double x = dot(zu, zv, d);
        const double c = -(1.0 - sigma(x));
        for (int32_t j = 0; j < d; ++j) g[j] += c * zv[j];
        if (gabs) add_scale(gabs, zv, d, c, sigma(x) * (1.0 - sigma(x)), dot_abs(zu, zv, d));
    } else if (model != ORC_TDIST) {
        /* Table "diffmodels": minus the listed force times the unit vector */
        const double t = dist(zu, zv, d);
        if (t == 0.0) return;                 /* the force vanishes with t */
        double scal, c, dc;                   /* c = scal / t; dc = dc/d(t^2) */
        if (model == ORC_FR) {
            scal = t * t;
            c = t;
            dc = 1.0 / (2.0 * t);
        } else if (model == ORC_LINLOG) {
            scal = log(1.0 + t);
            c = scal / t;
            dc = (t / (1.0 + t) - scal) / (2.0 * t * t * t);
        } else {                              /* ForceAtlas */
            scal = t;
            c = 1.0;
            dc = 0.0;
        }
        for (int32_t j = 0; j < d; ++j) g[j] += scal * (zu[j] - zv[j]) / t;
        if (gabs) {
            double df[d];
            for (int32_t j = 0; j < d; ++j) df[j] = zu[j] - zv[j];
            add_scale(gabs, df, d, c, dc, t * t);
        }
    } else {
        /* Eq. 8: 2t / (1 + t^2), times the unit vector (z_u - z_v)/t (Sec. III-B) */
        const double t = dist(zu, zv, d);
        if (t == 0.0) return;                 /* the force vanishes with t */
        const double scal = 2.0 * t / (1.0 + t * t);
        for (int32_t j = 0; j < d; ++j) g[j] += scal * (zu[j] - zv[j]) / t;
        if (gabs) {
            double df[d];
            for (int32_t j = 0; j < d; ++j) df[j] = zu[j] - zv[j];
            const double q = t * t;
            add_scale(gabs, df, d, 2.0 / (1.0 + q), 2.0 / ((1.0 + q) * (1.0 + q)), q);
        }
    }
}

/* repulsive: grad of f_r(u,w) with respect to z_u */
static void repulsive_grad(int model, const double *zu, const double *zw, int32_t d, double *g,
                           double *gabs)
{
    if (model == ORC_SIGMOID) {
        /* Eq. 6: sigma(z_u . z_w) z_w */
        const double x = dot(zu, zw, d);
        const double c = sigma(x);
        for (int32_t j = 0; j < d; ++j) g[j] += c * zw[j];
        if (gabs) add_scale(gabs, zw, d, c, sigma(x) * (1.0 - sigma(x)), dot_abs(zu, zw, d));
    } else if (model != ORC_TDIST) {
        /* Table "diffmodels", all three models: minus the force 1/t times
           the unit vector, with t^2 floored at 1e-8 */
        double t = dist(zu, zw, d);
        double t2 = t * t;
        if (t2 < ORC_T2_FLOOR) { t2 = ORC_T2_FLOOR; t = sqrt(t2); }
        const double scal = -1.0 / t;
        for (int32_t j = 0; j < d; ++j) g[j] += scal * (zu[j] - zw[j]) / t;
        if (gabs) {
            double df[d];
            for (int32_t j = 0; j < d; ++j) df[j] = zu[j] - zw[j];
            add_scale(gabs, df, d, 1.0 / t2, 1.0 / (t2 * t2), t2);
        }
    } else {
        /* Eq. 9: -2 / (t (1 + t^2)), times the unit vector (z_u - z_w)/t,
           with t^2 floored at 1e-8 */
        double t = dist(zu, zw, d);
        double t2 = t * t;
        if (t2 < ORC_T2_FLOOR) { t2 = ORC_T2_FLOOR; t = sqrt(t2); }
        const double scal = -2.0 / (t * (1.0 + t2));
        for (int32_t j = 0; j < d; ++j) g[j] += scal * (zu[j] - zw[j]) / t;
        if (gabs) {
            double df[d];
            for (int32_t j = 0; j < d; ++j) df[j] = zu[j] - zw[j];
            const double dc = 2.0 * (1.0 + 2.0 * t2) / (t2 * t2 * (1.0 + t2) * (1.0 + t2));
            add_scale(gabs, df, d, 2.0 / (t2 * (1.0 + t2)), dc, t2);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: GradMinibatch                                          */
/* ------------------------------------------------------------------ */

/*
 * grad[(u - u_begin) * d + j] receives the gradient of vertex u for
 * u in [u_begin, u_end).  The negative samples of u are either drawn from
 * Philox (samp_ptr == NULL) or read from samp_idx[samp_ptr[u]..samp_ptr[u+1])
 * (an injected S(u), used by the tests).  A sample equal to u is skipped.
 * If grad_abs is not NULL it receives the sum of the absolute values of the
 * per-pair terms, element by element.  If Zp is not NULL, partner rows
 * (neighbours and samples) are read from Zp and only z_u from Z: the
 * storage form that keeps partner rows in reduced precision beside a full
 * precision copy of each vertex's own row.
 */
/*
 * Algorithm 2 for the `count` vertices vlist[0..count) (vlist == NULL: the
 * range u_begin, u_begin + 1, ...); row i of grad is vertex i's gradient.
 * walk > 0: N(u) is the walk of Algorithm 3 (rForce2Vec) instead of the
 * neighbours of u.  shared_k >= 0: the samples are the shared set S_b of
 * minibatch shared_k (orc_sample_shared) instead of u's own; shared_k ==
 * -2: the shared set of minibatch u / shared_b.
 */
void orc_grad_core(int model, int64_t n, int32_t d, const int32_t *row_ptr,
                   const int32_t *col_idx, const double *Z, const double *Zp,
                   const int64_t *vlist, int64_t u_begin, int64_t count, int32_t s, int32_t walk,
                   int64_t shared_k, int64_t shared_b, uint64_t seed, int32_t epoch,
                   const int64_t *samp_ptr, const int32_t *samp_idx, double *grad,
                   double *grad_abs)
{
    if (Zp == NULL) Zp = Z;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < count; ++i) {
        const int64_t u = vlist ? vlist[i] : u_begin + i;
        const double *zu = Z + u * d;
        double ga[d], gr[d];            /* grad f_a(u), grad f_r(u) */
        double *gabs = grad_abs ? grad_abs + i * d : NULL;
        memset(ga, 0, sizeof ga);
        memset(gr, 0, sizeof gr);
        if (gabs) memset(gabs, 0, sizeof(double) * (size_t)d);
        if (walk > 0) {
            int32_t nw[walk];
            orc_walk(seed, row_ptr, col_idx, u, epoch, walk, nw);
            for (int32_t j = 0; j < walk; ++j) {
                if (nw[j] < 0 || nw[j] == u) continue;
                attractive_grad(model, zu, Zp + (int64_t)nw[j] * d, d, ga, gabs);
            }
        } else {
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                const int32_t v = col_idx[e];
                attractive_grad(model, zu, Zp + (int64_t)v * d, d, ga, gabs);
            }
        }
        if (samp_ptr == NULL) {
            const int64_t kb = (shared_k == -2) ? u / shared_b : shared_k;
            for (int32_t k = 0; k < s; ++k) {
                const int64_t w =
                    kb >= 0 ? orc_sample_shared(seed, (uint32_t)kb, (uint32_t)epoch, (uint32_t)k,
                                                (uint32_t)n)
                            : orc_sample(seed, (uint32_t)u, (uint32_t)epoch, (uint32_t)k,
                                         (uint32_t)n);
                if (w == u) continue;
                repulsive_grad(model, zu, Zp + w * d, d, gr, gabs);
            }
        } else {
            for (int64_t p = samp_ptr[u]; p < samp_ptr[u + 1]; ++p) {
                const int64_t w = samp_idx[p];
                if (w == u) continue;
                repulsive_grad(model, zu, Zp + w * d, d, gr, gabs);
            }
        }
        double *gu = grad + i * d;
        for (int32_t j = 0; j < d; ++j) gu[j] = ga[j] + gr[j];
    }
}

/* walk > 0: N(u) is the walk of Algorithm 3 (rForce2Vec) instead of the
   neighbours of u.  shared_b > 0: the samples of u are the set S_b of its
   minibatch k = u / shared_b (orc_sample_shared) instead of its own. */
void orc_grad_minibatch_ex(int model, int64_t n, int32_t d,
                           const int32_t *row_ptr, const int32_t *col_idx,
                           const double *Z, const double *Zp, int64_t u_begin,
                           int64_t u_end, int32_t s, int32_t walk, int64_t shared_b,
                           uint64_t seed, int32_t epoch, const int64_t *samp_ptr,
                           const int32_t *samp_idx, double *grad, double *grad_abs)
{
    orc_grad_core(model, n, d, row_ptr, col_idx, Z, Zp, NULL, u_begin, u_end - u_begin, s,
                  walk, shared_b > 0 ? -2 : -1, shared_b, seed, epoch, samp_ptr, samp_idx, grad,
                  grad_abs);
}

void orc_grad_minibatch_abs(int model, int64_t n, int32_t d,
                            const int32_t *row_ptr, const int32_t *col_idx,
                            const double *Z, const double *Zp, int64_t u_begin, int64_t u_end,
                            int32_t s, uint64_t seed, int32_t epoch,
                            const int64_t *samp_ptr, const int32_t *samp_idx,
                            double *grad, double *grad_abs)
{
    orc_grad_minibatch_ex(model, n, d, row_ptr, col_idx, Z, Zp, u_begin, u_end, s, 0, 0, seed,
                          epoch, samp_ptr, samp_idx, grad, grad_abs);
}

void orc_grad_minibatch(int model, int64_t n, int32_t d,
                        const int32_t *row_ptr, const int32_t *col_idx,
                        const double *Z, int64_t u_begin, int64_t u_end,
                        int32_t s, uint64_t seed, int32_t epoch,
                        const int64_t *samp_ptr, const int32_t *samp_idx,
                        double *grad)
{
    orc_grad_minibatch_abs(model, n, d, row_ptr, col_idx, Z, NULL, u_begin, u_end, s, seed,
                           epoch, samp_ptr, samp_idx, grad, NULL);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1                                                          */
/* ------------------------------------------------------------------ */

/*
 * The random partition of epoch e (the partition step of Alg. 1: random
 * minibatches, no vertex in two of them): perm lists the vertices in increasing order of the key
 * Philox(key, ctr=(v, e, 0, 3)).x0, ties by id; minibatch k is
 * perm[k b .. min((k+1) b, n)).
 */
typedef struct {
    uint32_t key;
    int64_t v;
} orc_keyed;

static int cmp_keyed(const void *a, const void *b)
{
    const orc_keyed *x = (const orc_keyed *)a, *y = (const orc_keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

int orc_partition(uint64_t seed, int64_t n, int32_t epoch, int64_t *perm)
{
    orc_keyed *t = (orc_keyed *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_keyed));
    if (!t) return -1;
    for (int64_t v = 0; v < n; ++v) {
        t[v].key = philox_x0(seed, (uint32_t)v, (uint32_t)epoch, 0u, 3u);
        t[v].v = v;
    }
    qsort(t, (size_t)n, sizeof(orc_keyed), cmp_keyed);
    for (int64_t i = 0; i < n; ++i) perm[i] = t[i].v;
    free(t);
    return 0;
}

double orc_learning_rate(double lr0, int32_t schedule, int32_t total_epochs, int32_t epoch)
{
    if (schedule == 1 && total_epochs > 0)
        return lr0 * (1.0 - (double)epoch / (double)total_epochs);
    return lr0;
}

/*
 * Runs epochs [start_epoch, start_epoch + epochs) of Algorithm 1 on Z in
 * place.  max_minibatches < 0 runs every minibatch of each epoch; otherwise
 * only the first max_minibatches of each epoch (used to time a bounded
 * sample of a large epoch).  walk > 0: rForce2Vec, N(u) from Algorithm 3;
 * shared != 0: one sample set S_b per minibatch; partition != 0: a new
 * random partition every epoch (orc_partition) instead of the id ranges
 * [k b, (k+1) b) (orc_train is none of these).
 * Returns 0, or -1 if memory ran out.
 */
int orc_train_ex(int model, int64_t n, int32_t d,
                 const int32_t *row_ptr, const int32_t *col_idx,
                 double *Z, int32_t s, int32_t walk, int32_t shared, int32_t partition,
                 int64_t b, uint64_t seed, double lr0, int32_t schedule, int32_t total_epochs,
                 int32_t start_epoch, int32_t epochs, int64_t max_minibatches,
                 const int64_t *samp_ptr, const int32_t *samp_idx)
{
    double *grad = (double *)malloc((size_t)b * (size_t)d * sizeof(double));
    int64_t *perm = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!grad || !perm) {
        free(grad);
        free(perm);
        return -1;
    }
    for (int32_t e = start_epoch; e < start_epoch + epochs; ++e) {
        const double eta = orc_learning_rate(lr0, schedule, total_epochs, e);
        /* the minibatches of this epoch */
        if (partition) {
            if (orc_partition(seed, n, e, perm) != 0) {
                free(grad);
                free(perm);
                return -1;
            }
        } else {
            for (int64_t i = 0; i < n; ++i) perm[i] = i;
        }
        int64_t nmb = 0;
        for (int64_t p0 = 0; p0 < n; p0 += b) {          /* each minibatch V_b */
            if (max_minibatches >= 0 && nmb >= max_minibatches) break;
            const int64_t k = nmb++;
            const int64_t p1 = (p0 + b < n) ? p0 + b : n;
            orc_grad_core(model, n, d, row_ptr, col_idx, Z, NULL, perm + p0, 0, p1 - p0, s,
                          walk, shared ? k : -1, b, seed, e, samp_ptr, samp_idx, grad, NULL);
            for (int64_t i = p0; i < p1; ++i)            /* Eq. 10 */
                for (int32_t j = 0; j < d; ++j) {
                    const int64_t u = perm[i];
                    double z = Z[u * d + j] - eta * grad[(i - p0) * d + j];
                    if (model != ORC_TDIST) {                /* bounded coordinates */
                        if (z > ORC_SIGMOID_BOUND) z = ORC_SIGMOID_BOUND;
                        if (z < -ORC_SIGMOID_BOUND) z = -ORC_SIGMOID_BOUND;
                    }
                    Z[u * d + j] = z;
                }
        }
    }
    free(grad);
    free(perm);
    return 0;
}

int orc_train(int model, int64_t n, int32_t d,
              const int32_t *row_ptr, const int32_t *col_idx,
              double *Z, int32_t s, int64_t b, uint64_t seed,
              double lr0, int32_t schedule, int32_t total_epochs,
              int32_t start_epoch, int32_t epochs, int64_t max_minibatches,
              const int64_t *samp_ptr, const int32_t *samp_idx)
{
    return orc_train_ex(model, n, d, row_ptr, col_idx, Z, s, 0, 0, 0, b, seed, lr0, schedule,
                        total_epochs, start_epoch, epochs, max_minibatches, samp_ptr, samp_idx);
}

/* ------------------------------------------------------------------ */
/* Loss (Eq. 2 with Eq. 3 / Eq. 7) and evaluation                       */
/* ------------------------------------------------------------------ */

/* log(1 + e^y), written so that e^y cannot overflow: for y > 0 it is
   y + log(1 + e^-y).  (With coordinates bounded by 4 and d = 128 a dot
   product reaches 2048, where e^y is infinite in FP64.) */
static double log1p_exp(double y)
{
    return y > 0.0 ? y + log1p(exp(-y)) : log1p(exp(y));
}

/* -log delta(z_u, z_v) for a neighbour v */
static double attractive_loss(int model, const double *zu, const double *zv, int32_t d)
{
    if (model == ORC_SIGMOID) {
        const double x = dot(zu, zv, d);
        return log1p_exp(-x);                           /* Eq. 3, first sum: -log sigma(x) */
    }
    const double t = dist(zu, zv, d);
    return log(1.0 + t * t);                            /* Eq. 7, first sum */
}

/* -log(1 - delta(z_u, z_w)) for a negative sample w */
static double repulsive_loss(int model, const double *zu, const double *zw, int32_t d)
{
    if (model == ORC_SIGMOID) {
        const double x = dot(zu, zw, d);
        return log1p_exp(x);                            /* Eq. 3, second sum: -log(1 - sigma(x)) */
    }
    const double t = dist(zu, zw, d);
    double t2 = t * t;
    if (t2 < ORC_T2_FLOOR) t2 = ORC_T2_FLOOR;
    return -log(t2 / (1.0 + t2));                       /* Eq. 7, second sum */
}

/* L(u) of Eq. 2 for one vertex, with the same sample rule as orc_grad_minibatch */
double orc_loss_vertex(int model, int64_t n, int32_t d,
                       const int32_t *row_ptr, const int32_t *col_idx,
                       const double *Z, int64_t u, int32_t s, uint64_t seed, int32_t epoch,
                       const int64_t *samp_ptr, const int32_t *samp_idx)
{
    const double *zu = Z + u * d;
    double L = 0.0;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        L += attractive_loss(model, zu, Z + (int64_t)col_idx[e] * d, d);
    if (samp_ptr == NULL) {
        for (int32_t k = 0; k < s; ++k) {
            const int64_t w = orc_sample(seed, (uint32_t)u, (uint32_t)epoch, (uint32_t)k,
                                         (uint32_t)n);
            if (w == u) continue;
            L += repulsive_loss(model, zu, Z + w * d, d);
        }
    } else {
        for (int64_t p = samp_ptr[u]; p < samp_ptr[u + 1]; ++p) {
            if (samp_idx[p] == u) continue;
            L += repulsive_loss(model, zu, Z + (int64_t)samp_idx[p] * d, d);
        }
    }
    return L;
}

/* sum of L(u) over all vertices */
double orc_loss_total(int model, int64_t n, int32_t d,
                      const int32_t *row_ptr, const int32_t *col_idx,
                      const double *Z, int32_t s, uint64_t seed, int32_t epoch,
                      const int64_t *samp_ptr, const int32_t *samp_idx)
{
    double total = 0.0;
    #pragma omp parallel for reduction(+:total) schedule(dynamic, 64)
    for (int64_t u = 0; u < n; ++u)
        total += orc_loss_vertex(model, n, d, row_ptr, col_idx, Z, u, s, seed, epoch,
                                 samp_ptr, samp_idx);
    return total;
}

/*
 * Link-prediction score of a pair: a larger score means "more likely an
 * edge".  Sigmoid model: z_u . z_v; t model: -||z_u - z_v||^2 (both monotone
 * in the model's similarity delta).
 */
void orc_scores(int model, int32_t d, const double *Z, const int32_t *pairs, int64_t npairs,
                double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npairs; ++i) {
        const double *a = Z + (int64_t)pairs[2 * i] * d;
        const double *b = Z + (int64_t)pairs[2 * i + 1] * d;
        if (model == ORC_SIGMOID) {
            out[i] = dot(a, b, d);
        } else {
            const double t = dist(a, b, d);
            out[i] = -(t * t);
        }
    }
}

static int cmp_double(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Mann-Whitney U / (P N): probability that a positive outscores a negative,
   ties counted one half.  Sorts neg in place. */
double orc_auc(const double *pos, int64_t npos, double *neg, int64_t nneg)
{
    if (npos <= 0 || nneg <= 0) return NAN;
    qsort(neg, (size_t)nneg, sizeof(double), cmp_double);
    double twice_u = 0.0;   /* counts are integers; exact in double up to 2^53 */
    for (int64_t i = 0; i < npos; ++i) {
        /* lo = #neg < pos[i], hi = #neg <= pos[i] */
        int64_t lo = 0, hi = nneg;
        while (lo < hi) { int64_t m = (lo + hi) / 2; if (neg[m] < pos[i]) lo = m + 1; else hi = m; }
        int64_t lo2 = lo, hi2 = nneg;
        while (lo2 < hi2) { int64_t m = (lo2 + hi2) / 2; if (neg[m] <= pos[i]) lo2 = m + 1; else hi2 = m; }
        twice_u += 2.0 * (double)lo + (double)(lo2 - lo);
    }
    return twice_u / (2.0 * (double)npos * (double)nneg);
}
